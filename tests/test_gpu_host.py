"""bp_decode_host: the decoder reading page-locked host LLRs and writing its
results into page-locked host memory in place.  Its outputs must equal the
oracle's and bp_decode's bit for bit, for both decoder kernels (N < 128: the
shared-memory kernel; N >= 128: the tensor-memory kernel), and buffers the
device cannot address must be refused before anything runs."""
import numpy as np
import pytest

from conftest import gpu_device
from test_gpu_parity import POLY8, POLY24, frames, oracle_outputs, osched

pytestmark = pytest.mark.gpu

CASES = [
    (64, 32, 8, POLY8, 2.5, dict(mode=1, rho_range_fixed=3, P_level=5, N_min=5, T0=5), 60, 400),
    (128, 64, 8, POLY8, 2.5, dict(mode=1, rho_range_fixed=3, P_level=6, N_min=5, T0=5), 60, 400),
    (1024, 512, 24, POLY24, 2.5, dict(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10), 300, 300),
]


def host_outputs(pcbp, code, B, pinned=True):
    import torch

    return (torch.full((B, pcbp.words_of(code.K)), -1, dtype=torch.int32).pin_memory() if pinned
            else torch.full((B, pcbp.words_of(code.K)), -1, dtype=torch.int32),
            torch.full((B,), -7, dtype=torch.int32).pin_memory() if pinned else torch.full((B,), -7, dtype=torch.int32),
            torch.full((B,), 9, dtype=torch.uint8).pin_memory() if pinned else torch.full((B,), 9, dtype=torch.uint8))


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c[0]}")
def test_host_buffers_decode_like_the_oracle_and_bp_decode(pcbp, oracle, case):
    import torch

    dev = gpu_device()
    N, K, r, poly, ebn0, kw, max_iters, B = case
    fr, pay, x, llr = frames(oracle, N, K, r, poly, B, ebn0, seed=N * 11 + 3)
    s = pcbp.sched(**{"seed": 777, "stop_kind": 1, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    h_llr = torch.from_numpy(np.ascontiguousarray(llr)).pin_memory()
    hb, hi, ho = host_outputs(pcbp, code, B)
    ws = torch.zeros(pcbp.bp_decode_workspace_size(code, B), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    pcbp.bp_decode_host(code, h_llr, s, max_iters, hb, hi, ho, ws, stream)
    stream.synchronize()
    rbits, riters, rok = oracle_outputs(oracle, fr, r, poly, llr, osched(oracle, s), max_iters)
    assert np.array_equal(hi.numpy(), riters)
    assert np.array_equal(ho.numpy(), rok)
    assert np.array_equal(pcbp.unpack_bits(hb, K).numpy(), rbits)
    # the same frames through bp_decode on device buffers
    d_out = tuple(t.to(dev) for t in host_outputs(pcbp, code, B, pinned=False))
    pcbp.bp_decode(code, h_llr.to(dev), s, max_iters, *d_out, ws)
    torch.cuda.synchronize()
    for h, d in zip((hb, hi, ho), d_out):
        assert torch.equal(h, d.cpu())
    assert (hi.numpy() < max_iters).any()


def test_host_entry_accepts_device_buffers(pcbp, oracle):
    import torch

    dev = gpu_device()
    N, K, r, poly, ebn0, kw, max_iters, B = CASES[1]
    fr, pay, x, llr = frames(oracle, N, K, r, poly, 64, ebn0, seed=91)
    s = pcbp.sched(**{"seed": 3, "stop_kind": 1, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    d_llr = torch.from_numpy(np.ascontiguousarray(llr)).to(dev)
    ws = torch.zeros(pcbp.bp_decode_workspace_size(code, 64), dtype=torch.uint8, device=dev)
    got = tuple(t.to(dev) for t in host_outputs(pcbp, code, 64, pinned=False))
    ref = tuple(t.to(dev) for t in host_outputs(pcbp, code, 64, pinned=False))
    pcbp.bp_decode_host(code, d_llr, s, max_iters, *got, ws)
    pcbp.bp_decode(code, d_llr, s, max_iters, *ref, ws)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_host_entry_refuses_pageable_memory(pcbp):
    """Ordinary (pageable) host tensors are not mapped into the device's
    address space: PC_EINVAL, and no output is touched."""
    import torch

    dev = gpu_device()
    code = pcbp.pc_construct(1024, 512, 24, POLY24)
    s = pcbp.sched(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10, stop_kind=1)
    ws = torch.zeros(pcbp.bp_decode_workspace_size(code, 8), dtype=torch.uint8, device=dev)
    pinned_llr = torch.zeros((8, 1024), dtype=torch.float32).pin_memory()
    pageable_llr = torch.zeros((8, 1024), dtype=torch.float32)
    for llr, pinned_out in ((pageable_llr, True), (pinned_llr, False)):
        hb, hi, ho = host_outputs(pcbp, code, 8, pinned=pinned_out)
        with pytest.raises(pcbp.PcError) as e:
            pcbp.bp_decode_host(code, llr, s, 10, hb, hi, ho, ws)
        assert e.value.status == pcbp.PC_EINVAL
        torch.cuda.synchronize()
        assert int(hi.min()) == -7 and int(hi.max()) == -7 and int(ho.min()) == 9


def test_host_decoder_matches_device_decoder(pcbp, oracle):
    import torch

    dev = gpu_device()
    N, K, r, poly, ebn0, kw, max_iters, B = CASES[1]
    fr, pay, x, llr = frames(oracle, N, K, r, poly, 500, ebn0, seed=5)
    s = pcbp.sched(**{"seed": 41, "stop_kind": 1, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    h_llr = torch.from_numpy(np.ascontiguousarray(llr)).pin_memory()
    hb, hi, ho = pcbp.HostDecoder(code, s, max_iters, dev)(h_llr)
    dec = pcbp.Decoder(code, s, max_iters, dev)
    dec(h_llr.to(dev))
    torch.cuda.synchronize()
    assert torch.equal(hb, dec.bits.cpu()) and torch.equal(hi, dec.iters.cpu()) and torch.equal(ho, dec.crc_ok.cpu())
    with pytest.raises(ValueError):
        pcbp.HostDecoder(code, s, max_iters, dev)(torch.from_numpy(np.ascontiguousarray(llr)))
