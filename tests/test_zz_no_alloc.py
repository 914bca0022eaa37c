"""bp_decode_noalloc: the decoder entry point for callers that cannot
allocate device memory while they decode (pipelines that allocate everything
up front because cudaMalloc synchronises the device, or hosts whose device
memory belongs to another allocator).  Its scratch is a fixed device array
inside the library, so its results must equal bp_decode's with a caller
workspace, on consecutive calls that reuse that array.

This file sorts last so that a run stopping at the first failure has run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_1911_08868_gb300 import inputs

from conftest import gpu_device

pytestmark = pytest.mark.gpu


def test_noalloc_matches_bp_decode_on_consecutive_calls(pcbp, oracle):
    import torch

    dev = gpu_device()
    N, K, r, poly, B, max_iters = 1024, 512, 24, 0x1B2B117, 3000, 300
    _, fr = oracle.construct(N, K)
    pay = inputs.payload_numpy(404, B, K - r)
    x = oracle.encode_frames(pay, fr, r, poly)
    llr = torch.from_numpy(
        inputs.bpsk_awgn_llr(x, inputs.noise_numpy(404, B, N), inputs.sigma2_of(2.5, K, r, N))).to(dev)
    code = pcbp.pc_construct(N, K, r, poly)
    sch = pcbp.sched(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10, seed=5, stop_kind=1)

    def outputs():
        return (torch.full((B, pcbp.words_of(K)), -1, dtype=torch.int32, device=dev),
                torch.full((B,), -1, dtype=torch.int32, device=dev),
                torch.full((B,), 7, dtype=torch.uint8, device=dev))

    ref = outputs()
    ws = torch.zeros(pcbp.bp_decode_workspace_size(code, B), dtype=torch.uint8, device=dev)
    pcbp.bp_decode(code, llr, sch, max_iters, *ref, ws)
    for call in range(2):          # the second call finds the first call's counter in the array
        got = outputs()
        pcbp.bp_decode_noalloc(code, llr, sch, max_iters, *got)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b), f"call {call}"
    assert int(ref[1].min()) >= 1 and (ref[1] < max_iters).any()


def test_noalloc_rejects_bad_arguments_like_bp_decode(pcbp):
    import torch

    dev = gpu_device()
    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    z = torch.zeros((4, 256), dtype=torch.float32, device=dev)
    o = torch.zeros((4, 4), dtype=torch.int32, device=dev)
    with pytest.raises(pcbp.PcError) as e:
        pcbp.bp_decode_noalloc(code, z, pcbp.sched(mode=1, P_range=9, P_level=5, N_min=5, T0=5), 10,
                               o, o[:, 0], o[:, 0].to(torch.uint8))
    assert e.value.status == pcbp.PC_EINVAL
    assert pcbp.bp_decode_workspace_size(code, 1 << 30) <= pcbp.PC_STATIC_SCRATCH_BYTES
