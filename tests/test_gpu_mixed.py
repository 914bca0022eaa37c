"""One persistent sweep over batches of different lengths and rates
(bp_decode_mixed): the results equal bp_decode on each batch alone (and the
oracle on sampled frames), directly and replayed from a CUDA graph."""
import numpy as np
import pytest

from paper_1911_08868_gb300 import inputs

from conftest import gpu_device

pytestmark = pytest.mark.gpu

POLY8, POLY24 = 0x9B, 0x1B2B117


def make_parts(pcbp, oracle, dev, sizes, B, seed, slots=0):
    import torch

    parts, refs = [], []
    for i, (N, rate) in enumerate(sizes):
        K = int(N * rate)
        r, poly = (8, POLY8) if N <= 256 else (24, POLY24)
        _, fr = oracle.construct(N, K)
        pay = inputs.payload_numpy(seed + i, B, K - r)
        x = oracle.encode_frames(pay, fr, r, poly)
        ebn0 = inputs.ebn0_numpy(seed + i, B, 1.0, 4.0)
        llr = inputs.bpsk_awgn_llr(x, inputs.noise_numpy(seed + i, B, N), inputs.sigma2_of(ebn0, K, r, N))
        code = pcbp.pc_construct(N, K, r, poly)
        n = N.bit_length() - 1
        sch = pcbp.sched(mode=1, rho_range_fixed=4, P_level=n - 1, N_min=10, T0=10, seed=100 + i, stop_kind=1)
        parts.append((code, sch, 300, torch.from_numpy(llr).to(dev), slots))
        refs.append((fr, r, poly, llr, sch))
    return parts, refs


def per_batch(pcbp, parts):
    import torch

    out = []
    for code, sch, max_iters, llr, *_ in parts:
        dec = pcbp.Decoder(code, sch, max_iters, llr.device)
        b, it, ok = dec(llr)
        out.append((b.clone(), it.clone(), ok.clone()))
    torch.cuda.synchronize()
    return out


SIZES = [(2048, 0.5), (1024, 0.75), (1024, 0.25), (512, 0.5), (256, 0.75), (128, 0.25), (128, 0.5), (256, 0.25)]


def test_mixed_matches_per_batch_and_oracle(pcbp, oracle):
    import torch

    dev = gpu_device()
    parts, refs = make_parts(pcbp, oracle, dev, SIZES, 700, seed=50)
    md = pcbp.MixedDecoder(parts, dev)
    bits, iters, ok = md()
    torch.cuda.synchronize()
    want = per_batch(pcbp, parts)
    for i in range(len(parts)):
        assert torch.equal(bits[i], want[i][0]), SIZES[i]
        assert torch.equal(iters[i], want[i][1]), SIZES[i]
        assert torch.equal(ok[i], want[i][2]), SIZES[i]
    # sampled frames against the oracle
    from test_gpu_parity import osched

    rng = np.random.default_rng(1)
    for i, (fr, r, poly, llr, sch) in enumerate(refs):
        K = parts[i][0].K
        got = pcbp.unpack_bits(bits[i], K).cpu().numpy()
        it = iters[i].cpu().numpy()
        for b in rng.choice(llr.shape[0], 6, replace=False):
            ref = oracle.decode(fr, r, poly, llr[b], osched(oracle, sch), 300, frame_id=int(b))
            assert it[b] == ref.iters and np.array_equal(got[b], oracle.info_bits(ref.uhat, fr))


def test_mixed_graph_replay_and_slot_override(pcbp, oracle):
    import torch

    dev = gpu_device()
    parts, _ = make_parts(pcbp, oracle, dev, SIZES[:5], 300, seed=77)
    md = pcbp.MixedDecoder(parts, dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        bits, iters, ok = md(s)                   # first call outside capture
    s.synchronize()
    first = [(b.clone(), i.clone(), o.clone()) for b, i, o in zip(bits, iters, ok)]
    for t in bits + iters + ok:
        t.fill_(0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        md(s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for k in range(len(parts)):
            assert torch.equal(md.bits[k], first[k][0]) and torch.equal(md.iters[k], first[k][1])
    one = [(p[0], p[1], p[2], p[3], 1) for p in parts]
    md1 = pcbp.MixedDecoder(one, dev)
    b1, i1, o1 = md1()
    torch.cuda.synchronize()
    for k in range(len(parts)):
        assert torch.equal(b1[k], first[k][0]) and torch.equal(i1[k], first[k][1]) and torch.equal(o1[k], first[k][2])


def test_mixed_box_plus_and_min_sum_batches(pcbp, oracle):
    """Box-plus and scaled min-sum batches in one sweep equal bp_decode on each."""
    import torch

    dev = gpu_device()
    parts, _ = make_parts(pcbp, oracle, dev, [(1024, 0.5), (256, 0.5), (128, 0.5)], 200, seed=91)
    bx = pcbp.sched(mode=1, rho_range_fixed=3, P_level=7, N_min=5, T0=5, seed=5, stop_kind=1, fkind=1)
    parts[1] = (parts[1][0], bx, 60, parts[1][3], 0)
    md = pcbp.MixedDecoder(parts, dev)
    bits, iters, ok = md()
    torch.cuda.synchronize()
    want = per_batch(pcbp, parts)
    for i in range(len(parts)):
        assert torch.equal(bits[i], want[i][0]) and torch.equal(iters[i], want[i][1])
        assert torch.equal(ok[i], want[i][2])


def test_mixed_threads_per_frame_choices_agree(pcbp, oracle, monkeypatch):
    """Both decoder kernels, chosen per batch by threads per frame (bp_kernel_threads; where the
    two counts coincide PCBP_DECODER=grouped picks the shared-memory kernel), give bp_decode's
    outputs."""
    import torch

    dev = gpu_device()
    sizes = [(2048, 0.5), (1024, 0.5), (512, 0.75), (256, 0.5), (128, 0.5)]
    parts, _ = make_parts(pcbp, oracle, dev, sizes, 250, seed=13)
    want = per_batch(pcbp, parts)
    for kernel in (0, 1):
        if kernel == 1:
            monkeypatch.setenv("PCBP_DECODER", "grouped")
        chosen = []
        for code, sch, max_iters, llr, slots in parts:
            chosen.append((code, sch, max_iters, llr, slots, pcbp.bp_kernel_threads(code, kernel)))
        md = pcbp.MixedDecoder(chosen, dev)
        bits, iters, ok = md()
        torch.cuda.synchronize()
        for i in range(len(parts)):
            assert torch.equal(bits[i], want[i][0]) and torch.equal(iters[i], want[i][1]), (sizes[i], kernel)
            assert torch.equal(ok[i], want[i][2])


def test_slot_limit_is_what_a_launch_uses(pcbp, oracle):
    """bp_slot_limit reports the frames-per-CTA count a batch asking for more is clamped to:
    a request at the limit and one above it decode alike, for both kernels."""
    import torch

    dev = gpu_device()
    sizes = [(1024, 0.5), (256, 0.5), (128, 0.5)]
    parts, _ = make_parts(pcbp, oracle, dev, sizes, 200, seed=29)
    for code, sch, max_iters, llr, _ in parts:
        N = code.N
        for tpf in sorted({t for t in (pcbp.bp_kernel_threads(code, k) for k in (0, 1)) if t}):
            lim = pcbp.bp_slot_limit(code, tpf, int(sch.fkind))
            assert 1 <= lim <= 1024 // tpf
            outs = []
            for slots in (lim, lim + 5):
                md = pcbp.MixedDecoder([(code, sch, max_iters, llr, slots, tpf)], dev)
                outs.append([t[0].clone() for t in md()])
            torch.cuda.synchronize()
            for a, b in zip(*outs):
                assert torch.equal(a, b), (N, tpf)
    with pytest.raises(pcbp.PcError) as e:
        pcbp.bp_slot_limit(parts[0][0], 96)
    assert e.value.status == pcbp.PC_EUNSUPPORTED


def test_all_lengths_rates_and_variants_in_one_table(pcbp, oracle):
    """Every TMEM length at three rates, with scaled min-sum and box-plus batches and the CRC,
    G-matrix and combined stops, in one table beside an N = 64 batch of the shared-memory kernel:
    every batch equals bp_decode alone."""
    import torch

    dev = gpu_device()
    sizes = [(N, R) for N in (2048, 1024, 512, 256, 128) for R in (0.25, 0.5, 0.75)] + [(64, 0.5)]
    parts, _ = make_parts(pcbp, oracle, dev, sizes, 160, seed=211)
    for i, (code, sch, max_iters, llr, slots) in enumerate(parts):
        n = code.n
        if i % 4 == 1:
            sch = pcbp.sched(mode=1, rho_range_fixed=3, P_level=n - 1, N_min=5, T0=5, seed=9 + i, stop_kind=1,
                             fkind=1)
            max_iters = 40
        elif i % 4 == 2:
            sch = pcbp.sched(mode=1, rho_range_fixed=4, P_level=n - 1, N_min=10, T0=10, seed=9 + i,
                             stop_kind=3, stop_from=2)
        elif i % 4 == 3:
            sch = pcbp.sched(mode=2, q_max=10, it_reset_full=30, seed=9 + i, stop_kind=2, stop_from=3, fkind=1)
            max_iters = 40
        parts[i] = (code, sch, max_iters, llr, slots)
    md = pcbp.MixedDecoder(parts, dev)
    bits, iters, ok = md()
    torch.cuda.synchronize()
    want = per_batch(pcbp, parts)
    for i in range(len(parts)):
        assert torch.equal(bits[i], want[i][0]), sizes[i]
        assert torch.equal(iters[i], want[i][1]), sizes[i]
        assert torch.equal(ok[i], want[i][2]), sizes[i]
