"""Parity of the CUDA decoder (through the C ABI) with the FP32 oracle.

Scaled min-sum fixes every operation's order and rounding, so the bar is
bit-exact: every message plane after every iteration (trace entry), and the
decided bits, iteration counts and CRC flags (production entry).  Inputs are
seeded synthetic BPSK/AWGN frames whose codewords come from the oracle's
encoder."""
import numpy as np
import pytest

from paper_1911_08868_gb300 import inputs

from conftest import gpu_device

pytestmark = pytest.mark.gpu

POLY8, POLY24 = 0x9B, 0x1B2B117


def frames(oracle, N, K, r, poly, B, ebn0, seed):
    _, fr = oracle.construct(N, K)
    pay = inputs.payload_numpy(seed, B, K - r)
    x = oracle.encode_frames(pay, fr, r, poly)
    llr = inputs.bpsk_awgn_llr(x, inputs.noise_numpy(seed, B, N), inputs.sigma2_of(ebn0, K, r, N))
    return fr, pay, x, llr


def osched(oracle, s):
    return oracle.Sched(mode=s.mode, P_range=s.P_range, P_level=s.P_level, N_min=s.N_min, D=s.D, T0=s.T0,
                        rho_range_fixed=s.rho_range_fixed, q_max=s.q_max, it_reset_full=s.it_reset_full,
                        stop_from=s.stop_from, stop_kind=s.stop_kind, fkind=s.fkind, alpha=float(np.float32(s.alpha)),
                        seed=s.seed, frame_base=s.frame_base)


def gpu_decode(pcbp, code, llr, s, max_iters, trace=False, events=None):
    import torch

    dev = gpu_device()
    B, N = llr.shape
    d_llr = torch.from_numpy(np.ascontiguousarray(llr)).to(dev)
    bits = torch.full((B, pcbp.words_of(code.K)), -1, dtype=torch.int32, device=dev)
    iters = torch.full((B,), -7, dtype=torch.int32, device=dev)
    ok = torch.full((B,), 9, dtype=torch.uint8, device=dev)
    ws = torch.zeros(pcbp.bp_decode_workspace_size(code, B), dtype=torch.uint8, device=dev)
    dump = None
    if trace:
        dump = torch.full((B, max(max_iters, 1), 2, code.n + 1, N), float("nan"), dtype=torch.float32, device=dev)
        pcbp.bp_decode_trace(code, d_llr, s, max_iters, events, dump, bits, iters, ok, ws)
    else:
        pcbp.bp_decode(code, d_llr, s, max_iters, bits, iters, ok, ws)
    torch.cuda.synchronize()
    out_bits = pcbp.unpack_bits(bits, code.K).cpu().numpy()
    return out_bits, iters.cpu().numpy(), ok.cpu().numpy(), None if dump is None else dump.cpu().numpy()


def assert_bitwise_equal(a, b, what):
    a32 = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    b32 = np.ascontiguousarray(b, dtype=np.float32).view(np.uint32)
    if not np.array_equal(a32, b32):
        idx = np.argwhere(a32 != b32)[0]
        raise AssertionError(f"{what}: first mismatch at {tuple(idx)}: gpu {a[tuple(idx)]!r} oracle {b[tuple(idx)]!r}")


def oracle_outputs(oracle, fr, r, poly, llr, os_, max_iters):
    u, it, ok = oracle.decode_batch(fr, r, poly, llr, os_, max_iters)
    return oracle.info_bits(u, fr), it, ok


# --------------------------------------------------------------------------- encoder
@pytest.mark.parametrize("N,K,r,poly", [(8, 4, 0, 0), (64, 40, 8, POLY8), (256, 128, 8, POLY8),
                                        (1024, 512, 24, POLY24), (2048, 1024, 24, POLY24), (128, 96, 32, 0x104C11DB7)])
def test_encode_matches_oracle(pcbp, oracle, N, K, r, poly):
    import torch

    dev = gpu_device()
    code = pcbp.pc_construct(N, K, r, poly)
    B = 77
    pay = inputs.payload_numpy(N + K, B, K - r)
    d_pay = torch.from_numpy(pay).to(dev)
    d_x = torch.full((B, N), 7, dtype=torch.uint8, device=dev)
    pcbp.pc_encode(code, d_pay, d_x)
    torch.cuda.synchronize()
    _, fr = oracle.construct(N, K)
    assert np.array_equal(d_x.cpu().numpy(), oracle.encode_frames(pay, fr, r, poly))


# --------------------------------------------------------------------------- every plane, every iteration
TRACE_CASES = [
    # N, K, r, poly, ebn0, sched kwargs, max_iters
    (8, 4, 0, 0, 1.0, dict(mode=1, P_range=2, P_level=2, N_min=2, T0=2, stop_kind=0), 12),
    (16, 8, 0, 0, 1.5, dict(mode=1, P_range=4, P_level=3, N_min=3, D=2, T0=1, stop_kind=2), 20),
    (64, 32, 8, POLY8, 2.0, dict(mode=1, P_range=5, P_level=5, N_min=2, D=8, T0=3, stop_kind=1, stop_from=4), 30),
    (64, 40, 0, 0, 2.0, dict(mode=2, it_reset_full=4, q_max=5, stop_kind=3), 30),
    (256, 128, 8, POLY8, 2.0, dict(mode=1, rho_range_fixed=4, P_level=7, N_min=5, T0=5, stop_kind=1), 25),
    (256, 128, 8, POLY8, 2.0, dict(mode=0, stop_kind=1, alpha=1.0), 25),
    (512, 256, 24, POLY24, 2.0, dict(mode=1, P_range=9, P_level=8, N_min=4, D=50, T0=6, stop_kind=1), 20),
]


@pytest.mark.parametrize("case", TRACE_CASES, ids=lambda c: f"N{c[0]}-mode{c[5]['mode']}")
def test_trace_every_plane_bit_exact(pcbp, oracle, case):
    N, K, r, poly, ebn0, kw, max_iters = case
    B = 37
    fr, pay, x, llr = frames(oracle, N, K, r, poly, B, ebn0, seed=N + 3)
    s = pcbp.sched(**{"seed": 77, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    bits, iters, ok, dump = gpu_decode(pcbp, code, llr, s, max_iters, trace=True)
    os_ = osched(oracle, s)
    switched = 0
    for b in range(B):
        ref = oracle.decode(fr, r, poly, llr[b], os_, max_iters, frame_id=b, dump=True)
        assert iters[b] == ref.iters, f"frame {b}"
        assert ok[b] == ref.crc_ok, f"frame {b}"
        assert np.array_equal(bits[b], oracle.info_bits(ref.uhat, fr)), f"frame {b}"
        assert_bitwise_equal(dump[b, : ref.iters], ref.dump[: ref.iters], f"frame {b} planes")
        first_switch = kw.get("T0", 1) if kw["mode"] == 1 else kw.get("it_reset_full", 10 ** 9)
        switched += ref.iters > first_switch
    if kw["mode"]:
        assert switched > 0   # the case exercises at least one switch


def test_trace_explicit_events_bit_exact(pcbp, oracle):
    """The k-th switch applies the k-th given event, e.g. Fig. 3's N = 8,
    rho_range = 2, rho_level = 1 subgraph and subgraphs that revert."""
    N, K = 64, 32
    fr, pay, x, llr = frames(oracle, N, K, 0, 0, 9, 1.0, seed=5)
    evs = [(1, 2, 3, [1, 0]), (2, 3, 1, [2, 0, 1]), (1, 6, 0, [5, 4, 3, 2, 1, 0]), (4, 3, 0, [1, 2, 0]),
           (3, 2, 3, [1, 0])]
    s = pcbp.sched(mode=1, P_range=2, P_level=1, N_min=2, T0=1, stop_kind=0)
    code = pcbp.pc_construct(N, K)
    bits, iters, ok, dump = gpu_decode(pcbp, code, llr, s, 14, trace=True, events=[pcbp.event(*e) for e in evs])
    oevs = [oracle.Event.make(*e) for e in evs]
    for b in range(len(llr)):
        ref = oracle.decode(fr, 0, 0, llr[b], osched(oracle, s), 14, frame_id=b, events=oevs, dump=True)
        assert iters[b] == ref.iters == 14
        assert_bitwise_equal(dump[b], ref.dump, f"frame {b}")


# --------------------------------------------------------------------------- production entry
DECODE_CASES = [
    (128, 64, 8, POLY8, 2.5, dict(mode=1, rho_range_fixed=3, P_level=6, N_min=5, T0=5), 60, 400),
    (256, 128, 8, POLY8, 3.0, dict(mode=0), 50, 2000),                  # the N = 256 plain-BP workload shape
    (512, 256, 24, POLY24, 2.5, dict(mode=1, rho_range_fixed=5, P_level=8, N_min=20, T0=20), 300, 300),
    (1024, 512, 24, POLY24, 2.5, dict(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10), 300, 300),
    (1024, 512, 24, POLY24, 2.0, dict(mode=2, it_reset_full=100, q_max=10), 1000, 60),
    (1024, 512, 24, POLY24, 2.5, dict(mode=1, P_range=2, P_level=6, D=8, N_min=4, T0=16, alpha=1.0), 200, 200),
    # the stop test from iteration 5 only (Sec. IV does not say how many first iterations skip it)
    (1024, 512, 24, POLY24, 3.0, dict(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10, stop_from=5), 300, 300),
    (2048, 1024, 24, POLY24, 2.25, dict(mode=1, rho_range_fixed=3, P_level=10, N_min=5, T0=5, stop_kind=3), 100, 150),
]


@pytest.mark.parametrize("case", DECODE_CASES, ids=lambda c: f"N{c[0]}-mode{c[5]['mode']}-a{c[5].get('alpha', 1)}")
def test_decode_outputs_bit_exact(pcbp, oracle, case):
    N, K, r, poly, ebn0, kw, max_iters, B = case
    fr, pay, x, llr = frames(oracle, N, K, r, poly, B, ebn0, seed=N * 7 + kw["mode"])
    s = pcbp.sched(**{"seed": 12345, "stop_kind": 1, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    bits, iters, ok, _ = gpu_decode(pcbp, code, llr, s, max_iters)
    rbits, riters, rok = oracle_outputs(oracle, fr, r, poly, llr, osched(oracle, s), max_iters)
    assert np.array_equal(iters, riters)
    assert np.array_equal(ok, rok)
    assert np.array_equal(bits, rbits)
    # the case spans converged and unconverged frames, and no frame stops before stop_from
    assert (iters < max_iters).any()
    assert iters.min() >= min(kw.get("stop_from", 1), max_iters)


@pytest.mark.parametrize("N,K", [(16, 8), (64, 32), (256, 128), (1024, 512)])
def test_decode_small_subgraph_events_bit_exact(pcbp, oracle, N, K):
    """rho_range = 2 starting at level 1 (m = 2): the permuted stages are
    narrower than a register group and take the per-PE path of the decoder."""
    fr, pay, x, llr = frames(oracle, N, K, 0, 0, 300, 1.5, seed=N + 11)
    s = pcbp.sched(mode=1, P_range=2, P_level=1, N_min=2, T0=2, seed=21, stop_kind=2)
    code = pcbp.pc_construct(N, K)
    bits, iters, ok, _ = gpu_decode(pcbp, code, llr, s, 40)
    rbits, riters, rok = oracle_outputs(oracle, fr, 0, 0, llr, osched(oracle, s), 40)
    assert np.array_equal(iters, riters)
    assert np.array_equal(bits, rbits)
    assert (iters > 2).any()


def test_edge_sizes_and_degenerate_cases(pcbp, oracle):
    cases = [
        (8, 8, 0, 0, dict(mode=0, stop_kind=0), 3, 5),        # K = N: nothing frozen, no stop
        (8, 1, 0, 0, dict(mode=0), 4, 3),                      # one information bit (repetition code)
        (32, 31, 0, 0, dict(mode=0, stop_kind=2), 6, 10),     # single frozen bit (even-weight code)
        (64, 48, 32, 0x104C11DB7, dict(mode=0), 5, 11),        # 32-bit CRC
        (256, 128, 8, POLY8, dict(mode=0), 0, 9),              # zero iterations
        (2048, 1024, 24, POLY24, dict(mode=1, rho_range_fixed=11, P_level=10, N_min=2, T0=2), 9, 5),  # full range
        (1024, 512, 24, POLY24, dict(mode=2, it_reset_full=1, q_max=0, stop_kind=0), 7, 33),  # switch every iter
    ]
    for N, K, r, poly, kw, max_iters, B in cases:
        fr, pay, x, llr = frames(oracle, N, K, r, poly, B, 1.0, seed=N + K)
        s = pcbp.sched(**{"seed": 4, "stop_kind": 1, **kw})
        code = pcbp.pc_construct(N, K, r, poly)
        bits, iters, ok, _ = gpu_decode(pcbp, code, llr, s, max_iters)
        rbits, riters, rok = oracle_outputs(oracle, fr, r, poly, llr, osched(oracle, s), max_iters)
        assert np.array_equal(iters, riters), (N, K, kw)
        assert np.array_equal(ok, rok), (N, K, kw)
        assert np.array_equal(bits, rbits), (N, K, kw)


def test_empty_batch_is_a_no_op(pcbp):
    import torch

    dev = gpu_device()
    code = pcbp.pc_construct(256, 128, 8, POLY8)
    z = torch.empty((0, 256), dtype=torch.float32, device=dev)
    e = torch.empty((0, 4), dtype=torch.int32, device=dev)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    pcbp.bp_decode(code, z, pcbp.sched(), 10, e, e[:, 0], e[:, 0].to(torch.uint8), ws)
    torch.cuda.synchronize()


def test_frame_base_shifts_the_event_stream(pcbp, oracle):
    """Frame b of a call with frame_base F draws the events of frame F + b, so a
    batch split into shards decodes exactly as the whole batch."""
    N, K, r = 256, 128, 8
    fr, pay, x, llr = frames(oracle, N, K, r, POLY8, 96, 2.0, seed=31)
    code = pcbp.pc_construct(N, K, r, POLY8)
    kw = dict(mode=1, rho_range_fixed=3, P_level=7, N_min=3, T0=3, seed=99, stop_kind=1)
    whole = gpu_decode(pcbp, code, llr, pcbp.sched(**kw), 40)
    a = gpu_decode(pcbp, code, llr[:40], pcbp.sched(**kw, frame_base=0), 40)
    b = gpu_decode(pcbp, code, llr[40:], pcbp.sched(**kw, frame_base=40), 40)
    for i in range(3):
        assert np.array_equal(whole[i], np.concatenate([a[i], b[i]]))


def test_repeated_calls_are_deterministic(pcbp, oracle):
    N, K, r = 1024, 512, 24
    fr, pay, x, llr = frames(oracle, N, K, r, POLY24, 500, 2.25, seed=8)
    code = pcbp.pc_construct(N, K, r, POLY24)
    s = pcbp.sched(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10, seed=1)
    first = gpu_decode(pcbp, code, llr, s, 300)
    for _ in range(2):
        again = gpu_decode(pcbp, code, llr, s, 300)
        for i in range(3):
            assert np.array_equal(first[i], again[i])


def _full_size_sampled(pcbp, oracle, sched_kw, max_iters, ebn0, seed, fer_max, N=1024, B=1 << 20):
    """B frames of length N, K = N/2 (CRC-24) in one launch.  Codewords come from a pool the
    oracle encodes, noise from torch's device generator.  The frames checked one by one against
    the oracle: 192 drawn at random, the first and the last, the 16 that ran the most iterations
    (each through many switches) and 16 more that switched at least once and then stopped."""
    import torch

    dev = gpu_device()
    K, r = N // 2, 24
    _, fr = oracle.construct(N, K)
    pool = 1024
    pay = inputs.payload_numpy(seed, pool, K - r)
    xpool = torch.from_numpy(oracle.encode_frames(pay, fr, r, POLY24)).to(dev)
    idx = torch.arange(B, device=dev) % pool
    gen = torch.Generator(device=dev).manual_seed(seed)
    llr = inputs.bpsk_awgn_llr_torch(xpool[idx], gen, inputs.sigma2_of(ebn0, K, r, N)).contiguous()
    code = pcbp.pc_construct(N, K, r, POLY24)
    s = pcbp.sched(**sched_kw)
    dec = pcbp.Decoder(code, s, max_iters, dev)
    bits, iters, ok = dec(llr)
    torch.cuda.synchronize()
    it = iters.cpu().numpy()
    first_switch = s.T0 if s.mode == 1 else s.it_reset_full
    rng = np.random.default_rng(0)
    longest = np.argsort(-it, kind="stable")[:16]
    switched = np.flatnonzero((it > first_switch) & (it < max_iters))
    mid = rng.choice(switched, min(16, len(switched)), replace=False) if len(switched) else switched
    sample = np.unique(np.concatenate([rng.choice(B, 192, replace=False), [0, B - 1], longest, mid]))
    assert it[longest].max() > 3 * first_switch        # frames that went through several switches
    h_llr = llr[torch.from_numpy(sample).to(dev)].cpu().numpy()
    gb = pcbp.unpack_bits(bits[torch.from_numpy(sample).to(dev)], K).cpu().numpy()
    os_ = osched(oracle, s)
    for j, b in enumerate(sample):
        ref = oracle.decode(fr, r, POLY24, h_llr[j], os_, max_iters, frame_id=int(b))
        assert int(iters[b]) == ref.iters and int(ok[b]) == ref.crc_ok, f"frame {b}"
        assert np.array_equal(gb[j], oracle.info_bits(ref.uhat, fr)), f"frame {b}"
    # whole-batch properties: every frame decoded, iterations within bounds, and the payload
    # recovered on nearly all frames
    assert it.min() >= 1 and it.max() <= max_iters
    got = pcbp.unpack_bits(bits, K)[:, : K - r]
    want = torch.from_numpy(pay).to(dev)[idx]
    fer = (got != want).any(dim=1).float().mean().item()
    assert fer < fer_max


def test_full_size_workload_sampled(pcbp, oracle):
    """The benchmark's launch: PP-BP s = 4, T = 10, max 300 iterations, Eb/N0 3 dB."""
    _full_size_sampled(pcbp, oracle, dict(mode=1, rho_range_fixed=4, P_level=9, N_min=10, T0=10, seed=3,
                                          stop_kind=1), 300, 3.0, 2024, 0.05)


@pytest.mark.parametrize("N,B", [(512, 1 << 20), (2048, 1 << 19)])
def test_full_size_other_lengths_sampled(pcbp, oracle, N, B):
    """The benchmark's schedule at the other lengths of the PP-BP configuration (N = 512 and
    2048, K = N/2, CRC-24), 2^20 and 2^19 frames."""
    n = N.bit_length() - 1
    _full_size_sampled(pcbp, oracle, dict(mode=1, rho_range_fixed=4, P_level=n - 1, N_min=10, T0=10, seed=3,
                                          stop_kind=1), 300, 2.75, 2026 + n, 0.1, N=N, B=B)


def test_full_size_fpbp_sampled(pcbp, oracle):
    """FP-BP at the same size: 10 stage orders of 100 iterations each (max 1000), Eb/N0 2.5 dB."""
    _full_size_sampled(pcbp, oracle, dict(mode=2, q_max=10, it_reset_full=100, seed=2, stop_kind=1),
                       1000, 2.5, 2025, 0.15)


# --------------------------------------------------------------------------- the two production kernels
KERNEL_CASES = [
    (128, 64, 8, POLY8, 2.0, dict(mode=1, rho_range_fixed=3, P_level=6, N_min=3, T0=3), 60, 3000),
    (128, 96, 8, POLY8, 2.5, dict(mode=2, it_reset_full=5, q_max=8, stop_kind=3), 50, 1500),
    (256, 128, 8, POLY8, 2.0, dict(mode=1, rho_range_fixed=4, P_level=7, N_min=3, T0=3), 60, 3000),
    (512, 256, 24, POLY24, 1.75, dict(mode=1, P_range=9, P_level=8, D=40, N_min=2, T0=2, stop_kind=3), 80, 1500),
    (1024, 512, 24, POLY24, 2.0, dict(mode=1, rho_range_fixed=4, P_level=9, N_min=4, T0=4), 120, 2000),
    (1024, 512, 24, POLY24, 1.5, dict(mode=1, P_range=2, P_level=1, N_min=2, T0=2, stop_kind=2), 40, 600),
    (1024, 512, 24, POLY24, 1.75, dict(mode=2, it_reset_full=7, q_max=12), 90, 800),
    (1024, 512, 24, POLY24, 2.0, dict(mode=1, rho_range_fixed=3, P_level=9, N_min=3, T0=3, fkind=1), 60, 800),
    (2048, 1024, 24, POLY24, 2.0, dict(mode=1, P_range=11, P_level=10, N_min=2, T0=2, stop_kind=3), 40, 300),
]


@pytest.mark.parametrize("case", KERNEL_CASES, ids=lambda c: f"N{c[0]}-mode{c[5]['mode']}-f{c[5].get('fkind', 0)}")
def test_tmem_and_grouped_kernels_agree(pcbp, oracle, monkeypatch, case):
    """From N = 128 on, bp_decode keeps the interior messages of each stage
    group in tensor memory (groups of 2 stages at N = 128, of 3 from 256);
    PCBP_DECODER=grouped selects the shared-memory
    kernel.  Same arithmetic, so identical outputs, box-plus included (whose
    transcendental functions the CPU oracle does not reproduce bit for bit)."""
    N, K, r, poly, ebn0, kw, max_iters, B = case
    _, _, _, llr = frames(oracle, N, K, r, poly, B, ebn0, seed=N * 13 + kw["mode"] + kw.get("fkind", 0))
    s = pcbp.sched(**{"seed": 777, "stop_kind": 1, **kw})
    code = pcbp.pc_construct(N, K, r, poly)
    monkeypatch.delenv("PCBP_DECODER", raising=False)
    bits, iters, ok, _ = gpu_decode(pcbp, code, llr, s, max_iters)
    monkeypatch.setenv("PCBP_DECODER", "grouped")
    gbits, giters, gok, _ = gpu_decode(pcbp, code, llr, s, max_iters)
    assert np.array_equal(iters, giters)
    assert np.array_equal(ok, gok)
    assert np.array_equal(bits, gbits)
    assert (iters > 2 * kw.get("T0", kw.get("it_reset_full", 1))).any()   # frames that went through switches


def test_partition_builders_agree_on_every_event_shape(pcbp):
    """The warp-parallel partition build used at a switch equals the single-threaded one for every
    (level, range) of N = 128..2048, three orders and blocks each; every partition, the no-event
    one included, has the group shape the sweeps assume (at least two groups, each middle group
    a single stage or a full group)."""
    checked, differ, irregular = pcbp.pc_partition_selfcheck(gpu_device())
    shapes = 3 * sum(1 for n in range(8, 12) for lv in range(1, n) for rg in range(2, 17) if lv + rg - 1 <= n)
    shapes += 3 * sum(1 for lv in range(1, 7) for rg in range(2, 17) if lv + rg - 1 <= 7)   # N = 128
    assert checked == shapes + 5            # + the no-event partition of each length
    assert differ == 0
    assert irregular == 0
