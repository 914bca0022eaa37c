"""Messages of the production decoder kernel (the one bp_decode runs for N >= 128) against the
oracle, through bp_decode_posterior: L at node level n+1 and R at node level 1 after each frame's
last iteration (Sec. II-B), and the PE function f itself through pc_f_eval.

Scaled min-sum: bit-exact with the FP32 oracle.  Exact box-plus: within 1e-5 of the FP64 oracle,
relative for |value| >= 1 and absolute below (err <= 1e-5 * max(1, |ref|)).  The correction
term of f lies in (-ln 2, ln 2) and is evaluated in FP32 with an absolute error of a few 1e-7
whatever the size of f, so below 1 the bound is an absolute one."""
import numpy as np
import pytest

from conftest import gpu_device
from test_gpu_parity import POLY24, POLY8, assert_bitwise_equal, frames, osched

pytestmark = pytest.mark.gpu

CODES = {128: (64, 8, POLY8), 256: (128, 8, POLY8), 512: (256, 24, POLY24), 1024: (512, 24, POLY24),
         2048: (1024, 24, POLY24)}


def gpu_posterior(pcbp, code, llr, s, max_iters):
    import torch

    dev = gpu_device()
    B, N = llr.shape
    d_llr = torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).to(dev)
    bits = torch.full((B, pcbp.words_of(code.K)), -1, dtype=torch.int32, device=dev)
    iters = torch.full((B,), -7, dtype=torch.int32, device=dev)
    ok = torch.full((B,), 9, dtype=torch.uint8, device=dev)
    post = torch.full((B, 2, N), float("nan"), dtype=torch.float32, device=dev)
    ws = torch.zeros(pcbp.bp_decode_workspace_size(code, B), dtype=torch.uint8, device=dev)
    pcbp.bp_decode_posterior(code, d_llr, s, max_iters, bits, iters, ok, post, ws)
    torch.cuda.synchronize()
    return (pcbp.unpack_bits(bits, code.K).cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(),
            post.cpu().numpy())


def oracle_posterior(oracle, fr, r, poly, llr_row, os_, max_iters, frame_id, dtype):
    res = oracle.decode(fr, r, poly, llr_row.astype(dtype), os_, max_iters, frame_id=frame_id, dump=True,
                        dtype=dtype)
    n = len(fr).bit_length() - 1
    last = res.dump[res.iters - 1]
    return res, last[0, n], last[1, 0]


SCHEDS = {
    # random subgraph ranges and levels, first switch after 2 iterations, then every 2: narrow
    # level-1 events give single-stage groups, wide ones subgraph-local groups
    "ppbp_random": dict(mode=1, P_range=5, N_min=2, T0=2, stop_kind=0, seed=21),
    "ppbp_s4": dict(mode=1, rho_range_fixed=4, N_min=2, T0=2, stop_kind=0, seed=22),
    "fpbp": dict(mode=2, it_reset_full=2, q_max=4, stop_kind=0, seed=23),
    "plain": dict(mode=0, stop_kind=0, seed=24),
}


@pytest.mark.parametrize("N", [128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("name", list(SCHEDS))
def test_min_sum_messages_bit_exact(pcbp, oracle, N, name):
    K, r, poly = CODES[N]
    n = N.bit_length() - 1
    B = 24
    fr, pay, x, llr = frames(oracle, N, K, r, poly, B, 2.0, seed=N + len(name))
    kw = dict(SCHEDS[name], alpha=0.9375)
    if kw["mode"] == 1:
        kw["P_level"] = n - 1
    s = pcbp.sched(**kw)
    os_ = osched(oracle, s)
    code = pcbp.pc_construct(N, K, r, poly)
    for max_iters in (1, 3, 6):
        bits, iters, ok, post = gpu_posterior(pcbp, code, llr, s, max_iters)
        for b in range(B):
            res, lu, r1 = oracle_posterior(oracle, fr, r, poly, llr[b], os_, max_iters, b, np.float32)
            assert iters[b] == res.iters == max_iters
            assert_bitwise_equal(post[b, 0], lu, f"L(n+1) N={N} {name} it={max_iters} frame {b}")
            assert_bitwise_equal(post[b, 1], r1, f"R(1) N={N} {name} it={max_iters} frame {b}")
            assert np.array_equal(bits[b], oracle.info_bits(res.uhat, fr))


@pytest.mark.parametrize("N", [256, 1024])
def test_min_sum_messages_bit_exact_with_crc_stop(pcbp, oracle, N):
    """Frames that stop early: the messages of the stopping iteration, R sweep completed."""
    K, r, poly = CODES[N]
    n = N.bit_length() - 1
    B = 48
    fr, pay, x, llr = frames(oracle, N, K, r, poly, B, 3.0, seed=3 * N)
    s = pcbp.sched(mode=1, rho_range_fixed=3, P_level=n - 1, N_min=3, T0=3, stop_kind=1, alpha=0.9375, seed=5)
    os_ = osched(oracle, s)
    code = pcbp.pc_construct(N, K, r, poly)
    bits, iters, ok, post = gpu_posterior(pcbp, code, llr, s, 30)
    assert len(set(iters.tolist())) > 2         # frames stop at different iterations
    for b in range(B):
        res, lu, r1 = oracle_posterior(oracle, fr, r, poly, llr[b], os_, 30, b, np.float32)
        assert iters[b] == res.iters and ok[b] == res.crc_ok
        assert_bitwise_equal(post[b, 0], lu, f"L(n+1) frame {b}")
        assert_bitwise_equal(post[b, 1], r1, f"R(1) frame {b}")


def _rel_err(got, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.array_equal(got[~fin], ref[~fin])
    return np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))


@pytest.mark.parametrize("N", [128, 256, 512, 1024, 2048])
@pytest.mark.parametrize("name", ["ppbp_random", "fpbp", "plain"])
def test_boxplus_messages_within_1e5(pcbp, oracle, N, name):
    K, r, poly = CODES[N]
    n = N.bit_length() - 1
    B = 16
    fr, pay, x, llr = frames(oracle, N, K, r, poly, B, 2.0, seed=7 * N + len(name))
    kw = dict(SCHEDS[name], fkind=1, alpha=1.0)
    if kw["mode"] == 1:
        kw["P_level"] = n - 1
    s = pcbp.sched(**kw)
    os_ = osched(oracle, s)
    code = pcbp.pc_construct(N, K, r, poly)
    worst = 0.0
    for max_iters in (1, 3, 5):
        _, iters, _, post = gpu_posterior(pcbp, code, llr, s, max_iters)
        for b in range(B):
            res, lu, r1 = oracle_posterior(oracle, fr, r, poly, llr[b], os_, max_iters, b, np.float64)
            for got, ref in ((post[b, 0], lu), (post[b, 1], r1)):
                worst = max(worst, _rel_err(got.astype(np.float64), ref).max())
    assert worst < 1e-5, worst


def test_f_eval_min_sum_matches_its_definition(pcbp):
    import torch

    dev = gpu_device()
    rng = np.random.default_rng(1)
    a = rng.normal(0, 5, 1 << 20).astype(np.float32)
    b = rng.normal(0, 5, 1 << 20).astype(np.float32)
    a[:1000] = 0.0
    b[1000:2000] = np.inf
    a[2000:3000] = -np.inf
    b[2000:2500] = np.inf
    for alpha in (1.0, 0.9375):
        out = torch.empty(len(a), dtype=torch.float32, device=dev)
        pcbp.pc_f_eval(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), out, 0, alpha)
        m = np.minimum(np.abs(a), np.abs(b))
        want = np.float32(alpha) * m
        want = np.where(np.signbit(a) != np.signbit(b), -want, want).astype(np.float32)
        assert_bitwise_equal(out.cpu().numpy(), want, f"min-sum f alpha={alpha}")


def test_f_eval_boxplus_error_bound(pcbp):
    """Box-plus f of the kernels against the exact value (FP64 on the same FP32 operands):
    |f - exact| <= 6e-7 + 2^-23 |exact| on 4M pairs, operands of equal magnitude, of opposite
    sign, tiny, large and infinite included."""
    import torch

    dev = gpu_device()
    rng = np.random.default_rng(2)
    M = 1 << 22
    a = rng.normal(0, 6, M).astype(np.float32)
    b = rng.normal(0, 6, M).astype(np.float32)
    a[: M // 16] = b[: M // 16]
    a[M // 16: M // 8] = -b[M // 16: M // 8]
    a[M // 8: M // 4] *= np.float32(1e-3)
    b[M // 4: M // 4 + 1000] = np.inf
    a[M // 4 + 1000: M // 4 + 2000] = -np.inf
    b[M // 4 + 1500: M // 4 + 2000] = np.inf
    a[M // 4 + 2000: M // 4 + 3000] = 0.0
    b[M // 4 + 3000: M // 4 + 5000] = rng.normal(0, 300, 2000).astype(np.float32)
    out = torch.empty(M, dtype=torch.float32, device=dev)
    pcbp.pc_f_eval(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), out, 1, 1.0)
    got = out.cpu().numpy().astype(np.float64)
    A, B = a.astype(np.float64), b.astype(np.float64)
    sm = np.where(np.signbit(a) != np.signbit(b), -1.0, 1.0) * np.minimum(np.abs(A), np.abs(B))
    with np.errstate(invalid="ignore"):
        corr = np.log1p(np.exp(-np.abs(A + B))) - np.log1p(np.exp(-np.abs(A - B)))
    inf = np.isinf(A) | np.isinf(B)
    exact = np.where(inf, sm, sm + np.nan_to_num(corr))
    assert np.array_equal(got[inf], exact[inf])
    err = np.abs(got[~inf] - exact[~inf])
    bound = 6e-7 + 2.0 ** -23 * np.abs(exact[~inf])
    assert np.all(err <= bound), float((err - bound).max())
