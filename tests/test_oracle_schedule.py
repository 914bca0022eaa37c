"""Pins of the oracle's switch schedule (Sec. III, Eq. 2, Algorithm 1; Sec. II-D
for FP-BP) against hand-derived iteration numbers.

A switch zeroes L and R at the interior node levels of a subgraph.  Every L
message of the graph is a min-sum combination that involves a channel LLR, so
with Gaussian channel LLRs the L messages are nonzero after every ordinary
iteration; an iteration whose dump shows a subgraph's interior all zero is
therefore an iteration that ended with a switch touching that subgraph.  The
expected iterations below are worked out by hand from T0 and Eq. 2
(N_it,reset <- iter + max(N_min, floor(N_zero / D))), with
N_zero = 2^(level + range - 1) (range - 1) (Sec. III), and written as literals.
"""
import numpy as np
import pytest

n, N = 5, 32
ALPHA = 0.9375


def _interior_mask(level, range_, block):
    """Node levels level+1 .. level+range-1 of the subgraph whose n-m low index
    bits equal `block` (m = level + range - 1), as a [(n+1), N] mask."""
    m = level + range_ - 1
    mask = np.zeros((n + 1, N), dtype=bool)
    for lev in range(level + 1, level + range_):
        for j in range(N):
            if j % (1 << (n - m)) == block:
                mask[lev - 1, j] = True
    return mask


def _zeroed_iters(dump, mask):
    """1-based iterations after which every L and R message under the mask is 0."""
    return [it + 1 for it in range(dump.shape[0]) if np.all(dump[it, 0][mask] == 0) and np.all(dump[it, 1][mask] == 0)]


def _code_and_llr(oracle, seed, dtype):
    _, fr = oracle.construct(N, 16)
    llr = np.random.default_rng(seed).normal(1.0, 2.0, N).astype(dtype)
    return fr, llr


# Three explicit events on disjoint node sets (level, range, block, order):
#   A = (1, 2, 3): m = 2, levels {2},    j % 8 == 3, N_zero = 2^2 * 1 = 4
#   B = (2, 3, 1): m = 4, levels {3, 4}, j odd,      N_zero = 2^4 * 2 = 32
#   C = (1, 3, 2): m = 3, levels {2, 3}, j % 4 == 2, N_zero = 2^3 * 2 = 16
EV_A, EV_B, EV_C = (1, 2, 3, [1, 0]), (2, 3, 1, [2, 0, 1]), (1, 3, 2, [1, 2, 0])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pp_switch_iterations_follow_eq2(oracle, dtype):
    """T0 = 2, N_min = 3, D = 4:
       switch 1 at 2 (T0), applies A, increment max(3, 4 // 4 = 1) = 3 -> next at 5;
       switch 2 at 5, applies B, increment max(3, 32 // 4 = 8) = 8   -> next at 13;
       switch 3 at 13, applies C, increment max(3, 16 // 4 = 4) = 4  -> next at 17,
       where the event list is exhausted: no switch.
    A switch also zeroes the previous event's subgraph (it reverts to the original order)."""
    fr, llr = _code_and_llr(oracle, 11, dtype)
    evs = [oracle.Event.make(*e) for e in (EV_A, EV_B, EV_C)]
    s = oracle.Sched(mode=1, T0=2, N_min=3, D=4, stop_kind=0, alpha=ALPHA)
    d = oracle.decode(fr, 0, 0, llr, s, 20, events=evs, dump=True, dtype=dtype).dump
    mA, mB, mC = (_interior_mask(*e[:3]) for e in (EV_A, EV_B, EV_C))
    assert mA.sum() == 4 and mB.sum() == 32 and mC.sum() == 16
    assert _zeroed_iters(d, mA) == [2, 5]          # applied at 2, reverted at 5
    assert _zeroed_iters(d, mB) == [5, 13]         # applied at 5, reverted at 13
    assert _zeroed_iters(d, mC) == [13]            # applied at 13, never reverted (no 4th switch)
    # L is nonzero everywhere else at every iteration
    for it in range(20):
        zero = d[it, 0] == 0
        assert not zero[0].any()                   # channel level
        expect = {2: mA, 5: mA | mB, 13: mB | mC}.get(it + 1, np.zeros_like(mA))
        assert np.array_equal(zero[1:n], expect[1:n])


def test_pp_switch_with_d_infinite_is_every_n_min(oracle):
    """D = 0 stands for D = infinity: Eq. 2 gives N_min after every switch
    (T0 = 3, N_min = 4: switches at 3, 7, 11, 15, 19)."""
    fr, llr = _code_and_llr(oracle, 12, np.float64)
    evs = [oracle.Event.make(*e) for e in (EV_A, EV_B, EV_A, EV_B, EV_A, EV_B)]
    s = oracle.Sched(mode=1, T0=3, N_min=4, D=0, stop_kind=0, alpha=ALPHA)
    d = oracle.decode(fr, 0, 0, llr, s, 20, events=evs, dump=True, dtype=np.float64).dump
    mA, mB = _interior_mask(*EV_A[:3]), _interior_mask(*EV_B[:3])
    # A applied at 3, 11, 19; B applied at 7, 15; each reverted at the next switch
    assert _zeroed_iters(d, mA) == [3, 7, 11, 15, 19]
    assert _zeroed_iters(d, mB) == [7, 11, 15, 19]


def test_switch_graph_reverts_to_the_original_order(oracle):
    """Reading R1 of Sec. III: after the second switch the graph is the
    original graph with only the second event's subgraph permuted.  The
    trajectory equals one built from single iterations (pinned separately by
    closed forms) on hand-chosen graphs and zero masks, and differs from the
    cumulative reading (both subgraphs left permuted)."""
    fr, llr = _code_and_llr(oracle, 13, np.float64)
    evA, evB = oracle.Event.make(*EV_A), oracle.Event.make(*EV_B)
    s = oracle.Sched(mode=1, T0=2, N_min=3, D=4, stop_kind=0, alpha=ALPHA)
    got = oracle.decode(fr, 0, 0, llr, s, 12, events=[evA, evB], dump=True, dtype=np.float64).dump

    def replay(cumulative):
        L = np.zeros((n + 1, N))
        R = np.zeros((n + 1, N))
        L[0] = llr
        R[n] = np.where(fr == 1, np.inf, 0.0)
        g0 = oracle.graph_from_event(n)
        gA = oracle.graph_from_event(n, evA)
        gB = oracle.graph_from_event(n, evB)
        gAB = gB.copy()
        mA_idx = _interior_mask(1, 2, 3)           # unused for graphs, kept for zeroing
        low_a = np.arange(N) % 8 == 3               # A's subgraph: stages 1..2 of indices j % 8 == 3
        gAB[:2, low_a] = gA[:2, low_a]
        sb = g0
        out = []
        for it in range(1, 13):
            oracle.bp_iteration(n, sb, L, R, ALPHA, 0)
            if it == 2:                             # T0
                sb = gA
                L[mA_idx] = 0
                R[mA_idx] = 0
            if it == 5:                             # 2 + max(3, 4 // 4)
                sb = gAB if cumulative else gB
                z = mA_idx | _interior_mask(2, 3, 1)
                L[z] = 0
                R[z] = 0
            out.append((L.copy(), R.copy()))
        return out

    ref = replay(False)
    for it in range(12):
        assert np.array_equal(got[it, 0], ref[it][0]) and np.array_equal(got[it, 1], ref[it][1]), it + 1
    cum = replay(True)
    assert not np.array_equal(cum[11][1], ref[11][1])   # the cumulative graph gives other messages


@pytest.mark.parametrize("q_max,expect", [(3, [3, 6]), (0, [3, 6, 9, 12]), (1, []), (2, [3])])
def test_fp_bp_switches_at_most_q_max_minus_one_times(oracle, q_max, expect):
    """FP-BP (Sec. II-D): q_max trellises, so at most q_max - 1 switches, one
    every it_reset_full = 3 iterations (q_max = 0: no cap); each switch zeroes
    every L and R at node levels 2..n."""
    fr, llr = _code_and_llr(oracle, 14, np.float64)
    s = oracle.Sched(mode=2, it_reset_full=3, q_max=q_max, stop_kind=0, alpha=ALPHA, seed=5)
    d = oracle.decode(fr, 0, 0, llr, s, 12, dump=True, dtype=np.float64).dump
    inner = np.zeros((n + 1, N), dtype=bool)
    inner[1:n] = True
    assert _zeroed_iters(d, inner) == expect


def test_no_switch_on_the_iteration_whose_stop_test_passes(oracle):
    """The stop test comes before the switch in an iteration: a frame that
    stops at iteration T0 is not switched there."""
    _, fr = oracle.construct(N, 16)
    pay = np.random.default_rng(2).integers(0, 2, 16).astype(np.uint8)
    x = oracle.encode_frames(pay[None], fr, 0, 0)[0]
    llr = (1 - 2 * x.astype(np.float64)) * 4.0 + np.random.default_rng(3).normal(0, 0.5, N)
    evs = [oracle.Event.make(*EV_B)]
    mB = _interior_mask(*EV_B[:3])
    base = dict(mode=1, T0=3, N_min=5, D=0, alpha=ALPHA)
    run = oracle.decode(fr, 0, 0, llr, oracle.Sched(**base, stop_kind=0), 6, events=evs, dump=True,
                        dtype=np.float64)
    assert _zeroed_iters(run.dump, mB) == [3]
    stop = oracle.decode(fr, 0, 0, llr, oracle.Sched(**base, stop_kind=2, stop_from=3), 6, events=evs,
                         dump=True, dtype=np.float64)
    assert stop.iters == 3
    assert _zeroed_iters(stop.dump[:3], mB) == []
    assert np.array_equal(stop.dump[:2], run.dump[:2])


def test_switch_on_the_last_iteration_keeps_the_decisions(oracle):
    """A switch in the final iteration zeroes interior levels only (never level
    n+1), so the decisions equal those of the same run without that switch."""
    fr, llr = _code_and_llr(oracle, 15, np.float64)
    evs = [oracle.Event.make(*EV_B)]
    a = oracle.decode(fr, 0, 0, llr, oracle.Sched(mode=1, T0=6, N_min=5, stop_kind=0, alpha=ALPHA), 6,
                      events=evs, dump=True, dtype=np.float64)
    b = oracle.decode(fr, 0, 0, llr, oracle.Sched(mode=0, stop_kind=0, alpha=ALPHA), 6, dump=True,
                      dtype=np.float64)
    assert _zeroed_iters(a.dump, _interior_mask(*EV_B[:3])) == [6]
    assert np.array_equal(a.uhat, b.uhat) and a.iters == b.iters == 6
