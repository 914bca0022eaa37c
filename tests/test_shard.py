"""Frame sharding: ranges tile the batch, and two gloo ranks decoding their
shards (CPU oracle, frame_base = shard start) sum to the unsplit counters."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1911_08868_gb300.shard import reduce_counters, shard_range


def test_shard_ranges_tile_the_batch():
    for total in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_range(total, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


N, K, R_, POLY, TOTAL, MAXIT = 128, 64, 8, 0x9B, 120, 40


def _counts(lo, hi):
    import oracle as O
    from paper_1911_08868_gb300 import inputs

    _, fr = O.construct(N, K)
    pay = inputs.payload_numpy(11, TOTAL, K - R_)[lo:hi]
    x = O.encode_frames(pay, fr, R_, POLY)
    llr = inputs.bpsk_awgn_llr(x, inputs.noise_numpy(11, TOTAL, N)[lo:hi], inputs.sigma2_of(2.0, K, R_, N))
    s = O.Sched(mode=1, rho_range_fixed=3, P_level=6, N_min=3, T0=3, seed=9, stop_kind=1, frame_base=lo)
    u, it, ok = O.decode_batch(fr, R_, POLY, llr, s, MAXIT, nthreads=1)
    got = O.info_bits(u, fr)[:, : K - R_]
    return {"frames": hi - lo, "frame_errors": int((got != pay).any(axis=1).sum()),
            "bit_errors": int((got != pay).sum()), "iterations": int(it.sum())}


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_range(TOTAL, world, rank)
    total = reduce_counters(_counts(lo, hi))
    out[rank] = total
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_unsplit_run():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        results = dict(out)
    whole = _counts(0, TOTAL)
    assert results[0] == results[1] == whole
    assert whole["iterations"] > TOTAL
