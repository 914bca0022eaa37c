"""Autotuner of the mixed-length sweep's launch shape per code length: threads per
frame (which decoder kernel) and frames resident per CTA ("slots").

For each length it decodes a synthetic batch (rate 1/2, BPSK/AWGN at the given
Eb/N0, the given schedule) with every candidate shape through a single-batch
MixedDecoder, times the launches with CUDA events and keeps the fastest.
Threads per frame: the counts bp_kernel_threads reports for the two kernels
(TMEM-resident stage groups: N/4 up to N = 256, N/8 from 512; shared-memory
groups: max(32, N/4); where they coincide the library runs the TMEM kernel).  Results are cached per GPU
name, library build and schedule in a JSON file ($PCBP_TUNE_CACHE, default ~/.cache/pcbp_tune.json).
"""
from __future__ import annotations

import json
import os
from pathlib import Path

SLOT_CANDIDATES = (1, 2, 3, 4, 6, 8, 12, 16, 24)
# pc_sched fields that select the kernel variant or change the work per frame
SCHED_KEY_FIELDS = ("fkind", "mode", "stop_kind", "stop_from", "rho_range_fixed", "P_range", "P_level", "T0",
                    "N_min", "D", "q_max", "it_reset_full", "alpha")


def cache_path() -> Path:
    return Path(os.environ.get("PCBP_TUNE_CACHE", str(Path.home() / ".cache" / "pcbp_tune.json")))


def crc_for(N: int):
    return (8, 0x9B) if N <= 256 else (24, 0x1B2B117)


def threads_candidates(pcbp, code):
    """Distinct threads-per-frame counts that select a decoder kernel for this code (where both
    kernels take the same count, the library runs the TMEM one)."""
    return sorted({t for t in (pcbp.bp_kernel_threads(code, k) for k in (0, 1)) if t})


def _synthetic(pcbp, inputs, dev, N, K, r, poly, B, ebn0, seed):
    import torch

    code = pcbp.pc_construct(N, K, r, poly)
    gen = torch.Generator(device=dev).manual_seed(seed)
    pay = inputs.payload_torch(gen, B, K - r, dev)
    x = torch.empty((B, N), dtype=torch.uint8, device=dev)
    pcbp.pc_encode(code, pay, x)
    llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(ebn0, K, r, N)).contiguous()
    return code, llr


def tune_launch(lengths, sched_for, max_iters: int = 300, frames: int = 16384, ebn0: float = 2.5,
                device="cuda", use_cache: bool = True, reps: int = 3) -> dict:
    """Fastest {"threads_per_frame": t, "slots": s} per length.  sched_for(n) returns the
    pc_sched for log2 N = n.  Candidate slot counts are capped at the kernel's limit on this
    device (bp_slot_limit), so every reported count is one the launch uses; equal timings are
    broken toward fewer slots."""
    import torch

    from . import inputs, pcbp

    dev = torch.device(device)
    lib = pcbp.library_path()
    # a rebuilt library (new kernels) is tuned afresh
    key = f"{torch.cuda.get_device_name(dev)}|{lib}|{os.stat(lib).st_mtime_ns}|{max_iters}|{frames}|{ebn0}|capped"
    cache = {}
    cp = cache_path()
    if use_cache and cp.exists():
        try:
            cache = json.loads(cp.read_text())
        except (OSError, ValueError):
            cache = {}
    entry = cache.get(key, {})
    best = {}
    for N in lengths:
        sch = sched_for(N.bit_length() - 1)
        # the kernel variant (f, stop test) and the work per frame depend on the schedule
        skey = f"{N}|" + "|".join(f"{getattr(sch, f)}" for f in SCHED_KEY_FIELDS)
        if skey in entry and isinstance(entry[skey], dict):
            best[N] = dict(entry[skey])
            continue
        K = N // 2
        r, poly = crc_for(N)
        code, llr = _synthetic(pcbp, inputs, dev, N, K, r, poly, frames, ebn0, seed=N)
        times = {}
        for tpf in threads_candidates(pcbp, code):
            limit = pcbp.bp_slot_limit(code, tpf, int(sch.fkind))
            for slots in sorted({min(c, limit) for c in SLOT_CANDIDATES}):
                md = pcbp.MixedDecoder([(code, sch, max_iters, llr, slots, tpf)], dev)
                md()
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record()
                for _ in range(reps):
                    md()
                t1.record()
                torch.cuda.synchronize()
                times[(tpf, slots)] = t0.elapsed_time(t1) / reps
        tpf, slots = min(times, key=lambda c: (round(times[c], 3), c[1]))
        best[N] = {"threads_per_frame": tpf, "slots": slots, "ms": times[(tpf, slots)]}
        entry[skey] = best[N]
    if use_cache:
        cache[key] = entry
        try:
            cp.parent.mkdir(parents=True, exist_ok=True)
            cp.write_text(json.dumps(cache, indent=1))
        except OSError:
            pass
    return best
