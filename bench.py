"""Throughput of the GB300 PP-BP polar decoder (arXiv 1911.08868).

Workload (one step): 1,000,000 synthetic BPSK/AWGN frames of the N = 1024,
K = 512 polar code with CRC-24 (0x1B2B117), Bhattacharyya construction at
0 dB, decoded by partially permuted multi-trellis BP with subgraphs of s = 4
stages switched every T = 10 iterations (P_level = n - 1), at most 300
iterations, scaled min-sum alpha = 0.9375, CRC stop, Eb/N0 = 3.0 dB.  The
LLRs (4.1 GB per step) are resident in HBM and larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 and no torchrun environment, bench.py re-launches itself
as N local ranks under torch.distributed.run (one per GPU, frames sharded,
weak scaling).

Prints one JSON line.  `value` is decoded information (payload) Gbit/s over
all ranks, timed with CUDA events around the decoder launches; `e2e` is the
same metric through the host-buffer API (bp_decode_host: the decoder reads
the page-locked host LLRs and writes the results into page-locked host memory
across the host-device link, every step).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "decoded info Gbit/s @N=1024 R=0.5 PPMT-BP, FER-matched; WBP fwd+bwd steps/s"
N, K, R_CRC, POLY = 1024, 512, 24, 0x1B2B117
EBN0 = 3.0
MAX_ITERS = 300
FRAMES = 1_000_000
SCHED = dict(mode=1, rho_range_fixed=4, P_level=9, N_min=10, D=0, T0=10, stop_from=1, stop_kind=1,
             alpha=0.9375, seed=3)
WORKLOAD = "PP-BP N=1024 K=512 CRC-24, s=4 T=10, max 300 it, min-sum a=0.9375, BPSK/AWGN Eb/N0=3.0 dB"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="wall-time budget of the CPU oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-wbp", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def free_port() -> int:
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def spawn_ranks(nproc: int, script: str, argv) -> int:
    """Runs `script argv` as nproc local ranks under torch.distributed.run (one process per GPU,
    rendezvous on 127.0.0.1) and returns its exit status; rank 0 prints the JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", f"--master-port={free_port()}", script, *argv]
    return subprocess.run(cmd).returncode


def needs_spawn(gpus: int) -> bool:
    """--gpus N > 1 outside torchrun: bench.py launches its own N ranks."""
    return gpus > 1 and "WORLD_SIZE" not in os.environ


def kernel_sha() -> str:
    """Hash of the N = 1024 bp_decode kernel's sources with comments and white space removed, so
    that the profiled traffic stays attached to the code it was measured on, not to its comments."""
    import re

    h = hashlib.sha256()
    for name in ("bp_kernel.cuh", "bp_kernel2.cuh", "bp_kernel3.cuh", "bp_inst3.cu"):
        text = (ROOT / "paper_1911_08868_gb300" / "csrc" / name).read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:12]


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    return json.loads(p.read_text()) if p.exists() else None


def profiled_traffic(sha: str):
    """DRAM bytes per launch of FRAMES frames from the committed ncu summary, if it was taken on this
    kernel source (the caller scales it to the launch's frame count: the traffic is one LLR read and
    one result write per frame)."""
    p = ROOT / "profiles" / "bp_decode_tmem_n1024_pp_s4t10.md"
    if not p.exists():
        return None
    vals = {}
    for ln in p.read_text().splitlines():
        if ln.startswith("traffic_"):
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.split()[0]
    if vals.get("traffic_kernel_sha") != sha:
        return None
    return float(vals["traffic_bytes_per_launch_full"])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for ln in (self.out or "").splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append(parts)
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle(frames_budget_s: float, seed: int = 97, threads: int = 0):
    """The oracle as it stands (FP32, OpenMP over frames) on host cores (all of
    them, or `threads`), on chunks of the workload until the wall-time budget is
    used."""
    import numpy as np

    import oracle as O
    from paper_1911_08868_gb300 import inputs

    _, fr = O.construct(N, K)
    s = O.Sched(**{**SCHED, "alpha": 0.9375})
    threads = threads or O.max_threads()
    chunk = max(256, 64 * threads)
    done = bits = iters_sum = errs = 0
    elapsed = 0.0
    c = 0
    while elapsed < frames_budget_s or done == 0:
        pay = inputs.payload_numpy(seed + c, chunk, K - R_CRC)
        x = O.encode_frames(pay, fr, R_CRC, POLY)
        llr = inputs.bpsk_awgn_llr(x, inputs.noise_numpy(seed + c, chunk, N), inputs.sigma2_of(EBN0, K, R_CRC, N))
        s.frame_base = done
        t0 = time.perf_counter()
        u, it, ok = O.decode_batch(fr, R_CRC, POLY, llr, s, MAX_ITERS, nthreads=threads)
        elapsed += time.perf_counter() - t0
        got = O.info_bits(u, fr)[:, : K - R_CRC]
        errs += int((got != pay).any(axis=1).sum())
        iters_sum += int(it.sum())
        done += chunk
        bits += chunk * (K - R_CRC)
        c += 1
    return {"gbps": bits / elapsed / 1e9, "frames": done, "seconds": elapsed, "cores": threads,
            "fer": errs / done, "errors": errs, "mean_iters": iters_sum / done}


def wilson(k: int, n: int, z: float = 1.96):
    if n == 0:
        return [0.0, 1.0]
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [max(0.0, c - h), min(1.0, c + h)]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    per = max(args.cpu_seconds / max(steps + warm, 1), 0.5)
    for _ in range(warm):
        cpu_oracle(per * 0.25, seed=1000)
    runs = [cpu_oracle(per, seed=2000 + i) for i in range(steps)]
    frames = sum(r["frames"] for r in runs)
    secs = sum(r["seconds"] for r in runs)
    gbps = frames * (K - R_CRC) / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbps, "unit": "Gbit/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": secs / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": runs[0]["frames"], "note": "bounded sample per step"},
        "cpu_baseline": {"value": gbps, "unit": "Gbit/s", "cores": runs[0]["cores"], "kind": "oracle",
                         "sample": f"{frames} frames over {steps} steps, ~{per:.1f} s each"},
        "e2e": {"value": gbps, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "fer": sum(r["errors"] for r in runs) / frames,
        "mean_iters": sum(r["mean_iters"] * r["frames"] for r in runs) / frames,
    }
    print(json.dumps(line), flush=True)


MIXED_FRAMES = 1 << 20
MIXED_PAIRS = 6          # alternating per-size / sweep timings
# two-sided 95% Student t quantiles by degrees of freedom
T975 = {1: 12.706, 2: 4.303, 3: 3.182, 4: 2.776, 5: 2.571, 6: 2.447, 7: 2.365, 8: 2.306, 9: 2.262, 10: 2.228}
MIXED_LENGTHS = (128, 256, 512, 1024, 2048)
MIXED_RATES = (0.25, 0.5, 0.75)


def mixed_sched(pcbp, n, seed):
    return pcbp.sched(mode=1, rho_range_fixed=4, P_level=n - 1, N_min=10, D=0, T0=10, stop_from=1,
                      stop_kind=1, alpha=0.9375, seed=seed)


def run_mixed(pcbp, inputs, dev, steps, warmup):
    """2^20 frames, N uniform on {128..2048}, rate uniform on {1/4, 1/2, 3/4}, Eb/N0 uniform on
    [1, 4] dB per frame, PP-BP s=4 T=10: 15 per-size bp_decode launches against one
    persistent mixed sweep (threads per frame and slots from the autotuner), both also replayed
    from CUDA graphs."""
    import numpy as np
    import torch

    from paper_1911_08868_gb300 import autotune

    rng = np.random.default_rng(7)
    classes = [(N, R) for N in MIXED_LENGTHS for R in MIXED_RATES]
    counts = rng.multinomial(MIXED_FRAMES, [1 / len(classes)] * len(classes))
    tuned = autotune.tune_launch(MIXED_LENGTHS, lambda n: mixed_sched(pcbp, n, 1), max_iters=MAX_ITERS, device=dev)
    gen = torch.Generator(device=dev).manual_seed(4321)
    parts, info_bits = [], 0
    order = sorted(range(len(classes)), key=lambda i: -classes[i][0] * counts[i])
    for ci in order:
        (N, R), B = classes[ci], int(counts[ci])
        K = int(N * R)
        r, poly = autotune.crc_for(N)
        code = pcbp.pc_construct(N, K, r, poly)
        pay = inputs.payload_torch(gen, B, K - r, dev)
        x = torch.empty((B, N), dtype=torch.uint8, device=dev)
        pcbp.pc_encode(code, pay, x)
        ebn0 = 1.0 + 3.0 * torch.rand(B, generator=gen, device=dev, dtype=torch.float64)
        llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(ebn0.cpu().numpy(), K, r, N)).contiguous()
        del x
        sch = mixed_sched(pcbp, N.bit_length() - 1, 1000 + ci)
        parts.append((code, sch, MAX_ITERS, llr, tuned[N]["slots"], tuned[N]["threads_per_frame"]))
        info_bits += B * (K - r)
    decs = [pcbp.Decoder(p[0], p[1], p[2], dev) for p in parts]
    md = pcbp.MixedDecoder(parts, dev)
    stream = torch.cuda.Stream(dev)

    def per_size():
        for d, p in zip(decs, parts):
            d(p[3], stream)

    def mixed():
        md(stream)

    def timed(fn, reps, warm=0):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                fn()
            stream.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
            stream.synchronize()
        return t0.elapsed_time(t1) / reps if reps else 0.0

    timed(per_size, 0, warmup)
    timed(mixed, 0, warmup)
    same = all(torch.equal(md.iters[i], decs[i].iters) and torch.equal(md.bits[i], decs[i].bits)
               for i in range(len(parts)))
    graphs = {}
    for name, fn in (("per_size", per_size), ("mixed", mixed)):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            fn()
            stream.synchronize()
            with torch.cuda.graph(g, stream=stream):
                fn()
        graphs[name] = g
    # alternating repeats (per-size, then the sweep; plain launches and graph replays), so that
    # clock and temperature drift falls on both sides alike; the speed-up of every pair gives a
    # mean and a 95% interval (Student t)
    pairs = max(MIXED_PAIRS, 2)
    t_per, t_mix, g_per, g_mix = [], [], [], []
    for _ in range(pairs):
        t_per.append(timed(per_size, 1))
        t_mix.append(timed(mixed, 1))
        g_per.append(timed(graphs["per_size"].replay, 1))
        g_mix.append(timed(graphs["mixed"].replay, 1))

    def ratio_ci(num, den):
        r = [a / b for a, b in zip(num, den)]
        m = statistics.mean(r)
        half = T975[len(r) - 1] * statistics.stdev(r) / math.sqrt(len(r))
        return m, [m - half, m + half]

    sp, sp_ci = ratio_ci(t_per, t_mix)
    spg, spg_ci = ratio_ci(g_per, g_mix)
    return {"frames": int(MIXED_FRAMES), "classes": len(classes), "launches_per_size": len(parts),
            "repeats": pairs, "per_size_ms": statistics.mean(t_per), "mixed_ms": statistics.mean(t_mix),
            "per_size_graph_ms": statistics.mean(g_per), "mixed_graph_ms": statistics.mean(g_mix),
            "per_size_ms_runs": t_per, "mixed_ms_runs": t_mix,
            "speedup": sp, "speedup_ci95": sp_ci, "speedup_graphs": spg, "speedup_graphs_ci95": spg_ci,
            "mixed_gbit_s": info_bits / (statistics.mean(g_mix) / 1e3) / 1e9,
            "tuned": {str(k): v for k, v in tuned.items()}, "outputs_identical": bool(same),
            "workload": "2^20 frames, N~U{128..2048}, R~U{1/4,1/2,3/4}, Eb/N0~U[1,4] dB, PP-BP s=4 T=10, "
                        "max 300 it, CRC-8 (N<=256) / CRC-24"}


VARIANT_FRAMES = 1 << 17
VARIANTS = {
    # the benchmark schedule at this frame count, for reference
    "ppbp_s4_t10": dict(SCHED),
    # FP-BP: q_max = 10 trellises of 100 iterations each (a full-order event and a whole-graph reset)
    "fpbp_q10_t100": dict(mode=2, it_reset_full=100, q_max=10, stop_from=1, stop_kind=1, alpha=0.9375, seed=3),
    # BP on the original graph only
    "plain_bp": dict(mode=0, stop_from=1, stop_kind=1, alpha=0.9375, seed=3),
    # unscaled min-sum, as the paper simulates
    "ppbp_alpha1": dict(SCHED, alpha=1.0),
    # CRC and G-matrix stop together
    "ppbp_crc_and_g": dict(SCHED, stop_kind=3),
    # exact box-plus f
    "ppbp_boxplus": dict(SCHED, fkind=1),
    # the stop test applied from iteration 5 only (Sec. IV leaves the number of untested first iterations open)
    "ppbp_stop_from5": dict(SCHED, stop_from=5),
}
VARIANT_MAX_ITERS = {"fpbp_q10_t100": 1000}


def run_variants(pcbp, inputs, dev, warmup):
    """Throughput, FER and mean iterations of the other schedules of the same code on the same
    2^17 frames (Eb/N0 3.0 dB): FP-BP, plain BP, unscaled min-sum, CRC + G-matrix stop, box-plus,
    the stop test from iteration 5."""
    import torch

    B = VARIANT_FRAMES
    code = pcbp.pc_construct(N, K, R_CRC, POLY)
    gen = torch.Generator(device=dev).manual_seed(777)
    pay = inputs.payload_torch(gen, B, K - R_CRC, dev)
    x = torch.empty((B, N), dtype=torch.uint8, device=dev)
    pcbp.pc_encode(code, pay, x)
    llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(EBN0, K, R_CRC, N)).contiguous()
    del x
    out = {"frames": B, "ebn0_db": EBN0}
    for name, kw in VARIANTS.items():
        max_iters = VARIANT_MAX_ITERS.get(name, MAX_ITERS)
        dec = pcbp.Decoder(code, pcbp.sched(**kw), max_iters, dev)
        for _ in range(max(1, min(warmup, 2))):
            dec(llr)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        dec(llr)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        got = pcbp.unpack_bits(dec.bits, K)[:, : K - R_CRC]
        errors = int((got != pay).any(dim=1).sum().item())
        out[name] = {"gbit_s": B * (K - R_CRC) / (ms / 1e3) / 1e9, "ms": ms, "max_iters": max_iters,
                     "fer": errors / B, "fer_ci95": wilson(errors, B),
                     "mean_iters": float(dec.iters.double().mean().item())}
        if name == "ppbp_boxplus":
            # the first frames, for the FP64 oracle of the CPU-baseline leg
            out["_boxplus_sample"] = {"llr": llr[:BOXPLUS_ORACLE_FRAMES].cpu().numpy(),
                                      "pay": pay[:BOXPLUS_ORACLE_FRAMES].cpu().numpy(),
                                      "bits": got[:BOXPLUS_ORACLE_FRAMES].cpu().numpy(),
                                      "iters": dec.iters[:BOXPLUS_ORACLE_FRAMES].cpu().numpy(), "kw": kw}
    return out


BOXPLUS_ORACLE_FRAMES = 16384


def boxplus_oracle_check(sample, gpu_row):
    """FP64 oracle (exact box-plus) on the first frames of the box-plus variant: its FER and
    Wilson interval beside the GPU's, and the share of frames decided identically."""
    import numpy as np

    import oracle as O

    _, fr = O.construct(N, K)
    B = len(sample["llr"])
    t0 = time.perf_counter()
    u, it, _ = O.decode_batch(fr, R_CRC, POLY, sample["llr"].astype(np.float64), O.Sched(**sample["kw"]), MAX_ITERS,
                              dtype=np.float64)
    secs = time.perf_counter() - t0
    got = O.info_bits(u, fr)[:, : K - R_CRC]
    errs = int((got != sample["pay"]).any(axis=1).sum())
    ci = wilson(errs, B)
    return {"frames": B, "fer": errs / B, "fer_ci95": ci, "seconds": secs, "cores": O.max_threads(),
            "gpu_fer_inside": bool(ci[0] <= gpu_row["fer"] <= ci[1]),
            "identical_decisions": float(np.mean(np.all(got == sample["bits"], axis=1))),
            "identical_iterations": float(np.mean(it == sample["iters"])), "dtype": "f64"}


def wbp_loss(logits, bits):
    import torch

    return torch.nn.functional.binary_cross_entropy_with_logits(-logits, bits.to(logits.dtype))


WBP_ROOF_UNIT = ("per training step: stage passes S = T n + (T-1)(n-1) (the forward's L and R sweeps; the "
                 "backward recomputes them and runs their adjoints), N/2 processing elements each; lane-ops "
                 "= B S (N/2) (8 forward + 8 recomputation + 16 adjoint); HBM bytes = LLRs (forward and "
                 "every backward launch), checkpoints written (T-1) and read (T), gradient planes between "
                 "backward launches read and written (T-1 each), logits and their gradient")


def wbp_roofline(N, K, T, B, seconds):
    """Achieved fraction of the derived ALU issue peak and of the measured HBM bandwidth for one
    weighted-BP training step (algorithmic counts, WBP_ROOF_UNIT)."""
    n = N.bit_length() - 1
    S = T * n + (T - 1) * (n - 1)
    lane_ops = B * S * (N // 2) * (8 + 8 + 16)
    plane = B * (n - 1) * N * 4
    hbm = B * N * 4 * (1 + T) + (T - 1) * plane + T * plane + 2 * (T - 1) * plane + 2 * B * K * 4
    peaks = measured_peaks() or {}
    alu_peak = 152 * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    hbm_peak = peaks.get("hbm_gbs", 6800.0) * 1e9
    fa, fh = lane_ops / seconds / alu_peak, hbm / seconds / hbm_peak
    return {"bound": "alu" if fa >= fh else "hbm", "lane_ops": lane_ops, "tlane_op_s": lane_ops / seconds / 1e12,
            "frac_alu": fa, "hbm_bytes": hbm, "hbm_gbs": hbm / seconds / 1e9, "frac_hbm": fh}


def run_wbp(pcbp, inputs, dev, steps, warmup):
    """Weighted BP fwd+bwd training steps/s at batch 4096 (Eb/N0 uniform on [1, 4] dB, weights
    initialised to 0.9375, BCE on the information bits), and the largest relative error of the FP64
    kernels' gradient against FP64 central finite differences at N = 16 and 64."""
    import torch

    out = {"batch": 4096, "steps_per_s": {}, "ms_per_step": {}, "roofline": {},
           "roofline_unit": WBP_ROOF_UNIT}
    B = 4096
    for N in (256, 1024):
        K = N // 2
        code = pcbp.pc_construct(N, K)
        n = N.bit_length() - 1
        gen = torch.Generator(device=dev).manual_seed(N)
        pay = inputs.payload_torch(gen, B, K, dev)
        x = torch.empty((B, N), dtype=torch.uint8, device=dev)
        pcbp.pc_encode(code, pay, x)
        ebn0 = (1.0 + 3.0 * torch.rand(B, generator=gen, device=dev, dtype=torch.float64)).cpu().numpy()
        llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(ebn0, K, 0, N)).contiguous()
        for T in (5, 10, 20):
            w = torch.full((T, n, N // 2, 4), 0.9375, device=dev, requires_grad=True)

            def step():
                loss = wbp_loss(pcbp.wbp(llr, w, code, T), pay)
                w.grad = None
                loss.backward()

            for _ in range(max(1, warmup)):
                step()
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            reps = max(1, min(steps, 5))
            t0.record()
            for _ in range(reps):
                step()
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / reps
            out["ms_per_step"][f"N{N}_T{T}"] = ms
            out["steps_per_s"][f"N{N}_T{T}"] = 1e3 / ms
            out["roofline"][f"N{N}_T{T}"] = wbp_roofline(N, K, T, B, ms / 1e3)
    # gradient error of the FP64 kernels against central differences
    errs = {}
    for N, T in ((16, 3), (64, 3)):
        K = N // 2
        code = pcbp.pc_construct(N, K)
        n = N.bit_length() - 1
        gen = torch.Generator(device=dev).manual_seed(3 * N)
        Bc = 8
        pay = inputs.payload_torch(gen, Bc, K, dev)
        x = torch.empty((Bc, N), dtype=torch.uint8, device=dev)
        pcbp.pc_encode(code, pay, x)
        llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(1.5, K, 0, N)).double().contiguous()
        w = (0.9375 + 0.05 * torch.randn((T, n, N // 2, 4), generator=gen, device=dev, dtype=torch.float64))
        w.requires_grad_()
        wbp_loss(pcbp.wbp(llr, w, code, T), pay).backward()
        g = w.grad.flatten()
        idx = torch.argsort(g.abs(), descending=True)[:32]
        eps, worst = 1e-6, 0.0
        with torch.no_grad():
            for i in idx.tolist():
                wp = w.detach().clone().flatten()
                wm = wp.clone()
                wp[i] += eps
                wm[i] -= eps
                lp = wbp_loss(pcbp.wbp(llr, wp.view_as(w), code, T), pay)
                lm = wbp_loss(pcbp.wbp(llr, wm.view_as(w), code, T), pay)
                fd = float((lp - lm) / (2 * eps))
                worst = max(worst, abs(fd - float(g[i])) / max(abs(fd), 1e-12))
        errs[f"N{N}"] = worst
    out["grad_max_rel_err_vs_fd64"] = errs
    out["grad_check"] = "32 largest-gradient weights, central differences eps 1e-6, FP64 kernels, T=3, batch 8"
    out["train"] = run_wbp_train(pcbp, inputs, dev)
    return out


def run_wbp_train(pcbp, inputs, dev, N=256, T=5, steps=400, lr=2e-3):
    """Trains the per-edge weights (Adam, BCE) on fresh encoder + channel frames every step (batch
    4096, Eb/N0 uniform on [1, 4] dB), then compares FER on held-out frames with the fixed-scale
    decoder: bp_decode, plain BP, alpha = 0.9375, exactly T iterations (no early stop)."""
    import torch

    K = N // 2
    n = N.bit_length() - 1
    B = 4096
    code = pcbp.pc_construct(N, K)
    gen = torch.Generator(device=dev).manual_seed(2024)

    def frames(count, ebn0=None):
        pay = inputs.payload_torch(gen, count, K, dev)
        x = torch.empty((count, N), dtype=torch.uint8, device=dev)
        pcbp.pc_encode(code, pay, x)
        if ebn0 is None:
            e = (1.0 + 3.0 * torch.rand(count, generator=gen, device=dev, dtype=torch.float64)).cpu().numpy()
        else:
            e = ebn0
        return pay, inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(e, K, 0, N)).contiguous()

    w = torch.full((T, n, N // 2, 4), 0.9375, device=dev, requires_grad=True)
    opt = torch.optim.Adam([w], lr=lr)
    losses = []
    t0 = time.perf_counter()
    for _ in range(steps):
        pay, llr = frames(B)
        loss = wbp_loss(pcbp.wbp(llr, w, code, T), pay)
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss.item()))
    train_s = time.perf_counter() - t0
    fixed_dec = pcbp.Decoder(code, pcbp.sched(mode=0, stop_kind=0, alpha=0.9375), T, dev)
    test = {}
    for ebn0 in (2.0, 3.0, 4.0):
        errs_w = errs_f = total = 0
        for _ in range(16):
            pay, llr = frames(B, ebn0)
            with torch.no_grad():
                logits = pcbp.wbp(llr, w.detach(), code, T)
            got_w = (logits < 0).to(torch.uint8)
            bits, _, _ = fixed_dec(llr)
            got_f = pcbp.unpack_bits(bits, K)
            errs_w += int((got_w != pay).any(dim=1).sum().item())
            errs_f += int((got_f != pay).any(dim=1).sum().item())
            total += B
        test[f"{ebn0:.1f}dB"] = {"frames": total, "fer_trained": errs_w / total, "fer_fixed_alpha": errs_f / total,
                                 "ci95_trained": wilson(errs_w, total), "ci95_fixed_alpha": wilson(errs_f, total)}
    return {"N": N, "K": K, "T": T, "steps": steps, "batch": B, "optimizer": f"Adam lr {lr}",
            "loss_first10": sum(losses[:10]) / 10, "loss_last10": sum(losses[-10:]) / 10,
            "train_seconds": train_s, "test": test}


def run_ours(args):
    import numpy as np
    import torch

    from paper_1911_08868_gb300 import _build

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    from paper_1911_08868_gb300 import inputs, pcbp

    from paper_1911_08868_gb300.shard import reduce_counters, shard_range

    B = args.frames                       # frames per rank (weak scaling)
    lo, hi = shard_range(world * B, world, rank)
    code = pcbp.pc_construct(N, K, R_CRC, POLY)
    sch = pcbp.sched(**SCHED, frame_base=lo)
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    pay = inputs.payload_torch(gen, B, K - R_CRC, dev)
    x = torch.empty((B, N), dtype=torch.uint8, device=dev)
    pcbp.pc_encode(code, pay, x)
    llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(EBN0, K, R_CRC, N)).contiguous()
    del x
    torch.cuda.synchronize()
    dec = pcbp.Decoder(code, sch, MAX_ITERS, dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        dec(llr)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        t_all0.record(stream)
        for i in range(args.steps):
            starts[i].record(stream)
            dec(llr)
            ends[i].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = t_all0.elapsed_time(t_all1)
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    # outcome of the decode (identical every step)
    iters = dec.iters.to(torch.int64)
    ok = dec.crc_ok.to(torch.int64)
    got = pcbp.unpack_bits(dec.bits, K)[:, : K - R_CRC]
    frame_err = (got != pay).any(dim=1)
    job = reduce_counters({"frames": B, "frame_errors": int(frame_err.sum().item()),
                           "bit_errors": int((got != pay).sum().item()), "iterations": int(iters.sum().item())})
    errors = job["frame_errors"]
    mean_iters = job["iterations"] / job["frames"]
    half_sweeps = int((2 * iters - ok).sum().item())   # a CRC stop skips that iteration's R sweep
    info_bits = B * (K - R_CRC)
    value = world * info_bits * args.steps / (total_ms / 1e3) / 1e9

    # roofline: plain-ALU bound.  Per PE and half sweep: 2 f (min, scale,
    # sign) + 2 adds = 8 lane-ops; a half sweep has n N / 2 PEs.
    n = N.bit_length() - 1
    lane_ops = half_sweeps * (n * N // 2) * 8
    mean_launch_s = statistics.mean(launch_ms) / 1e3
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_mhz_max = (peaks or {}).get("sm_max_mhz", 2070.0)
    peak_ops = props.multi_processor_count * 128 * sm_mhz_max * 1e6
    achieved = lane_ops / mean_launch_s
    sha = kernel_sha()
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tlane-op/s",
            "frac": achieved / peak_ops, "traffic": (None if profiled_traffic(sha) is None else profiled_traffic(sha) * B / FRAMES),
            "algorithmic_bytes": B * N * 4 + B * (4 * math.ceil(K / 32) + 5),
            "hbm_gbs": (B * N * 4 + B * (4 * math.ceil(K / 32) + 5)) / mean_launch_s / 1e9,
            "peak_source": ("issue rate 128 lanes/clk/SM x %d SMs x %.0f MHz (MEASURED_PEAKS sm_max_mhz)"
                            % (props.multi_processor_count, sm_mhz_max)),
            "kernel_sha": sha}

    clocks = clk.summary()
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step_per_gpu": B, "N": N, "K": K, "crc": R_CRC,
                       "ebn0_db": EBN0, "max_iters": MAX_ITERS,
                       "l2": "inputs larger than L2 (%.1f GB of LLRs per step)" % (B * N * 4 / 1e9),
                       "parallelism": f"frame shards x{world}"},
            "frames_per_s": world * B * args.steps / (total_ms / 1e3),
            "mean_iters": mean_iters, "fer": errors / job["frames"], "fer_ci95": wilson(errors, job["frames"]),
            "ber": job["bit_errors"] / (job["frames"] * (K - R_CRC)),
            "roofline": roof, "gpu_launches": args.steps, "clocks": clocks,
        }

    if not args.no_e2e:
        hdec = pcbp.HostDecoder(code, sch, MAX_ITERS, dev)
        h_llr = torch.empty((B, N), dtype=torch.float32, pin_memory=True)
        h_llr.copy_(llr)
        del llr
        torch.cuda.empty_cache()
        hdec(h_llr)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e_steps = max(1, min(args.steps, 5))
        for _ in range(e_steps):
            hb, hi, ho = hdec(h_llr)
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        if rank == 0:
            same = bool(torch.equal(hi, dec.iters.cpu()))
            line["e2e"] = {"value": world * info_bits * e_steps / el / 1e9, "unit": "Gbit/s",
                           "h2d_bytes_per_step": B * N * 4,
                           "d2h_bytes_per_step": B * (4 * math.ceil(K / 32) + 4 + 1), "steps": e_steps,
                           "path": "bp_decode_host: the kernel reads the page-locked host LLRs and writes the "
                                   "results into page-locked host memory across the host-device link",
                           "matches_device_run": same}

    if rank == 0 and not args.no_wbp:
        line["wbp"] = run_wbp(pcbp, inputs, dev, args.steps, args.warmup)

    boxplus_sample = None
    if rank == 0 and not args.no_variants:
        line["variants"] = run_variants(pcbp, inputs, dev, args.warmup)
        boxplus_sample = line["variants"].pop("_boxplus_sample", None)

    if rank == 0 and not args.no_mixed:
        del dec
        torch.cuda.empty_cache()
        line["mixed"] = run_mixed(pcbp, inputs, dev, args.steps, args.warmup)

    if rank == 0 and not args.no_cpu:
        cb = cpu_oracle(args.cpu_seconds)
        cb1 = cpu_oracle(min(3.0, args.cpu_seconds), seed=197, threads=1)
        line["cpu_baseline"] = {"value": cb["gbps"], "unit": "Gbit/s", "cores": cb["cores"], "kind": "oracle",
                                "sample": f"{cb['frames']} frames of the same workload (fresh seeds), "
                                          f"{cb['seconds']:.1f} s",
                                "fer": cb["fer"], "fer_ci95": wilson(cb["errors"], cb["frames"]),
                                "mean_iters": cb["mean_iters"],
                                "value_1core": cb1["gbps"],
                                "sample_1core": f"{cb1['frames']} frames, {cb1['seconds']:.1f} s on 1 core"}
        if boxplus_sample is not None:
            line["variants"]["ppbp_boxplus"]["oracle"] = boxplus_oracle_check(boxplus_sample,
                                                                             line["variants"]["ppbp_boxplus"])
        lo, hi_ = line["cpu_baseline"]["fer_ci95"]
        line["fer_matched"] = bool(lo <= line["fer"] <= hi_ or line["fer_ci95"][0] <= cb["fer"] <= line["fer_ci95"][1])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if needs_spawn(args.gpus):
        sys.exit(spawn_ranks(args.gpus, str(Path(__file__).resolve()), sys.argv[1:]))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
