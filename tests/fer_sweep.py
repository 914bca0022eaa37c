"""FER curves of the decoder against the oracle (verification; not a test pytest collects).

PP-BP grid (s in {3, 4, 5}, T in {5, 10, 20}), FP-BP (10 orders of 100 iterations) and plain BP at
Eb/N0 1.5 .. 4.0 dB on the benchmark code (N = 1024, K = 512, CRC-24), 1,000,000 frames per point
on the GPU; for the benchmark schedule and FP-BP the oracle decodes the first frames of every point
too (same frame ids), and the JSON line reports its FER interval and whether its decisions and
iteration counts equal the GPU's.  Run on a GB300:

    python tests/fer_sweep.py [--frames 1000000] [--n 1024|512|2048] [--oracle-frames 4096]
"""
import argparse
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402

SWEEP_EBN0 = tuple(1.5 + 0.25 * i for i in range(11))
SWEEP_SCHEDULES = {f"ppbp_s{s_}_t{t_}": dict(mode=1, rho_range_fixed=s_, P_level=9, N_min=t_, D=0, T0=t_, stop_from=1,
                                             stop_kind=1, alpha=0.9375, seed=3)
                   for s_ in (3, 4, 5) for t_ in (5, 10, 20)}
SWEEP_SCHEDULES["fpbp_q10_t100"] = bench.VARIANTS["fpbp_q10_t100"]
SWEEP_SCHEDULES["plain_bp"] = bench.VARIANTS["plain_bp"]
SWEEP_ORACLE = ("ppbp_s4_t10", "fpbp_q10_t100")


def run_sweep(args):
    """FER and mean iterations of the PP-BP grid (s in {3,4,5}, T in {5,10,20}), FP-BP and plain BP
    at Eb/N0 1.5..4.0 dB on the benchmark code; for the benchmark schedule and FP-BP, the oracle
    decodes the first frames of every point too (same frame ids): its FER interval, and whether its
    decisions and iteration counts equal the GPU's on those frames."""
    import numpy as np
    import torch

    import oracle as O
    from paper_1911_08868_gb300 import _build

    _build.build()
    from paper_1911_08868_gb300 import inputs, pcbp

    dev = torch.device("cuda", 0)
    B, Bo = args.frames, args.oracle_frames
    N, K = args.n, args.n // 2          # the sweep's code (the benchmark code by default)
    n = N.bit_length() - 1
    schedules = {k: dict(v) for k, v in SWEEP_SCHEDULES.items()}
    if N != 1024:
        schedules = {k: v for k, v in schedules.items() if k in ("ppbp_s4_t10", "fpbp_q10_t100", "plain_bp")}
    for v in schedules.values():
        if v.get("mode") == 1:
            v["P_level"] = n - 1
    code = pcbp.pc_construct(N, K, bench.R_CRC, bench.POLY)
    _, fr = O.construct(N, K)
    threads = O.max_threads()
    rows = []
    for ebn0 in SWEEP_EBN0:
        gen = torch.Generator(device=dev).manual_seed(5000 + int(round(ebn0 * 100)))
        pay = inputs.payload_torch(gen, B, K - bench.R_CRC, dev)
        x = torch.empty((B, N), dtype=torch.uint8, device=dev)
        pcbp.pc_encode(code, pay, x)
        llr = inputs.bpsk_awgn_llr_torch(x, gen, inputs.sigma2_of(ebn0, K, bench.R_CRC, N)).contiguous()
        del x
        sub_llr = llr[:Bo].cpu().numpy()
        sub_pay = pay[:Bo].cpu().numpy()
        for name, kw in schedules.items():
            max_iters = bench.VARIANT_MAX_ITERS.get(name, bench.MAX_ITERS)
            dec = pcbp.Decoder(code, pcbp.sched(**kw), max_iters, dev)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            dec(llr)
            t1.record()
            torch.cuda.synchronize()
            got = pcbp.unpack_bits(dec.bits, K)[:, : K - bench.R_CRC]
            errors = int((got != pay).any(dim=1).sum().item())
            row = {"schedule": name, "ebn0_db": ebn0, "frames": B, "fer": errors / B, "errors": errors,
                   "fer_ci95": bench.wilson(errors, B), "mean_iters": float(dec.iters.double().mean().item()),
                   "gbit_s": B * (K - bench.R_CRC) / (t0.elapsed_time(t1) / 1e3) / 1e9}
            if name in SWEEP_ORACLE:
                os_ = O.Sched(**kw)
                u, it, ok = O.decode_batch(fr, bench.R_CRC, bench.POLY, sub_llr, os_, max_iters, nthreads=threads)
                ogot = O.info_bits(u, fr)[:, : K - bench.R_CRC]
                oerr = int((ogot != sub_pay).any(axis=1).sum())
                oci = bench.wilson(oerr, Bo)
                gsub = got[:Bo].cpu().numpy()
                gits = dec.iters[:Bo].cpu().numpy()
                row["oracle"] = {"frames": Bo, "fer": oerr / Bo, "fer_ci95": oci, "mean_iters": float(it.mean()),
                                 "identical_decisions": bool(np.array_equal(ogot, gsub)),
                                 "identical_iterations": bool(np.array_equal(it, gits)),
                                 "intervals_overlap": bool(oci[0] <= row["fer_ci95"][1] and row["fer_ci95"][0] <= oci[1])}
            rows.append(row)
        del llr, pay
    print(json.dumps({"sweep": rows, "code": f"N={N} K={K} CRC-24 (0x1B2B117)", "data": "synthetic BPSK/AWGN",
                      "oracle_cores": threads, "dtype": "f32"}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--frames", type=int, default=1_000_000)
    ap.add_argument("--n", type=int, default=1024, choices=(512, 1024, 2048),
                    help="code length (K = N/2, CRC-24); N != 1024 runs the s=4 T=10 PP-BP, FP-BP and plain BP "
                         "schedules only")
    ap.add_argument("--oracle-frames", type=int, default=4096)
    run_sweep(ap.parse_args())


if __name__ == "__main__":
    main()
