"""Builds the oracle (TEST INFRASTRUCTURE ONLY) as oracle/liboracle.so.

Plain gcc, C11, -O2 with -ffp-contract=off so that each FP32/FP64 operation
is rounded where it is written, and OpenMP for the frame loop.
"""
from __future__ import annotations

import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
LIB = HERE / "liboracle.so"
SRCS = [HERE / "pcbp_oracle.c"]
DEPS = SRCS + [HERE / "pcbp_oracle.h", HERE / "bp_real.inc", Path(__file__)]


def build(force: bool = False) -> Path:
    if not force and LIB.exists() and all(d.stat().st_mtime <= LIB.stat().st_mtime for d in DEPS):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           *map(str, SRCS), "-o", str(LIB), "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"oracle build failed:\n{res.stdout}\n{res.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force=True))
