"""Builds libpcbp.so in-tree with nvcc for sm_103a (no cmake, no setuptools).

The decoder kernels are instantiated once per code length from
``csrc/bp_inst.cu`` and ``csrc/bp_inst2.cu`` (n = 3..11) and
``csrc/bp_inst3.cu`` (n = 7..11); those translation units compile in
parallel.  Objects go
to ``_build/`` at the repository root; the library is written next to this
file.  A rebuild only recompiles objects older than their sources or any
header.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
CHECKED = os.environ.get("PCBP_CHECKED") == "1"   # bounds-checked decoder (debug build)
BUILD = ROOT / ("_build_checked" if CHECKED else "_build")
LIB = PKG / "libpcbp.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
LOGNS = range(3, 12)
LOGNS_TMEM = range(7, 12)    # the TMEM kernel needs 2^KB positions on every lane of a warp


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpcbp")
    return cand


def _headers() -> list[Path]:
    return sorted(CSRC.glob("*.h")) + sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def _stale(obj: Path, src: Path) -> bool:
    if not obj.exists():
        return True
    t = obj.stat().st_mtime
    return any(p.stat().st_mtime > t for p in [src, *_headers(), Path(__file__)])


def _jobs() -> list[tuple[Path, Path, list[str]]]:
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
              f"-I{INCLUDE}", f"-I{CSRC}", *(["-DPCBP_CHECKED"] if CHECKED else [])]
    jobs = []
    for n in LOGNS:
        obj = BUILD / f"bp_inst_{n}.o"
        jobs.append((obj, CSRC / "bp_inst.cu", [*common, f"-DPCBP_LOGN={n}", "-c", str(CSRC / "bp_inst.cu"),
                                                "-o", str(obj)]))
    kb = os.environ.get("PCBP_KB")      # register-group width override (2^KB positions per thread)
    for n in LOGNS:
        obj = BUILD / (f"bp_inst2_{n}_kb{int(kb)}.o" if kb else f"bp_inst2_{n}.o")
        extra = [f"-DPCBP_KB={int(kb)}"] if kb else []
        jobs.append((obj, CSRC / "bp_inst2.cu", [*common, f"-DPCBP_LOGN={n}", *extra, "-c",
                                                 str(CSRC / "bp_inst2.cu"), "-o", str(obj)]))
    kb3 = os.environ.get("PCBP_KB3")    # the same override for the tensor-memory kernel, for the
    kb3_logn = os.environ.get("PCBP_KB3_LOGN")   # lengths where a warp still owns 32 x 2^KB positions
    for n in LOGNS_TMEM:                         # (and only log2 N in PCBP_KB3_LOGN, when given)
        use = kb3 is not None and n - int(kb3) >= 5 and (not kb3_logn or str(n) in kb3_logn.split(","))
        obj = BUILD / (f"bp_inst3_{n}_kb{int(kb3)}.o" if use else f"bp_inst3_{n}.o")
        extra = [f"-DPCBP_KB3={int(kb3)}"] if use else []
        jobs.append((obj, CSRC / "bp_inst3.cu", [*common, f"-DPCBP_LOGN={n}", *extra, "-c",
                                                 str(CSRC / "bp_inst3.cu"), "-o", str(obj)]))
    for name in ("bp_decode.cu", "bp_decode_static.cu", "bp_selfcheck.cu", "wbp.cu"):
        obj = BUILD / (Path(name).stem + ".o")
        jobs.append((obj, CSRC / name, [*common, "-c", str(CSRC / name), "-o", str(obj)]))
    for name in ("pcbp_host.cpp",):
        obj = BUILD / (Path(name).stem + ".o")
        jobs.append((obj, CSRC / name, [*common, "-x", "cu", "-c", str(CSRC / name), "-o", str(obj)]))
    return jobs


def build(verbose: bool = False, force: bool = False) -> Path:
    """Compile (as needed) and link libpcbp.so; returns its path."""
    BUILD.mkdir(exist_ok=True)
    jobs = _jobs()
    todo = [j for j in jobs if force or _stale(j[0], j[1])]

    def run(job):
        obj, _, cmd = job
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"compile failed for {obj.name}:\n{res.stdout}\n{res.stderr}")
        return res.stderr

    if todo:
        workers = max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(workers) as ex:
            for msg in ex.map(run, todo):
                if verbose and msg:
                    print(msg)
    objs = [str(j[0]) for j in jobs]
    stamp = LIB.with_name(LIB.name + ".inputs")   # relink when the set of objects changes (checked <-> normal)
    same_set = stamp.exists() and stamp.read_text() == "\n".join(objs)
    if (force or todo or not same_set or not LIB.exists()
            or any(Path(o).stat().st_mtime > LIB.stat().st_mtime for o in objs)):
        cmd = [_nvcc(), *ARCH, "-shared", "-o", str(LIB), *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        stamp.write_text("\n".join(objs))
    return LIB


if __name__ == "__main__":
    import sys

    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
