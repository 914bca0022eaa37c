"""ctypes wrapper of the oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain CPU restatement of arXiv 1911.08868 (polar code
construction, CRC, encoding and partially permuted multi-trellis BP) used to
check the CUDA decoder.  Only tests/, ``__graft_entry__.smoke`` and the CPU
baseline of ``bench.py`` may import it; the product package never does.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(str(path))
        u8p, i8p = C.POINTER(C.c_uint8), C.POINTER(C.c_int8)
        f32p, f64p, i32p = C.POINTER(C.c_float), C.POINTER(C.c_double), C.POINTER(C.c_int32)
        L.orc_construct.argtypes = [C.c_int, C.c_int, C.c_double, f64p, u8p]
        L.orc_crc_residue.argtypes = [u8p, C.c_int, C.c_int, C.c_uint64]
        L.orc_crc_residue.restype = C.c_uint64
        L.orc_crc_compute.argtypes = [u8p, C.c_int, C.c_int, C.c_uint64]
        L.orc_crc_compute.restype = C.c_uint64
        L.orc_encode.argtypes = [C.c_int, u8p, u8p]
        L.orc_place_info.argtypes = [C.c_int, u8p, u8p, u8p]
        L.orc_graph_encode.argtypes = [C.c_int, i8p, u8p, u8p]
        L.orc_graph_from_event.argtypes = [C.c_int, C.c_void_p, i8p]
        L.orc_splitmix.argtypes = [C.c_uint64]
        L.orc_splitmix.restype = C.c_uint64
        L.orc_hash.argtypes = [C.c_uint64] * 4
        L.orc_hash.restype = C.c_uint64
        L.orc_draw_event.argtypes = [C.c_int, C.c_void_p, C.c_uint64, C.c_int, C.c_void_p]
        L.orc_n_zero.argtypes = [C.c_void_p]
        L.orc_n_zero.restype = C.c_int64
        L.orc_reset_increment.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_f_f64.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
        L.orc_f_f64.restype = C.c_double
        L.orc_f_f32.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int]
        L.orc_f_f32.restype = C.c_float
        L.orc_bp_iteration_f64.argtypes = [C.c_int, i8p, f64p, f64p, C.c_double, C.c_int]
        L.orc_bp_iteration_f32.argtypes = [C.c_int, i8p, f32p, f32p, C.c_float, C.c_int]
        for sfx, fp in (("f64", f64p), ("f32", f32p)):
            fn = getattr(L, f"orc_decode_{sfx}")
            fn.argtypes = [C.c_int, u8p, C.c_int, C.c_uint64, fp, C.c_void_p, C.c_int, C.c_uint64,
                           C.c_void_p, C.c_int, u8p, i32p, i32p, fp]
            fb = getattr(L, f"orc_decode_batch_{sfx}")
            fb.argtypes = [C.c_int, u8p, C.c_int, C.c_uint64, fp, C.c_void_p, C.c_int, C.c_int64, C.c_int,
                           u8p, i32p, i32p]
        L.orc_max_threads.restype = C.c_int
        _LIB = L
    return _LIB


class Event(C.Structure):
    _fields_ = [("level", C.c_int32), ("range", C.c_int32), ("block", C.c_int64), ("order", C.c_int32 * 16)]

    @staticmethod
    def make(level: int, range_: int, block: int, order) -> "Event":
        ev = Event()
        ev.level, ev.range, ev.block = level, range_, block
        for i in range(16):
            ev.order[i] = order[i] if i < len(order) else i
        return ev

    def as_tuple(self):
        return (self.level, self.range, self.block, tuple(self.order[: self.range]))


class _Sched(C.Structure):
    _fields_ = [(name, C.c_int32) for name in (
        "mode", "P_range", "P_level", "N_min", "D", "T0", "rho_range_fixed",
        "q_max", "it_reset_full", "stop_from", "stop_kind", "fkind")] + [
        ("alpha", C.c_double), ("seed", C.c_uint64), ("frame_base", C.c_uint64)]


@dataclass
class Sched:
    """Decoder schedule; the same fields as the library's pc_sched."""
    mode: int = 0
    P_range: int = 2
    P_level: int = 1
    N_min: int = 1
    D: int = 0
    T0: int = 1
    rho_range_fixed: int = 0
    q_max: int = 0
    it_reset_full: int = 0
    stop_from: int = 1
    stop_kind: int = 1
    fkind: int = 0
    alpha: float = 0.9375
    seed: int = 0
    frame_base: int = 0

    def c(self) -> _Sched:
        s = _Sched()
        for name, _ in _Sched._fields_:
            setattr(s, name, getattr(self, name))
        return s


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint8))


def construct(N: int, K: int, design_ebn0_db: float = 0.0):
    """(log Bhattacharyya bounds, frozen mask) of the length-N, K-information code."""
    n = N.bit_length() - 1
    lz = np.zeros(N, dtype=np.float64)
    fr = np.zeros(N, dtype=np.uint8)
    rc = lib().orc_construct(n, K, design_ebn0_db, lz.ctypes.data_as(C.POINTER(C.c_double)),
                             fr.ctypes.data_as(C.POINTER(C.c_uint8)))
    if rc:
        raise ValueError("orc_construct failed")
    return lz, fr


def crc_residue(bits, r: int, poly: int) -> int:
    a, p = _u8(bits)
    return int(lib().orc_crc_residue(p, len(a), r, poly))


def crc_compute(payload, r: int, poly: int) -> int:
    a, p = _u8(payload)
    return int(lib().orc_crc_compute(p, len(a), r, poly))


def crc_bits(payload, r: int, poly: int) -> np.ndarray:
    """payload || CRC(payload), CRC most significant bit first."""
    c = crc_compute(payload, r, poly)
    tail = np.array([(c >> (r - 1 - i)) & 1 for i in range(r)], dtype=np.uint8)
    return np.concatenate([np.asarray(payload, dtype=np.uint8), tail])


def encode(u) -> np.ndarray:
    a, p = _u8(u)
    n = len(a).bit_length() - 1
    x = np.zeros_like(a)
    lib().orc_encode(n, p, x.ctypes.data_as(C.POINTER(C.c_uint8)))
    return x


def place_info(frozen, info) -> np.ndarray:
    fr, pf = _u8(frozen)
    inf, pi = _u8(info)
    u = np.zeros_like(fr)
    lib().orc_place_info(len(fr).bit_length() - 1, pf, pi, u.ctypes.data_as(C.POINTER(C.c_uint8)))
    return u


def encode_frames(payload: np.ndarray, frozen: np.ndarray, r: int, poly: int) -> np.ndarray:
    """Codewords x for a batch of payload rows (payload || CRC on the info positions)."""
    out = np.zeros((payload.shape[0], len(frozen)), dtype=np.uint8)
    for b in range(payload.shape[0]):
        a = crc_bits(payload[b], r, poly) if r > 0 else np.asarray(payload[b], dtype=np.uint8)
        out[b] = encode(place_info(frozen, a))
    return out


def graph_from_event(n: int, ev: Event | None = None) -> np.ndarray:
    sb = np.zeros((n, 1 << n), dtype=np.int8)
    lib().orc_graph_from_event(n, C.byref(ev) if ev is not None else None,
                               sb.ctypes.data_as(C.POINTER(C.c_int8)))
    return sb


def graph_encode(n: int, stage_bit: np.ndarray, u) -> np.ndarray:
    sb = np.ascontiguousarray(stage_bit, dtype=np.int8)
    a, p = _u8(u)
    x = np.zeros_like(a)
    rc = lib().orc_graph_encode(n, sb.ctypes.data_as(C.POINTER(C.c_int8)), p, x.ctypes.data_as(C.POINTER(C.c_uint8)))
    if rc:
        raise ValueError("invalid stage table")
    return x


def splitmix(state: int) -> int:
    return int(lib().orc_splitmix(state))


def hash64(seed: int, frame: int, k: int, d: int) -> int:
    return int(lib().orc_hash(seed, frame, k, d))


def draw_event(n: int, sched: Sched, frame_id: int, k: int) -> Event:
    ev = Event()
    s = sched.c()
    if lib().orc_draw_event(n, C.byref(s), frame_id, k, C.byref(ev)):
        raise ValueError("invalid schedule for draw_event")
    return ev


def n_zero(ev: Event) -> int:
    return int(lib().orc_n_zero(C.byref(ev)))


def reset_increment(sched: Sched, ev: Event) -> int:
    s = sched.c()
    return int(lib().orc_reset_increment(C.byref(s), C.byref(ev)))


def f(a: float, b: float, alpha: float = 1.0, fkind: int = 0, dtype=np.float64):
    if dtype == np.float32:
        return np.float32(lib().orc_f_f32(np.float32(a), np.float32(b), np.float32(alpha), fkind))
    return float(lib().orc_f_f64(a, b, alpha, fkind))


def bp_iteration(n: int, stage_bit: np.ndarray, L: np.ndarray, R: np.ndarray, alpha: float = 1.0,
                 fkind: int = 0):
    """One round-trip iteration on explicit planes [(n+1), N] (modified in place)."""
    sb = np.ascontiguousarray(stage_bit, dtype=np.int8)
    if L.dtype == np.float32:
        lib().orc_bp_iteration_f32(n, sb.ctypes.data_as(C.POINTER(C.c_int8)),
                                   L.ctypes.data_as(C.POINTER(C.c_float)), R.ctypes.data_as(C.POINTER(C.c_float)),
                                   alpha, fkind)
    else:
        lib().orc_bp_iteration_f64(n, sb.ctypes.data_as(C.POINTER(C.c_int8)),
                                   L.ctypes.data_as(C.POINTER(C.c_double)), R.ctypes.data_as(C.POINTER(C.c_double)),
                                   alpha, fkind)


@dataclass
class DecodeResult:
    uhat: np.ndarray
    iters: int
    crc_ok: int
    dump: np.ndarray | None = field(default=None)


def decode(frozen: np.ndarray, r: int, poly: int, llr: np.ndarray, sched: Sched, max_iters: int,
           frame_id: int = 0, events: list[Event] | None = None, dump: bool = False,
           dtype=np.float32) -> DecodeResult:
    """Algorithm 1 on one frame; dump -> [max_iters, 2, n+1, N] planes after each iteration."""
    N = len(frozen)
    n = N.bit_length() - 1
    fr, pf = _u8(frozen)
    ctype = C.c_float if dtype == np.float32 else C.c_double
    x = np.ascontiguousarray(llr, dtype=dtype)
    uhat = np.zeros(N, dtype=np.uint8)
    it = C.c_int32(0)
    ok = C.c_int32(0)
    d = np.full((max(max_iters, 1), 2, n + 1, N), np.nan, dtype=dtype) if dump else None
    evs = (Event * len(events))(*events) if events else None
    fn = lib().orc_decode_f32 if dtype == np.float32 else lib().orc_decode_f64
    s = sched.c()
    rc = fn(n, pf, r, poly, x.ctypes.data_as(C.POINTER(ctype)), C.byref(s), max_iters, frame_id,
            evs, len(events) if events else 0, uhat.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(it),
            C.byref(ok), d.ctypes.data_as(C.POINTER(ctype)) if d is not None else None)
    if rc:
        raise ValueError("orc_decode failed")
    return DecodeResult(uhat, it.value, ok.value, d)


def decode_batch(frozen: np.ndarray, r: int, poly: int, llr: np.ndarray, sched: Sched, max_iters: int,
                 nthreads: int = 0, dtype=np.float32):
    """Frame loop (OpenMP): returns (uhat [B, N], iters [B], crc_ok [B])."""
    N = len(frozen)
    n = N.bit_length() - 1
    fr, pf = _u8(frozen)
    ctype = C.c_float if dtype == np.float32 else C.c_double
    x = np.ascontiguousarray(llr, dtype=dtype).reshape(-1, N)
    B = x.shape[0]
    uhat = np.zeros((B, N), dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int32)
    ok = np.zeros(B, dtype=np.int32)
    fn = lib().orc_decode_batch_f32 if dtype == np.float32 else lib().orc_decode_batch_f64
    s = sched.c()
    rc = fn(n, pf, r, poly, x.ctypes.data_as(C.POINTER(ctype)), C.byref(s), max_iters, B, nthreads,
            uhat.ctypes.data_as(C.POINTER(C.c_uint8)), iters.ctypes.data_as(C.POINTER(C.c_int32)),
            ok.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc:
        raise ValueError("orc_decode_batch failed")
    return uhat, iters, ok


def max_threads() -> int:
    return int(lib().orc_max_threads())


def info_bits(uhat: np.ndarray, frozen: np.ndarray) -> np.ndarray:
    """Decided information vector(s): the non-frozen positions in ascending order."""
    return uhat[..., frozen == 0]
