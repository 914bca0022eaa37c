"""Thin ctypes binding of libpcbp.so (include/pcbp.h): argument marshalling only.

Every function has the C name and forwards device pointers of torch CUDA
tensors; all decoding work runs in the library's kernels.  Importing this
module raises ImportError when libpcbp.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "libpcbp.so"
if not _LIB_PATH.exists():
    raise ImportError(f"{_LIB_PATH} is not built; run `python -m paper_1911_08868_gb300._build` "
                      "(needs nvcc) — the decoder has no CPU fallback")
_lib = C.CDLL(str(_LIB_PATH))

PC_OK, PC_EINVAL, PC_ENOMEM, PC_ECUDA, PC_ETIMEOUT, PC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
PC_NMAX = 2048
PC_MAX_EVENTS = 32

EXPORTED = ("pc_construct", "pc_encode", "bp_decode_workspace_size", "bp_decode", "bp_decode_host", "bp_decode_trace",
            "bp_decode_posterior", "pc_f_eval",
            "bp_decode_noalloc", "pc_partition_selfcheck", "pc_build_info", "bp_kernel_threads", "bp_slot_limit",
            "bp_mixed_table_size", "bp_mixed_prepare", "bp_mixed_workspace_size", "bp_decode_mixed",
            "wbp_weights_count", "wbp_ckpt_count", "wbp_workspace_size", "wbp_forward", "wbp_backward",
            "wbp_forward_f64", "wbp_backward_f64", "pc_status_string")
PC_MAX_BATCHES = 64
PC_STATIC_SCRATCH_BYTES = 4096


class PcCode(C.Structure):
    _fields_ = [("N", C.c_int32), ("n", C.c_int32), ("K", C.c_int32), ("crc_len", C.c_int32),
                ("crc_poly", C.c_uint64), ("frozen_mask", C.c_uint32 * (PC_NMAX // 32)),
                ("info_idx", C.c_int32 * PC_NMAX)]

    def frozen(self):
        return [(self.frozen_mask[j >> 5] >> (j & 31)) & 1 for j in range(self.N)]

    def info_positions(self):
        return [self.info_idx[k] for k in range(self.K)]


class PcSched(C.Structure):
    _fields_ = [(name, C.c_int32) for name in (
        "mode", "P_range", "P_level", "N_min", "D", "T0", "rho_range_fixed",
        "q_max", "it_reset_full", "stop_from", "stop_kind", "fkind")] + [
        ("alpha", C.c_float), ("reserved", C.c_int32), ("seed", C.c_uint64), ("frame_base", C.c_uint64)]


class PcEvent(C.Structure):
    _fields_ = [("level", C.c_int32), ("range", C.c_int32), ("block", C.c_int64), ("order", C.c_int32 * 16)]


class PcBatch(C.Structure):
    _fields_ = [("code", C.POINTER(PcCode)), ("sched", PcSched), ("max_iters", C.c_int32), ("slots", C.c_int32),
                ("threads_per_frame", C.c_int32), ("reserved", C.c_int32), ("B", C.c_int64), ("d_llr", C.c_void_p),
                ("d_bits", C.c_void_p), ("d_iters", C.c_void_p), ("d_crc_ok", C.c_void_p)]


_vp = C.c_void_p
_lib.pc_construct.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_double, C.POINTER(PcCode)]
_lib.pc_encode.argtypes = [C.POINTER(PcCode), _vp, _vp, C.c_int64, _vp]
_lib.bp_decode_workspace_size.argtypes = [C.POINTER(PcCode), C.c_int64, C.POINTER(C.c_size_t)]
_lib.bp_decode.argtypes = [C.POINTER(PcCode), _vp, C.POINTER(PcSched), C.c_int32, C.c_int64, _vp, _vp, _vp, _vp,
                           _vp]
_lib.bp_decode_host.argtypes = [C.POINTER(PcCode), _vp, C.POINTER(PcSched), C.c_int32, C.c_int64, _vp, _vp, _vp,
                                _vp, _vp]
_lib.bp_decode_trace.argtypes = [C.POINTER(PcCode), _vp, C.POINTER(PcSched), C.c_int32, C.c_int64,
                                 C.POINTER(PcEvent), C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.bp_decode_posterior.argtypes = [C.POINTER(PcCode), _vp, C.POINTER(PcSched), C.c_int32, C.c_int64, _vp, _vp,
                                     _vp, _vp, _vp, _vp]
_lib.pc_f_eval.argtypes = [_vp, _vp, _vp, C.c_int64, C.c_int32, C.c_float, _vp]
_lib.bp_decode_noalloc.argtypes = [C.POINTER(PcCode), _vp, C.POINTER(PcSched), C.c_int32, C.c_int64, _vp, _vp,
                                   _vp, _vp]
_lib.pc_partition_selfcheck.argtypes = [_vp, _vp]
_lib.bp_mixed_table_size.argtypes = [C.c_int32, C.POINTER(C.c_size_t)]
_lib.bp_mixed_prepare.argtypes = [C.POINTER(PcBatch), C.c_int32, _vp, C.c_size_t]
_lib.bp_mixed_workspace_size.argtypes = [C.c_int32, C.POINTER(C.c_size_t)]
_lib.bp_decode_mixed.argtypes = [_vp, C.c_int32, _vp, _vp]
_lib.bp_slot_limit.argtypes = [C.POINTER(PcCode), C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
_lib.bp_kernel_threads.argtypes = [C.POINTER(PcCode), C.c_int32, C.POINTER(C.c_int32)]
_lib.pc_build_info.argtypes = [C.POINTER(C.c_int32)]
_lib.wbp_weights_count.argtypes = [C.POINTER(PcCode), C.c_int32, C.POINTER(C.c_size_t)]
_lib.wbp_ckpt_count.argtypes = [C.POINTER(PcCode), C.c_int32, C.c_int64, C.POINTER(C.c_size_t)]
_lib.wbp_workspace_size.argtypes = [C.POINTER(PcCode), C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]
for _nm in ("wbp_forward", "wbp_forward_f64"):
    getattr(_lib, _nm).argtypes = [C.POINTER(PcCode), _vp, _vp, C.c_int32, C.c_int64, _vp, _vp, _vp, _vp]
for _nm in ("wbp_backward", "wbp_backward_f64"):
    getattr(_lib, _nm).argtypes = [C.POINTER(PcCode), _vp, _vp, C.c_int32, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.pc_status_string.argtypes = [C.c_int]
_lib.pc_status_string.restype = C.c_char_p


class PcError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status} ({_lib.pc_status_string(status).decode()})")
        self.status = status


def _check(fn: str, status: int):
    if status != PC_OK:
        raise PcError(fn, status)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _on_current_device(t) -> bool:
    """The C calls launch on the calling thread's current device and hand it the pointers as they
    are, so a device tensor must live on that device (another GPU's memory would be dereferenced
    by the wrong device)."""
    import torch

    return t.device == torch.device("cuda", torch.cuda.current_device())


def _require(fn: str, *checks):
    """Raise PcError(PC_EINVAL) unless every (tensor, dtype, shape, where) check holds: the C calls
    receive bare pointers, so the tensors behind them must have the layout the call assumes.
    where: "cuda" (memory of the current device), "any" (host memory, which the call checks
    itself, or memory of the current device)."""
    for t, dtype, shape, where in checks:
        ok = (t is not None and t.dtype == dtype and tuple(t.shape) == tuple(shape) and t.is_contiguous()
              and (where != "cuda" or t.is_cuda) and (not t.is_cuda or _on_current_device(t)))
        if not ok:
            raise PcError(fn, PC_EINVAL)


def _require_workspace(fn: str, ws, nbytes: int, where: str = "cuda"):
    if (ws is None or not ws.is_contiguous() or ws.numel() * ws.element_size() < nbytes
            or (where == "cuda" and not ws.is_cuda) or (ws.is_cuda and not _on_current_device(ws))):
        raise PcError(fn, PC_EINVAL)


def _require_stream(fn: str, stream):
    """A stream object passed in must belong to the current device (raw handles are passed through)."""
    if stream is None or isinstance(stream, int):
        return
    import torch

    dev = getattr(stream, "device", None)
    if dev is not None and torch.device(dev) != torch.device("cuda", torch.cuda.current_device()):
        raise PcError(fn, PC_EINVAL)


def _decode_checks(code, llr, bits, iters, crc_ok, where):
    import torch

    B = llr.shape[0] if llr is not None and llr.dim() == 2 else -1
    return ((llr, torch.float32, (B, code.N), where), (bits, torch.int32, (B, words_of(code.K)), where),
            (iters, torch.int32, (B,), where), (crc_ok, torch.uint8, (B,), where))


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def library_path() -> str:
    return str(_LIB_PATH)


def sched(mode: int = 0, *, P_range: int = 2, P_level: int = 1, N_min: int = 1, D: int = 0, T0: int = 1,
          rho_range_fixed: int = 0, q_max: int = 0, it_reset_full: int = 0, stop_from: int = 1,
          stop_kind: int = 1, fkind: int = 0, alpha: float = 0.9375, seed: int = 0,
          frame_base: int = 0) -> PcSched:
    s = PcSched()
    s.mode, s.P_range, s.P_level, s.N_min, s.D, s.T0 = mode, P_range, P_level, N_min, D, T0
    s.rho_range_fixed, s.q_max, s.it_reset_full = rho_range_fixed, q_max, it_reset_full
    s.stop_from, s.stop_kind, s.fkind, s.alpha = stop_from, stop_kind, fkind, alpha
    s.seed, s.frame_base = seed, frame_base
    return s


def event(level: int, range_: int, block: int, order) -> PcEvent:
    e = PcEvent()
    e.level, e.range, e.block = level, range_, block
    for i in range(16):
        e.order[i] = order[i] if i < len(order) else i
    return e


def pc_construct(N: int, K: int, crc_len: int = 0, crc_poly: int = 0, design_ebn0_db: float = 0.0) -> PcCode:
    code = PcCode()
    _check("pc_construct", _lib.pc_construct(N, K, crc_len, crc_poly, design_ebn0_db, C.byref(code)))
    return code


def pc_encode(code: PcCode, payload, x_out, stream=None):
    """payload: uint8 CUDA tensor [B, K - crc_len]; x_out: uint8 CUDA tensor [B, N]."""
    import torch

    B = x_out.shape[0]
    _require("pc_encode", (payload, torch.uint8, (B, code.K - code.crc_len), "cuda"),
             (x_out, torch.uint8, (B, code.N), "cuda"))
    _require_stream("pc_encode", stream)
    _check("pc_encode", _lib.pc_encode(C.byref(code), _ptr(payload), _ptr(x_out), B, _stream(stream)))


def bp_decode_workspace_size(code: PcCode, B: int) -> int:
    out = C.c_size_t(0)
    _check("bp_decode_workspace_size", _lib.bp_decode_workspace_size(C.byref(code), B, C.byref(out)))
    return out.value


def bp_decode(code: PcCode, llr, sch: PcSched, max_iters: int, bits, iters, crc_ok, workspace, stream=None):
    """llr: float32 [B, N]; bits: int32 [B, ceil(K/32)]; iters: int32 [B]; crc_ok: uint8 [B] (CUDA tensors)."""
    B = llr.shape[0]
    _require("bp_decode", *_decode_checks(code, llr, bits, iters, crc_ok, "cuda"))
    _require_workspace("bp_decode", workspace, bp_decode_workspace_size(code, B))
    _require_stream("bp_decode", stream)
    _check("bp_decode", _lib.bp_decode(C.byref(code), _ptr(llr), C.byref(sch), max_iters, B, _ptr(bits),
                                       _ptr(iters), _ptr(crc_ok), _ptr(workspace), _stream(stream)))


def bp_decode_host(code: PcCode, llr, sch: PcSched, max_iters: int, bits, iters, crc_ok, workspace, stream=None):
    """bp_decode on tensors in page-locked host memory (or on the device): the kernel reads and
    writes them in place.  Asynchronous on the stream."""
    B = llr.shape[0]
    _require("bp_decode_host", *_decode_checks(code, llr, bits, iters, crc_ok, "any"))
    _require_workspace("bp_decode_host", workspace, bp_decode_workspace_size(code, B))
    _require_stream("bp_decode_host", stream)
    _check("bp_decode_host", _lib.bp_decode_host(C.byref(code), _ptr(llr), C.byref(sch), max_iters, B, _ptr(bits),
                                                 _ptr(iters), _ptr(crc_ok), _ptr(workspace), _stream(stream)))


def bp_decode_trace(code: PcCode, llr, sch: PcSched, max_iters: int, events, dump, bits, iters, crc_ok, workspace,
                    stream=None):
    """As bp_decode, recording every plane into dump [B, max_iters, 2, n+1, N]; events: list of PcEvent or None."""
    import torch

    B = llr.shape[0]
    # the dump's layout is [B][max_iters][2][n+1][N]; with no iterations nothing is written
    dump_shape = (B, max_iters, 2, code.n + 1, code.N) if max_iters > 0 else (tuple(dump.shape) if dump is not None else ())
    _require("bp_decode_trace", *_decode_checks(code, llr, bits, iters, crc_ok, "cuda"),
             (dump, torch.float32, dump_shape, "cuda"))
    _require_workspace("bp_decode_trace", workspace, bp_decode_workspace_size(code, B))
    if events is None:
        evp, nev = None, 0
    else:
        arr = (PcEvent * max(len(events), 1))(*events)
        evp, nev = arr, len(events)
    _require_stream("bp_decode_trace", stream)
    _check("bp_decode_trace", _lib.bp_decode_trace(C.byref(code), _ptr(llr), C.byref(sch), max_iters, B, evp, nev,
                                                   _ptr(dump), _ptr(bits), _ptr(iters), _ptr(crc_ok),
                                                   _ptr(workspace), _stream(stream)))


def bp_decode_posterior(code: PcCode, llr, sch: PcSched, max_iters: int, bits, iters, crc_ok, post, workspace,
                        stream=None):
    """bp_decode that also writes post [B, 2, N] float32: L at node level n+1 and R at node level 1
    after each frame's last iteration (N >= 128, no G-matrix stop)."""
    import torch

    B = llr.shape[0]
    _require("bp_decode_posterior", *_decode_checks(code, llr, bits, iters, crc_ok, "cuda"),
             (post, torch.float32, (B, 2, code.N), "cuda"))
    _require_workspace("bp_decode_posterior", workspace, bp_decode_workspace_size(code, B))
    _require_stream("bp_decode_posterior", stream)
    _check("bp_decode_posterior", _lib.bp_decode_posterior(C.byref(code), _ptr(llr), C.byref(sch), max_iters, B,
                                                           _ptr(bits), _ptr(iters), _ptr(crc_ok), _ptr(post),
                                                           _ptr(workspace), _stream(stream)))


def pc_f_eval(a, b, out, fkind: int, alpha: float = 1.0, stream=None):
    """out = f(a, b) elementwise as the decoder kernels evaluate it (float32 CUDA tensors of one shape)."""
    import torch

    shape = tuple(a.shape)
    _require("pc_f_eval", (a, torch.float32, shape, "cuda"), (b, torch.float32, shape, "cuda"),
             (out, torch.float32, shape, "cuda"))
    _require_stream("pc_f_eval", stream)
    _check("pc_f_eval", _lib.pc_f_eval(_ptr(a), _ptr(b), _ptr(out), a.numel(), fkind, alpha, _stream(stream)))


def bp_decode_noalloc(code: PcCode, llr, sch: PcSched, max_iters: int, bits, iters, crc_ok, stream=None):
    """bp_decode without a workspace argument: for callers that cannot allocate device memory
    while decoding.  Its scratch is a fixed device array inside the library, shared by every call:
    calls must not overlap on the GPU, and the first call on a device must precede any stream
    capture."""
    B = llr.shape[0]
    _require("bp_decode_noalloc", *_decode_checks(code, llr, bits, iters, crc_ok, "cuda"))
    _require_stream("bp_decode_noalloc", stream)
    _check("bp_decode_noalloc", _lib.bp_decode_noalloc(C.byref(code), _ptr(llr), C.byref(sch), max_iters, B,
                                                       _ptr(bits), _ptr(iters), _ptr(crc_ok), _stream(stream)))


def words_of(K: int) -> int:
    return int(math.ceil(K / 32))


class Decoder:
    """Owns the output and workspace tensors of repeated bp_decode calls on one device."""

    def __init__(self, code: PcCode, sch: PcSched, max_iters: int, device="cuda"):
        import torch

        self.code, self.sched, self.max_iters = code, sch, max_iters
        self.device = torch.device(device)
        self._B = -1
        self.workspace = torch.empty(bp_decode_workspace_size(code, 1), dtype=torch.uint8, device=self.device)

    def _ensure(self, B: int):
        import torch

        if B != self._B:
            self.bits = torch.empty((B, words_of(self.code.K)), dtype=torch.int32, device=self.device)
            self.iters = torch.empty(B, dtype=torch.int32, device=self.device)
            self.crc_ok = torch.empty(B, dtype=torch.uint8, device=self.device)
            self._B = B

    def __call__(self, llr, stream=None):
        import torch

        self._ensure(llr.shape[0])
        with torch.cuda.device(self.device):
            bp_decode(self.code, llr, self.sched, self.max_iters, self.bits, self.iters, self.crc_ok,
                      self.workspace, stream)
        return self.bits, self.iters, self.crc_ok


def unpack_bits(words, K: int):
    """[B, ceil(K/32)] int32 words -> [B, K] uint8 bits (bit k in word k/32 at position k%32)."""
    import torch

    w = words.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(32, device=w.device, dtype=torch.int64)
    bits = (w.unsqueeze(-1) >> shifts) & 1
    return bits.reshape(w.shape[0], -1)[:, :K].to(torch.uint8)


class HostDecoder:
    """Decodes LLRs that live in page-locked host memory with one bp_decode_host
    call: the kernel reads each frame's LLRs across the host-device link and
    writes bits, iterations and CRC flags into page-locked host tensors, with
    no staging copies.  Output tensors are allocated once per batch size."""

    def __init__(self, code: PcCode, sch: PcSched, max_iters: int, device="cuda"):
        import torch

        self.code, self.sched, self.max_iters = code, sch, max_iters
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)
        self.workspace = torch.empty(bp_decode_workspace_size(code, 1), dtype=torch.uint8, device=self.device)
        self._shape = None

    def _ensure(self, B: int):
        import torch

        if self._shape != B:
            KW = words_of(self.code.K)
            self.h_bits = torch.empty((B, KW), dtype=torch.int32, pin_memory=True)
            self.h_iters = torch.empty(B, dtype=torch.int32, pin_memory=True)
            self.h_ok = torch.empty(B, dtype=torch.uint8, pin_memory=True)
            self._shape = B

    def __call__(self, h_llr):
        """h_llr: page-locked float32 [B, N] host tensor -> (bits, iters, crc_ok) host tensors (synchronised)."""
        if h_llr.is_cuda or not h_llr.is_pinned():
            raise ValueError("h_llr must be a page-locked host tensor (tensor.pin_memory())")
        if not h_llr.is_contiguous():
            raise ValueError("h_llr must be contiguous")
        import torch

        self._ensure(h_llr.shape[0])
        # work the caller queued on its current stream (e.g. an asynchronous fill of h_llr) comes first
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.device(self.device):
            bp_decode_host(self.code, h_llr, self.sched, self.max_iters, self.h_bits, self.h_iters, self.h_ok,
                           self.workspace, self.stream)
        self.stream.synchronize()
        return self.h_bits, self.h_iters, self.h_ok


def pc_partition_selfcheck(device="cuda"):
    """(partitions checked, event shapes whose two partition builds differ, partitions whose
    group shape the sweeps do not assume) of the N >= 128 decoder."""
    import torch

    out = torch.zeros(3, dtype=torch.int32, device=device)
    _check("pc_partition_selfcheck", _lib.pc_partition_selfcheck(_ptr(out), _stream(None)))
    torch.cuda.synchronize()
    return int(out[0].item()), int(out[1].item()), int(out[2].item())


def build_checked() -> bool:
    """True for a library built with PCBP_CHECKED (bounds-checked decoder)."""
    out = C.c_int32(0)
    _check("pc_build_info", _lib.pc_build_info(C.byref(out)))
    return bool(out.value & 1)


def bp_kernel_threads(code: PcCode, kernel: int):
    """Threads per frame that select a decoder kernel (0: TMEM stage groups, 1: shared-memory
    stage groups) for this code, or None where that kernel has no build for N."""
    out = C.c_int32(0)
    rc = _lib.bp_kernel_threads(C.byref(code), kernel, C.byref(out))
    if rc == PC_EUNSUPPORTED:
        return None
    _check("bp_kernel_threads", rc)
    return out.value


def bp_slot_limit(code: PcCode, threads_per_frame: int = 0, fkind: int = 0) -> int:
    """Largest frames-per-CTA count of the decoder kernel for this code and threads per frame."""
    out = C.c_int32(0)
    _check("bp_slot_limit", _lib.bp_slot_limit(C.byref(code), threads_per_frame, fkind, C.byref(out)))
    return out.value


def bp_mixed_table_size(n_batches: int) -> int:
    out = C.c_size_t(0)
    _check("bp_mixed_table_size", _lib.bp_mixed_table_size(n_batches, C.byref(out)))
    return out.value


def bp_mixed_workspace_size(n_batches: int) -> int:
    out = C.c_size_t(0)
    _check("bp_mixed_workspace_size", _lib.bp_mixed_workspace_size(n_batches, C.byref(out)))
    return out.value


def bp_mixed_prepare(batches, h_table):
    arr = (PcBatch * len(batches))(*batches)
    _check("bp_mixed_prepare", _lib.bp_mixed_prepare(arr, len(batches), C.cast(h_table, C.c_void_p),
                                                     C.sizeof(h_table)))


def bp_decode_mixed(h_table, n_batches, workspace, stream=None):
    _require_stream("bp_decode_mixed", stream)
    _check("bp_decode_mixed", _lib.bp_decode_mixed(C.cast(h_table, C.c_void_p), n_batches, _ptr(workspace),
                                                   _stream(stream)))


class MixedDecoder:
    """Batches of different codes decoded in one persistent sweep (bp_decode_mixed).

    parts: list of (code, sched, max_iters, llr [B, N] CUDA float32 tensor, slots) or
    (..., slots, threads_per_frame) (0: the bp_decode kernel for that length).  Output
    tensors per batch are allocated here (`bits[i]`, `iters[i]`, `crc_ok[i]`); the launch
    table is prepared once, so `__call__` only enqueues a memset and one launch per batch (it
    can be captured in a CUDA graph after a first uncaptured call)."""

    def __init__(self, parts, device="cuda"):
        import torch

        self.device = torch.device(device)
        self.codes = [p[0] for p in parts]          # keep the host structs alive
        self.llr = [p[3] for p in parts]
        self.bits, self.iters, self.crc_ok, self.batches = [], [], [], []
        for part in parts:
            code, sch, max_iters, llr, slots = part[:5]
            tpf = part[5] if len(part) > 5 else 0
            B = llr.shape[0]
            _require("bp_mixed_prepare", (llr, torch.float32, (B, code.N), "cuda"))
            bits = torch.empty((B, words_of(code.K)), dtype=torch.int32, device=self.device)
            iters = torch.empty(B, dtype=torch.int32, device=self.device)
            ok = torch.empty(B, dtype=torch.uint8, device=self.device)
            self.bits.append(bits)
            self.iters.append(iters)
            self.crc_ok.append(ok)
            b = PcBatch()
            b.code = C.pointer(code)
            b.sched = sch
            b.max_iters, b.slots, b.threads_per_frame, b.B = max_iters, slots, tpf, B
            b.d_llr, b.d_bits, b.d_iters, b.d_crc_ok = (llr.data_ptr(), bits.data_ptr(), iters.data_ptr(),
                                                        ok.data_ptr())
            self.batches.append(b)
        nb = len(self.batches)
        with torch.cuda.device(self.device):
            self.table = (C.c_char * max(bp_mixed_table_size(nb), 1))()
            bp_mixed_prepare(self.batches, self.table)
        self.workspace = torch.zeros(bp_mixed_workspace_size(nb), dtype=torch.uint8, device=self.device)

    def __call__(self, stream=None):
        bp_decode_mixed(self.table, len(self.batches), self.workspace, stream)
        return self.bits, self.iters, self.crc_ok


def wbp_weights_count(code: PcCode, T: int) -> int:
    out = C.c_size_t(0)
    _check("wbp_weights_count", _lib.wbp_weights_count(C.byref(code), T, C.byref(out)))
    return out.value


def wbp_ckpt_count(code: PcCode, T: int, B: int) -> int:
    out = C.c_size_t(0)
    _check("wbp_ckpt_count", _lib.wbp_ckpt_count(C.byref(code), T, B, C.byref(out)))
    return out.value


def wbp_workspace_size(code: PcCode, T: int, B: int, real_bytes: int) -> int:
    out = C.c_size_t(0)
    _check("wbp_workspace_size", _lib.wbp_workspace_size(C.byref(code), T, B, real_bytes, C.byref(out)))
    return out.value


def _wbp_checks(fn, code, llr, w, T):
    """llr [B, N] float32 or float64 CUDA tensor; w the same dtype with wbp_weights_count elements."""
    import torch

    if llr is None or llr.dtype not in (torch.float32, torch.float64) or llr.dim() != 2:
        raise PcError(fn, PC_EINVAL)
    B = llr.shape[0]
    _require(fn, (llr, llr.dtype, (B, code.N), "cuda"), (w, llr.dtype, tuple(w.shape) if w is not None else (), "cuda"))
    if w.numel() != wbp_weights_count(code, T):
        raise PcError(fn, PC_EINVAL)
    return B


def wbp_forward(code: PcCode, llr, w, T: int, logits, ckpt, workspace, stream=None):
    fn = "wbp_forward_f64" if llr.element_size() == 8 else "wbp_forward"
    B = _wbp_checks(fn, code, llr, w, T)
    _require(fn, (logits, llr.dtype, (B, code.K), "cuda"))
    if ckpt is not None:
        _require(fn, (ckpt, llr.dtype, tuple(ckpt.shape), "cuda"))
        if ckpt.numel() < wbp_ckpt_count(code, T, B):
            raise PcError(fn, PC_EINVAL)
    _require_workspace(fn, workspace, wbp_workspace_size(code, T, B, llr.element_size()))
    _require_stream(fn, stream)
    _check(fn, getattr(_lib, fn)(C.byref(code), _ptr(llr), _ptr(w), T, llr.shape[0], _ptr(logits), _ptr(ckpt),
                                 _ptr(workspace), _stream(stream)))


def wbp_backward(code: PcCode, llr, w, T: int, ckpt, glogits, gw, gllr, workspace, stream=None):
    fn = "wbp_backward_f64" if llr.element_size() == 8 else "wbp_backward"
    B = _wbp_checks(fn, code, llr, w, T)
    _require(fn, (glogits, llr.dtype, (B, code.K), "cuda"), (gw, llr.dtype, tuple(w.shape), "cuda"),
             (ckpt, llr.dtype, tuple(ckpt.shape) if ckpt is not None else (), "cuda"))
    if ckpt.numel() < wbp_ckpt_count(code, T, B):
        raise PcError(fn, PC_EINVAL)
    if gllr is not None:
        _require(fn, (gllr, llr.dtype, (B, code.N), "cuda"))
    _require_workspace(fn, workspace, wbp_workspace_size(code, T, B, llr.element_size()))
    _require_stream(fn, stream)
    _check(fn, getattr(_lib, fn)(C.byref(code), _ptr(llr), _ptr(w), T, llr.shape[0], _ptr(ckpt), _ptr(glogits),
                                 _ptr(gw), _ptr(gllr), _ptr(workspace), _stream(stream)))


def _wbp_function():
    import torch

    class WBPFunction(torch.autograd.Function):
        """logits = weighted BP(llr, w): forward and hand-written backward kernels."""

        @staticmethod
        def forward(ctx, llr, w, code, T):
            llr = llr.contiguous()
            w = w.contiguous()
            B = llr.shape[0]
            logits = torch.empty((B, code.K), dtype=llr.dtype, device=llr.device)
            ckpt = torch.empty(wbp_ckpt_count(code, T, B), dtype=llr.dtype, device=llr.device)
            ws = torch.empty(wbp_workspace_size(code, T, B, llr.element_size()), dtype=torch.uint8,
                             device=llr.device)
            wbp_forward(code, llr, w, T, logits, ckpt, ws)
            ctx.save_for_backward(llr, w, ckpt)
            ctx.code, ctx.T, ctx.ws = code, T, ws
            return logits

        @staticmethod
        def backward(ctx, glogits):
            llr, w, ckpt = ctx.saved_tensors
            gw = torch.zeros_like(w)
            gllr = torch.empty_like(llr) if ctx.needs_input_grad[0] else None
            wbp_backward(ctx.code, llr, w, ctx.T, ckpt, glogits.contiguous(), gw, gllr, ctx.ws)
            return gllr, gw, None, None

    return WBPFunction


def wbp(llr, w, code: PcCode, T: int):
    """Differentiable weighted BP: logits [B, K] from llr [B, N] and w [T, n, N/2, 4] (CUDA tensors)."""
    global _WBP
    try:
        fn = _WBP
    except NameError:
        fn = _WBP = _wbp_function()
    return fn.apply(llr, w, code, T)
