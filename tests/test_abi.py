"""C ABI checks that need no GPU: the library loads, exports every function
include/pcbp.h declares, and its host-side logic (construction, argument
validation) behaves as documented."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


def _has_cuda():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


# The validation tests pass placeholder addresses that are only ever checked
# on the host.  They run only where no GPU exists, so that a validation bug
# can never turn into a launch on those addresses.
no_gpu_only = pytest.mark.skipif(_has_cuda(), reason="placeholder pointers: host-only check")


def declared_functions():
    names = []
    for hdr in sorted((ROOT / "include").glob("*.h")):
        text = hdr.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(pcbp):
    names = declared_functions()
    assert "bp_decode" in names and "pc_construct" in names
    lib = C.CDLL(pcbp.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pcbp.EXPORTED) <= set(names)


def test_build_info_reports_the_checked_build(pcbp):
    """pc_build_info bit 0 is set exactly for a library built with PCBP_CHECKED=1 (the build the
    tests load follows the same environment variable)."""
    import os

    assert pcbp.build_checked() == (os.environ.get("PCBP_CHECKED") == "1")
    lib = C.CDLL(pcbp.library_path())
    lib.pc_build_info.argtypes = [C.c_void_p]
    assert lib.pc_build_info(None) == pcbp.PC_EINVAL


@pytest.mark.parametrize("N,K,db", [(8, 4, 0.0), (64, 32, 0.0), (256, 128, 0.0), (1024, 512, 0.0),
                                    (2048, 1024, 0.0), (512, 384, 1.5), (128, 32, -2.0), (2048, 1536, 0.0)])
def test_pc_construct_matches_oracle(pcbp, oracle, N, K, db):
    code = pcbp.pc_construct(N, K, 0, 0, db)
    _, fr = oracle.construct(N, K, db)
    assert code.N == N and code.n == N.bit_length() - 1 and code.K == K
    assert np.array_equal(np.array(code.frozen(), dtype=np.uint8), fr)
    assert code.info_positions() == list(np.nonzero(fr == 0)[0])


def test_pc_construct_crc_poly_normalised(pcbp):
    c8 = pcbp.pc_construct(256, 128, 8, 0x9B)
    assert c8.crc_poly == 0x19B and c8.crc_len == 8
    c24 = pcbp.pc_construct(1024, 512, 24, 0x1B2B117)
    assert c24.crc_poly == 0x1B2B117


@pytest.mark.parametrize("args", [(12, 6, 0, 0), (4, 2, 0, 0), (4096, 2048, 0, 0), (64, 0, 0, 0), (64, 65, 0, 0),
                                  (64, 8, 8, 0x9B), (64, 32, 33, 1), (64, 32, 8, 0x3FF)])
def test_pc_construct_rejects_bad_arguments(pcbp, args):
    with pytest.raises(pcbp.PcError) as e:
        pcbp.pc_construct(*args)
    assert e.value.status == pcbp.PC_EINVAL


def _call_decode(pcbp, code, sch, max_iters=10, B=4, llr=1, bits=1, iters=1, ok=1, ws=256):
    p = lambda v: C.c_void_p(v) if v else None
    return pcbp._lib.bp_decode(C.byref(code), p(llr * 4096), C.byref(sch), max_iters, B, p(bits * 4096),
                               p(iters * 4096), p(ok * 4096), p(ws * 4096), None)


@no_gpu_only
def test_bp_decode_validates_before_touching_the_device(pcbp):
    """Every argument error returns PC_EINVAL on the host; nothing is launched
    (these calls run on a machine without a GPU)."""
    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    ok = pcbp.sched(mode=1, P_range=3, P_level=5, N_min=5, T0=5)
    bad_scheds = [
        pcbp.sched(mode=3),
        pcbp.sched(mode=1, P_range=9, P_level=5, N_min=5, T0=5),          # P_range > n
        pcbp.sched(mode=1, P_range=3, P_level=8, N_min=5, T0=5),          # P_level > n - 1
        pcbp.sched(mode=1, P_range=3, P_level=5, N_min=0, T0=5),          # N_min < 1
        pcbp.sched(mode=1, P_range=3, P_level=5, N_min=5, T0=0),          # T0 < 1
        pcbp.sched(mode=1, rho_range_fixed=1, P_level=5, N_min=5, T0=5),  # rho_range < 2
        pcbp.sched(mode=2, it_reset_full=0),
        pcbp.sched(stop_kind=4),
        pcbp.sched(alpha=0.0),
        pcbp.sched(alpha=float("nan")),
    ]
    for s in bad_scheds:
        assert _call_decode(pcbp, code, s) == pcbp.PC_EINVAL
    assert _call_decode(pcbp, code, pcbp.sched(fkind=2)) == pcbp.PC_EUNSUPPORTED
    assert _call_decode(pcbp, code, ok, max_iters=-1) == pcbp.PC_EINVAL
    assert _call_decode(pcbp, code, ok, B=-1) == pcbp.PC_EINVAL
    assert _call_decode(pcbp, code, ok, llr=0) == pcbp.PC_EINVAL
    assert _call_decode(pcbp, code, ok, bits=0) == pcbp.PC_EINVAL
    assert _call_decode(pcbp, code, ok, ws=0) == pcbp.PC_EINVAL
    # misaligned LLR pointer (must be 16-byte aligned)
    assert pcbp._lib.bp_decode(C.byref(code), C.c_void_p(4096 + 4), C.byref(ok), 10, 4, C.c_void_p(4096),
                               C.c_void_p(4096), C.c_void_p(4096), C.c_void_p(8192), None) == pcbp.PC_EINVAL
    # B == 0 is a no-op that succeeds without any device call
    assert _call_decode(pcbp, code, ok, B=0) == pcbp.PC_OK
    # a corrupted code (frozen mask inconsistent with K) is rejected
    bad = pcbp.pc_construct(256, 128, 8, 0x9B)
    bad.frozen_mask[0] ^= 1
    assert _call_decode(pcbp, bad, ok) == pcbp.PC_EINVAL


def test_bp_decode_host_validates_before_touching_the_device(pcbp):
    """Argument errors of the host-buffer entry return PC_EINVAL before any
    pointer is examined; B == 0 succeeds at once."""
    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    s = pcbp.sched(mode=1, P_range=3, P_level=5, N_min=5, T0=5)
    p = lambda v: C.c_void_p(v) if v else None

    def call(B=4, max_iters=10, llr=1, bits=1, iters=1, ok=1, ws=1, sch=s):
        return pcbp._lib.bp_decode_host(C.byref(code), p(llr * 4096), C.byref(sch), max_iters, B, p(bits * 4096),
                                        p(iters * 4096), p(ok * 4096), p(ws * 4096), None)

    assert call(B=0) == pcbp.PC_OK
    assert call(B=-1) == pcbp.PC_EINVAL
    assert call(max_iters=-1) == pcbp.PC_EINVAL
    for arg in ("llr", "bits", "iters", "ok", "ws"):
        assert call(**{arg: 0}) == pcbp.PC_EINVAL
    bad = pcbp.pc_construct(256, 128, 8, 0x9B)
    bad.frozen_mask[0] ^= 1
    assert pcbp._lib.bp_decode_host(C.byref(bad), p(4096), C.byref(s), 10, 4, p(4096), p(4096), p(4096), p(4096),
                                    None) == pcbp.PC_EINVAL


@no_gpu_only
def test_bp_decode_host_rejects_unmapped_pointers_without_a_device(pcbp):
    """Placeholder addresses are neither mapped host memory nor device memory:
    rejected on the host (no device here, so the runtime query itself fails)."""
    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    s = pcbp.sched(mode=1, P_range=3, P_level=5, N_min=5, T0=5)
    rc = pcbp._lib.bp_decode_host(C.byref(code), C.c_void_p(4096), C.byref(s), 10, 4, C.c_void_p(4096),
                                  C.c_void_p(4096), C.c_void_p(4096), C.c_void_p(8192), None)
    assert rc in (pcbp.PC_EINVAL, pcbp.PC_ECUDA)


@no_gpu_only
def test_trace_validates_events(pcbp):
    code = pcbp.pc_construct(64, 32)
    s = pcbp.sched(mode=1, P_range=3, P_level=4, N_min=2, T0=2)
    good = pcbp.event(2, 3, 1, [2, 0, 1])
    bad = [pcbp.event(5, 3, 0, [0, 1, 2]),      # level + range - 1 > n
           pcbp.event(2, 3, 4, [0, 1, 2]),      # block >= N / 2^m = 4
           pcbp.event(1, 3, 0, [0, 0, 1]),      # not a permutation
           pcbp.event(1, 1, 0, [0])]            # range < 2
    p = C.c_void_p(4096)
    for ev in bad:
        arr = (pcbp.PcEvent * 2)(good, ev)
        assert pcbp._lib.bp_decode_trace(C.byref(code), p, C.byref(s), 5, 2, arr, 2, p, p, p, p, C.c_void_p(8192),
                                         None) == pcbp.PC_EINVAL
    arr = (pcbp.PcEvent * 1)(good)
    assert pcbp._lib.bp_decode_trace(C.byref(code), p, C.byref(s), 5, 2, arr, 1, None, p, p, p, C.c_void_p(8192),
                                     None) == pcbp.PC_EINVAL   # no dump buffer


def test_workspace_size_and_status_strings(pcbp):
    code = pcbp.pc_construct(1024, 512, 24, 0x1B2B117)
    assert pcbp.bp_decode_workspace_size(code, 10**6) >= 8
    assert pcbp._lib.pc_status_string(pcbp.PC_EINVAL) == b"invalid argument"
    assert pcbp._lib.pc_status_string(12345) == b"unknown status"


@no_gpu_only
def test_pc_encode_validates(pcbp):
    code = pcbp.pc_construct(64, 32, 8, 0x9B)
    assert pcbp._lib.pc_encode(C.byref(code), C.c_void_p(4096), None, 4, None) == pcbp.PC_EINVAL
    assert pcbp._lib.pc_encode(C.byref(code), C.c_void_p(4096), C.c_void_p(4096), -1, None) == pcbp.PC_EINVAL
    assert pcbp._lib.pc_encode(C.byref(code), C.c_void_p(4096), C.c_void_p(4096), 0, None) == pcbp.PC_OK


@no_gpu_only
def test_mixed_entry_points_validate_on_the_host(pcbp):
    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    b = pcbp.PcBatch()
    b.code = C.pointer(code)
    b.sched = pcbp.sched(mode=1, P_range=3, P_level=5, N_min=5, T0=5)
    b.max_iters, b.slots, b.B = 10, 0, 4
    b.d_llr = b.d_bits = b.d_iters = b.d_crc_ok = 4096
    assert pcbp.bp_mixed_table_size(3) > 0 and pcbp.bp_mixed_workspace_size(3) >= 24
    h = (C.c_char * pcbp.bp_mixed_table_size(1))()
    bad = pcbp.PcBatch.from_buffer_copy(b)
    bad.sched = pcbp.sched(mode=1, P_range=30, P_level=5, N_min=5, T0=5)
    arr = (pcbp.PcBatch * 1)(bad)
    assert pcbp._lib.bp_mixed_prepare(arr, 1, C.cast(h, C.c_void_p), C.sizeof(h)) == pcbp.PC_EINVAL
    nob = pcbp.PcBatch.from_buffer_copy(b)
    nob.d_llr = None
    arr = (pcbp.PcBatch * 1)(nob)
    assert pcbp._lib.bp_mixed_prepare(arr, 1, C.cast(h, C.c_void_p), C.sizeof(h)) == pcbp.PC_EINVAL
    # a valid batch (box-plus included) gets past validation to the device query
    bx = pcbp.PcBatch.from_buffer_copy(b)
    bx.sched = pcbp.sched(fkind=1)
    arr = (pcbp.PcBatch * 1)(bx)
    assert pcbp._lib.bp_mixed_prepare(arr, 1, C.cast(h, C.c_void_p), C.sizeof(h)) == pcbp.PC_ECUDA
    # threads per frame: the counts bp_kernel_threads reports (at N = 256 both kernels take N/4 = 64)
    # only; reserved must be 0
    for tpf, want in ((48, pcbp.PC_EUNSUPPORTED), (16, pcbp.PC_EUNSUPPORTED), (32, pcbp.PC_EUNSUPPORTED),
                      (64, pcbp.PC_ECUDA)):
        bt = pcbp.PcBatch.from_buffer_copy(b)
        bt.threads_per_frame = tpf
        arr = (pcbp.PcBatch * 1)(bt)
        assert pcbp._lib.bp_mixed_prepare(arr, 1, C.cast(h, C.c_void_p), C.sizeof(h)) == want, tpf
    br = pcbp.PcBatch.from_buffer_copy(b)
    br.reserved = 1
    arr = (pcbp.PcBatch * 1)(br)
    assert pcbp._lib.bp_mixed_prepare(arr, 1, C.cast(h, C.c_void_p), C.sizeof(h)) == pcbp.PC_EINVAL
    arr = (pcbp.PcBatch * 1)(b)
    assert pcbp._lib.bp_mixed_prepare(arr, 1, C.cast(h, C.c_void_p), 8) == pcbp.PC_ENOMEM
    assert pcbp._lib.bp_mixed_prepare(arr, 65, C.cast(h, C.c_void_p), C.sizeof(h)) == pcbp.PC_EINVAL
    # decode: nothing to do, missing workspace, a table bp_mixed_prepare did not write
    assert pcbp._lib.bp_decode_mixed(C.cast(h, C.c_void_p), 0, None, None) == pcbp.PC_OK
    assert pcbp._lib.bp_decode_mixed(C.cast(h, C.c_void_p), 1, None, None) == pcbp.PC_EINVAL
    assert pcbp._lib.bp_decode_mixed(None, 1, C.c_void_p(4096), None) == pcbp.PC_EINVAL
    zeros = (C.c_char * pcbp.bp_mixed_table_size(1))()
    assert pcbp._lib.bp_decode_mixed(C.cast(zeros, C.c_void_p), 1, C.c_void_p(4096), None) == pcbp.PC_EINVAL

@no_gpu_only
def test_wbp_entry_points_validate_on_the_host(pcbp):
    """Argument errors of the weighted-BP calls return PC_EINVAL before anything
    touches a device: T out of range, NULL buffers, a misaligned workspace, and
    weights not aligned to a pair (the kernels load a processing element's two
    weights of a sweep at once)."""
    code = pcbp.pc_construct(64, 32)
    p = C.c_void_p
    fwd, fwd64 = pcbp._lib.wbp_forward, pcbp._lib.wbp_forward_f64
    bwd = pcbp._lib.wbp_backward
    assert fwd(C.byref(code), p(4096), p(8192), 0, 4, p(4096), None, p(8192), None) == pcbp.PC_EINVAL
    assert fwd(C.byref(code), None, p(8192), 2, 4, p(4096), None, p(8192), None) == pcbp.PC_EINVAL
    assert fwd(C.byref(code), p(4096), p(8192), 2, 4, p(4096), None, p(8192 + 16), None) == pcbp.PC_EINVAL
    assert fwd(C.byref(code), p(4096), p(8192 + 4), 2, 4, p(4096), None, p(8192), None) == pcbp.PC_EINVAL
    assert fwd64(C.byref(code), p(4096), p(8192 + 8), 2, 4, p(4096), None, p(8192), None) == pcbp.PC_EINVAL
    assert bwd(C.byref(code), p(4096), p(8192 + 4), 2, 4, p(4096), p(4096), p(4096), None, p(8192),
               None) == pcbp.PC_EINVAL
    assert fwd(C.byref(code), p(4096), p(8192), 2, 0, p(4096), None, p(8192), None) == pcbp.PC_OK


def test_slot_limit_validates_on_the_host(pcbp):
    code = pcbp.pc_construct(1024, 512, 24, 0x1B2B117)
    out = C.c_int32(0)
    assert pcbp._lib.bp_slot_limit(C.byref(code), 128, 0, None) == pcbp.PC_EINVAL
    assert pcbp._lib.bp_slot_limit(None, 128, 0, C.byref(out)) == pcbp.PC_EINVAL
    assert pcbp._lib.bp_slot_limit(C.byref(code), -1, 0, C.byref(out)) == pcbp.PC_EINVAL
    assert pcbp._lib.bp_slot_limit(C.byref(code), 128, 2, C.byref(out)) == pcbp.PC_EINVAL
    assert pcbp._lib.bp_slot_limit(C.byref(code), 100, 0, C.byref(out)) == pcbp.PC_EUNSUPPORTED


def test_kernel_threads_is_a_host_query(pcbp):
    """Threads per frame of each decoder kernel, without a device: the TMEM kernel takes N/4 up
    to N = 256 and N/8 from 512 and has no build below N = 128; the shared-memory kernel takes
    max(32, N/4)."""
    want = {64: (None, 32), 128: (32, 32), 256: (64, 64), 512: (64, 128), 1024: (128, 256), 2048: (256, 512)}
    for N, (t0, t1) in want.items():
        code = pcbp.pc_construct(N, N // 2)
        assert pcbp.bp_kernel_threads(code, 0) == t0, N
        assert pcbp.bp_kernel_threads(code, 1) == t1, N
    out = C.c_int32(0)
    code = pcbp.pc_construct(256, 128)
    assert pcbp._lib.bp_kernel_threads(C.byref(code), 2, C.byref(out)) == pcbp.PC_EINVAL
    assert pcbp._lib.bp_kernel_threads(C.byref(code), 0, None) == pcbp.PC_EINVAL


def test_binding_rejects_tensors_the_calls_cannot_use(pcbp):
    """The C calls take bare pointers, so the binding checks dtype, shape, contiguity and device
    first and raises PcError(PC_EINVAL) with nothing enqueued (no GPU needed to see the refusal)."""
    import torch

    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    B, KW = 4, pcbp.words_of(128)
    llr = torch.zeros((B, 256), dtype=torch.float32)
    bits = torch.zeros((B, KW), dtype=torch.int32)
    iters = torch.zeros(B, dtype=torch.int32)
    ok = torch.zeros(B, dtype=torch.uint8)
    ws = torch.zeros(256, dtype=torch.uint8)
    s = pcbp.sched()
    bad = [
        (llr, bits, iters, ok, ws),                                   # host tensors for a device call
        (llr.double(), bits, iters, ok, ws),                          # wrong dtype
        (llr[:, :128], bits, iters, ok, ws),                          # wrong N
        (torch.zeros((B, 512), dtype=torch.float32)[:, ::2], bits, iters, ok, ws),   # not contiguous
        (llr, bits[:, :2], iters, ok, ws),                            # too few words per frame
        (llr, bits, iters[:2], ok, ws),                               # wrong batch
        (llr, bits, iters, ok.to(torch.int32), ws),                   # wrong flag dtype
    ]
    for args in bad:
        with pytest.raises(pcbp.PcError) as e:
            pcbp.bp_decode(code, args[0], s, 10, *args[1:])
        assert e.value.status == pcbp.PC_EINVAL
    with pytest.raises(pcbp.PcError) as e:                            # host call: layout still checked
        pcbp.bp_decode_host(code, llr, s, 10, bits, iters[:3], ok, ws)
    assert e.value.status == pcbp.PC_EINVAL
    with pytest.raises(pcbp.PcError) as e:
        pcbp.pc_encode(code, torch.zeros((B, 120), dtype=torch.uint8), torch.zeros((B, 256), dtype=torch.uint8))
    assert e.value.status == pcbp.PC_EINVAL
    with pytest.raises(pcbp.PcError) as e:
        pcbp.wbp_forward(code, llr, torch.zeros(10, dtype=torch.float64), 1, torch.zeros((B, 128)), None, ws)
    assert e.value.status == pcbp.PC_EINVAL


class _FakeDeviceTensor:
    """Stands in for a contiguous CUDA tensor on a given device, so that the binding's device check
    can be exercised without a GPU."""

    def __init__(self, shape, dtype, index):
        import torch

        self.shape, self.dtype = tuple(shape), dtype
        self.device = torch.device("cuda", index)
        self.is_cuda = True

    def is_contiguous(self):
        return True

    def dim(self):
        return len(self.shape)

    def numel(self):
        out = 1
        for d in self.shape:
            out *= d
        return out

    def element_size(self):
        return self.dtype.itemsize

    def data_ptr(self):
        raise AssertionError("the binding took a pointer of a tensor it should have refused")


class _NoCalls:
    def __getattr__(self, name):
        if name == "pc_status_string":
            import ctypes

            return lambda status: ctypes.c_char_p(b"invalid argument").value
        raise AssertionError(f"C call {name} reached although the arguments were refused")


def test_binding_rejects_tensors_of_another_device(pcbp, monkeypatch):
    """The C calls launch on the current device: tensors (or a stream) of another GPU are refused
    with PcError(PC_EINVAL) before any C call."""
    import torch

    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    ws_bytes = pcbp.bp_decode_workspace_size(code, 4)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(pcbp, "bp_decode_workspace_size", lambda code, B: ws_bytes)
    monkeypatch.setattr(pcbp, "_lib", _NoCalls())
    B, KW = 4, pcbp.words_of(128)

    def args(dev_llr=0, dev_ws=0, dev_out=0):
        return (_FakeDeviceTensor((B, 256), torch.float32, dev_llr), _FakeDeviceTensor((B, KW), torch.int32, dev_out),
                _FakeDeviceTensor((B,), torch.int32, dev_out), _FakeDeviceTensor((B,), torch.uint8, dev_out),
                _FakeDeviceTensor((ws_bytes,), torch.uint8, dev_ws))

    s = pcbp.sched()
    for kw in ({"dev_llr": 1}, {"dev_ws": 1}, {"dev_out": 1}):
        llr, bits, iters, ok, ws = args(**kw)
        calls = [lambda: pcbp.bp_decode(code, llr, s, 10, bits, iters, ok, ws),
                 lambda: pcbp.bp_decode_host(code, llr, s, 10, bits, iters, ok, ws)]
        if "dev_ws" not in kw:      # bp_decode_noalloc takes no workspace
            calls.append(lambda: pcbp.bp_decode_noalloc(code, llr, s, 10, bits, iters, ok))
        for call in calls:
            with pytest.raises(pcbp.PcError) as e:
                call()
            assert e.value.status == pcbp.PC_EINVAL, kw

    class _Stream:
        device = torch.device("cuda", 1)
        cuda_stream = 0

    llr, bits, iters, ok, ws = args()
    for call in (lambda: pcbp.bp_decode(code, llr, s, 10, bits, iters, ok, ws, _Stream()),
                 lambda: pcbp.bp_decode_noalloc(code, llr, s, 10, bits, iters, ok, _Stream()),
                 lambda: pcbp.pc_encode(code, _FakeDeviceTensor((B, 120), torch.uint8, 0),
                                        _FakeDeviceTensor((B, 256), torch.uint8, 0), _Stream())):
        with pytest.raises(pcbp.PcError) as e:
            call()
        assert e.value.status == pcbp.PC_EINVAL


@no_gpu_only
def test_posterior_and_f_eval_validate_before_touching_the_device(pcbp):
    """bp_decode_posterior refuses lengths that run another kernel, the G-matrix stop and a missing
    output; pc_f_eval refuses an unknown f and a negative count; all on the host."""
    p = C.c_void_p
    s = pcbp.sched(mode=1, P_range=3, P_level=5, N_min=5, T0=5)
    code = pcbp.pc_construct(256, 128, 8, 0x9B)
    small = pcbp.pc_construct(64, 32, 8, 0x9B)
    post = pcbp._lib.bp_decode_posterior

    def call(c, sch, out=p(65536), B=4):
        return post(C.byref(c), p(4096), C.byref(sch), 10, B, p(8192), p(12288), p(16384), out, p(32768), None)

    assert call(small, s) == pcbp.PC_EUNSUPPORTED                  # N < 128: another kernel
    assert call(code, pcbp.sched(stop_kind=3)) == pcbp.PC_EUNSUPPORTED
    assert call(code, s, out=None) == pcbp.PC_EINVAL
    assert call(code, s, out=p(65536 + 2)) == pcbp.PC_EINVAL        # misaligned
    assert call(code, pcbp.sched(mode=3)) == pcbp.PC_EINVAL
    assert call(code, s, B=0) == pcbp.PC_OK
    f = pcbp._lib.pc_f_eval
    assert f(p(4096), p(8192), p(12288), 10, 2, 1.0, None) == pcbp.PC_EINVAL
    assert f(p(4096), p(8192), p(12288), -1, 0, 1.0, None) == pcbp.PC_EINVAL
    assert f(None, p(8192), p(12288), 10, 0, 1.0, None) == pcbp.PC_EINVAL
    assert f(p(4098), p(8192), p(12288), 10, 0, 1.0, None) == pcbp.PC_EINVAL
    assert f(None, None, None, 0, 1, 1.0, None) == pcbp.PC_OK
