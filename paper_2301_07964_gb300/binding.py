"""Thin ctypes binding of the C ABI in ``include/hts.h``.

The functions below carry the C names and marshal arguments only: matrices may be given as
device pointers (int) or as CUDA torch tensors in column-major layout (stride(0) == 1), whose
data pointer is passed; streams may be a torch.cuda.Stream, a raw handle or None (legacy
default stream).  Every step of the reduction runs in the CUDA library; if the library
cannot be loaded these functions raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhts.so")

HTS_OK = 0
HTS_ERR_ARG = 1
HTS_ERR_CUDA = 2
HTS_ERR_WORKSPACE = 3
HTS_ERR_TIMEOUT = 4
HTS_ERR_NONFINITE = 5
HTS_ERR_UNSUPPORTED = 6

HTS_COMP_NONE = 0
HTS_COMP_INIT = 1
HTS_COMP_UPDATE = 2

HTS_GEMM_FP64 = 0
HTS_GEMM_EMU_BF16 = 1

HTS_FLAG_NO_CLEAN = 1
HTS_FLAG_SERIAL_UPDATES = 2
HTS_FLAG_TEST_STALL = 1 << 30
HTS_FLAG_TEST_DIRECT_RQ = 1 << 29


class hts_params(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("p", ctypes.c_int), ("emu_slices", ctypes.c_int),
                ("tile_m", ctypes.c_int), ("tile_n", ctypes.c_int), ("flags", ctypes.c_int)]


HTS_K_NKINDS = 12
KERNEL_KINDS = {0: "k_s2_generate", 1: "k_s2_apply_right", 2: "k_s2_apply_left", 3: "util", 4: "stage1",
                5: "k_s2_apply_right_qz", 6: "k_reduce_batched", 7: "k_s2_form_u", 8: "k_s2_emu_apply_right",
                9: "k_s2_emu_apply_left", 10: "k_s2_emu_apply_qz", 11: "k_s2_update"}


class hts_kernel_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("mma_flops", ctypes.c_double)]


class HTSError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s failed: %s" % (what, status_string(status)))


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_RED_ARGS = [_VP, _I, _I, _VP, _I, _VP, _I, _I, _VP, _I, _I, _VP, _I, _I,
             ctypes.POINTER(hts_params), _VP, ctypes.c_size_t, _VP]
_REDUCE_FUNCS = ("hts_reduce_stage1", "hts_reduce_stage2", "hts_reduce")


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises OSError if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libhts.so not built at %s (run __graft_entry__.build())" % path)
    lib = ctypes.CDLL(path)
    lib.hts_create.argtypes = [ctypes.POINTER(_VP), _I]
    lib.hts_create.restype = _I
    lib.hts_destroy.argtypes = [_VP]
    lib.hts_destroy.restype = None
    lib.hts_workspace_size.argtypes = [_I, _I, ctypes.POINTER(hts_params), ctypes.POINTER(ctypes.c_size_t)]
    lib.hts_workspace_size.restype = _I
    for name in _REDUCE_FUNCS:
        f = getattr(lib, name)
        f.argtypes = _RED_ARGS
        f.restype = _I
    lib.hts_reduce_stage2_noalloc.argtypes = _RED_ARGS[:15] + [_VP]
    lib.hts_reduce_stage2_noalloc.restype = _I
    IP = ctypes.POINTER(ctypes.c_int)
    PP = ctypes.POINTER(_VP)
    lib.hts_workspace_size_batched.argtypes = [_I, IP, IP, ctypes.POINTER(hts_params), ctypes.POINTER(ctypes.c_size_t)]
    lib.hts_workspace_size_batched.restype = _I
    lib.hts_reduce_batched.argtypes = [_VP, _I, IP, IP, PP, IP, PP, IP, _I, PP, IP, _I, PP, IP, _I,
                                       ctypes.POINTER(hts_params), _VP, ctypes.c_size_t, _VP]
    lib.hts_reduce_batched.restype = _I
    lib.hts_plan_batched.argtypes = [_VP, _I, IP, IP, PP, IP, PP, IP, _I, PP, IP, _I, PP, IP, _I,
                                     ctypes.POINTER(hts_params), _VP, ctypes.c_size_t, _VP]
    lib.hts_plan_batched.restype = _I
    lib.hts_reduce_batched_planned.argtypes = [_VP, _I, _VP, ctypes.c_size_t, _VP]
    lib.hts_reduce_batched_planned.restype = _I
    lib.hts_sync_status.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_int)]
    lib.hts_sync_status.restype = _I
    lib.hts_status_string.argtypes = [_I]
    lib.hts_status_string.restype = ctypes.c_char_p
    lib.hts_profile_begin.argtypes = [_VP, _I]
    lib.hts_profile_begin.restype = _I
    lib.hts_profile_end.argtypes = [_VP, ctypes.POINTER(hts_kernel_profile), ctypes.POINTER(ctypes.c_int)]
    lib.hts_profile_end.restype = _I
    lib.hts_probe_fp64_peak.argtypes = [_VP, ctypes.POINTER(ctypes.c_double)]
    lib.hts_probe_fp64_peak.restype = _I
    lib.hts_fallback_count.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_longlong)]
    lib.hts_fallback_count.restype = _I
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("expected a device pointer or a torch tensor, got %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    raise TypeError("expected a torch.cuda.Stream, an int handle or None")


def _params(p):
    if p is None:
        return None
    if isinstance(p, hts_params):
        return ctypes.byref(p)
    if isinstance(p, dict):
        return ctypes.byref(hts_params(**p))
    raise TypeError("params must be hts_params, dict or None")


def status_string(status: int) -> str:
    try:
        return load().hts_status_string(int(status)).decode()
    except OSError:
        return "status %d" % status


def hts_create(device: int = 0):
    ctx = _VP()
    st = load().hts_create(ctypes.byref(ctx), int(device))
    if st != HTS_OK:
        raise HTSError(st, "hts_create")
    return ctx


def hts_destroy(ctx):
    load().hts_destroy(ctx)


def hts_workspace_size(n: int, r: int, params=None) -> int:
    out = ctypes.c_size_t(0)
    st = load().hts_workspace_size(int(n), int(r), _params(params), ctypes.byref(out))
    if st != HTS_OK:
        raise HTSError(st, "hts_workspace_size")
    return out.value


def _reduce(name, ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params, work,
            work_bytes, stream):
    f = getattr(load(), name)
    return f(ctx, int(n), int(r), _ptr(A), int(lda), _ptr(B), int(ldb), int(compq), _ptr(Q), int(ldq),
             int(compz), _ptr(Z), int(ldz), int(mode), _params(params), _ptr(work), int(work_bytes),
             _stream(stream))


def hts_reduce_stage1(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params, work,
                      work_bytes, stream=None) -> int:
    return _reduce("hts_reduce_stage1", ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode,
                   params, work, work_bytes, stream)


def hts_reduce_stage2(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params, work,
                      work_bytes, stream=None) -> int:
    return _reduce("hts_reduce_stage2", ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode,
                   params, work, work_bytes, stream)


def hts_reduce_stage2_noalloc(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params,
                              stream=None) -> int:
    """Stage 2 with the library's fixed scratch array instead of a caller workspace."""
    return load().hts_reduce_stage2_noalloc(ctx, int(n), int(r), _ptr(A), int(lda), _ptr(B), int(ldb),
                                            int(compq), _ptr(Q), int(ldq), int(compz), _ptr(Z), int(ldz),
                                            int(mode), _params(params), _stream(stream))


def hts_reduce(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params, work,
               work_bytes, stream=None) -> int:
    return _reduce("hts_reduce", ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode,
                   params, work, work_bytes, stream)


def _iarr(vals):
    return (ctypes.c_int * max(1, len(vals)))(*[int(v) for v in vals])


def _parr(vals):
    return (_VP * max(1, len(vals)))(*[_ptr(v) for v in vals])


def hts_workspace_size_batched(n, r, params=None) -> int:
    out = ctypes.c_size_t(0)
    st = load().hts_workspace_size_batched(len(n), _iarr(n), _iarr(r), _params(params), ctypes.byref(out))
    if st != HTS_OK:
        raise HTSError(st, "hts_workspace_size_batched")
    return out.value


def hts_plan_batched(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params, work, work_bytes,
                     stream=None) -> int:
    """Same arguments as hts_reduce_batched; writes the plan into work."""
    count = len(n)
    Qs = Q if Q is not None else [None] * count
    Zs = Z if Z is not None else [None] * count
    return load().hts_plan_batched(ctx, count, _iarr(n), _iarr(r), _parr(A), _iarr(lda), _parr(B), _iarr(ldb),
                                   int(compq), _parr(Qs), _iarr(ldq if ldq is not None else [1] * count),
                                   int(compz), _parr(Zs), _iarr(ldz if ldz is not None else [1] * count),
                                   int(mode), _params(params), _ptr(work), int(work_bytes), _stream(stream))


def hts_reduce_batched_planned(ctx, count, work, work_bytes, stream=None) -> int:
    return load().hts_reduce_batched_planned(ctx, int(count), _ptr(work), int(work_bytes), _stream(stream))


def hts_reduce_batched(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, params, work, work_bytes,
                       stream=None) -> int:
    """Lists of length count: sizes, r, matrices (device pointers or tensors) and leading dimensions."""
    count = len(n)
    Qs = Q if Q is not None else [None] * count
    Zs = Z if Z is not None else [None] * count
    return load().hts_reduce_batched(ctx, count, _iarr(n), _iarr(r), _parr(A), _iarr(lda), _parr(B), _iarr(ldb),
                                     int(compq), _parr(Qs), _iarr(ldq if ldq is not None else [1] * count),
                                     int(compz), _parr(Zs), _iarr(ldz if ldz is not None else [1] * count),
                                     int(mode), _params(params), _ptr(work), int(work_bytes), _stream(stream))


def hts_sync_status(ctx, stream=None):
    """Returns (status, [pencil, group, k, j])."""
    info = (ctypes.c_int * 4)()
    st = load().hts_sync_status(ctx, _stream(stream), info)
    return st, list(info)


def hts_profile_begin(ctx, max_launches: int):
    st = load().hts_profile_begin(ctx, int(max_launches))
    if st != HTS_OK:
        raise HTSError(st, "hts_profile_begin")


def hts_profile_end(ctx):
    """Returns ({kind name: {launches, ms, flops, bytes, mma_flops}}, dropped)."""
    out = (hts_kernel_profile * HTS_K_NKINDS)()
    dropped = ctypes.c_int(0)
    st = load().hts_profile_end(ctx, out, ctypes.byref(dropped))
    if st != HTS_OK:
        raise HTSError(st, "hts_profile_end")
    res = {}
    for k in range(HTS_K_NKINDS):
        if out[k].launches:
            res[KERNEL_KINDS.get(k, "kind%d" % k)] = dict(launches=out[k].launches, ms=out[k].ms,
                                                         flops=out[k].flops, bytes=out[k].bytes,
                                                         mma_flops=out[k].mma_flops)
    return res, dropped.value


def hts_probe_fp64_peak(stream=None) -> float:
    v = ctypes.c_double(0.0)
    st = load().hts_probe_fp64_peak(_stream(stream), ctypes.byref(v))
    if st != HTS_OK:
        raise HTSError(st, "hts_probe_fp64_peak")
    return v.value


def hts_fallback_count(ctx, stream=None) -> int:
    """Chase steps whose elimination-based opposite reflector was redone with the RQ since the
    previous query (waits for the stream)."""
    v = ctypes.c_longlong(0)
    st = load().hts_fallback_count(ctx, _stream(stream), ctypes.byref(v))
    if st != HTS_OK:
        raise HTSError(st, "hts_fallback_count")
    return v.value
