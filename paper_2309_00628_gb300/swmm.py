"""ctypes binding of libswmm (include/swmm.h): argument marshalling only.

Every function keeps the C name and returns the C status, except where noted.
All arithmetic runs in the CUDA library; if the library has not been built this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SW_OK, SW_EINVAL, SW_ENOMEM, SW_EBUDGET, SW_ECUDA, SW_ETIMEOUT, SW_EUNSUPPORTED = range(7)
STATUS_NAMES = ["SW_OK", "SW_EINVAL", "SW_ENOMEM", "SW_EBUDGET", "SW_ECUDA", "SW_ETIMEOUT", "SW_EUNSUPPORTED"]

SW_ALGO_NAIVE, SW_ALGO_STRASSEN, SW_ALGO_WINOGRAD, SW_ALGO_WINOGRAD_KNUTH = 0x0, 0x1, 0x2, 0x3
SW_SCHED_FUSED, SW_SCHED_TWO_TEMP, SW_SCHED_IN_PLACE, SW_SCHED_ALLOC = 0x00, 0x10, 0x20, 0x30
SW_PAD, SW_PEEL = 0x000, 0x100
SW_LEAF_TF32, SW_LEAF_BF16X3, SW_LEAF_TF32X3, SW_LEAF_F64_WTILE = 0x0000, 0x1000, 0x2000, 0x3000
SW_NOALLOC_SCRATCH_BYTES = 32 << 20  # the static device array of sw_smm_noalloc


class sw_problem(ctypes.Structure):
    """C <- A B, FP32, row-major, device pointers (include/swmm.h)."""
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("k", ctypes.c_int)]


class sw_server_cfg(ctypes.Structure):
    """Serving-loop parameters (include/swmm.h); zero fields take the documented defaults."""
    _fields_ = [("sm_share", ctypes.c_int), ("max_inflight", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
                ("idle_us", ctypes.c_int)]


class sw_request(ctypes.Structure):
    """One served product: elem_bytes 4 (as sw_smm) or 8 (as sw_dmm), device pointers."""
    _fields_ = [("elem_bytes", ctypes.c_int), ("A", ctypes.c_void_p), ("lda", ctypes.c_int),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int), ("C", ctypes.c_void_p), ("ldc", ctypes.c_int),
                ("m", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int), ("cutoff", ctypes.c_int),
                ("variant", ctypes.c_uint32)]


class SwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_lib = None
_V, _I, _U, _S, _P = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t, ctypes.POINTER


def library_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = False):
    """Load libswmm.so; raises if it is not built (or builds it when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    so = _build.lib_path()
    if not os.path.exists(so):
        if not build_if_missing:
            raise RuntimeError(f"libswmm is not built ({so} missing): run __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(so)
    lib.sw_create.argtypes = [_P(_V), _S]
    lib.sw_destroy.argtypes = [_V]
    lib.sw_last_error.argtypes = [_V]
    lib.sw_last_error.restype = ctypes.c_char_p
    lib.sw_mm_workspace_size.argtypes = [_I, _I, _I, _I, _U, _I, _P(_S)]
    lib.sw_mm_depth.argtypes = [_I, _I, _I, _I, _U, _I, _P(_I)]
    mm = [_V, _V, _I, _V, _I, _V, _I, _I, _I, _I, _I, _U, _V]
    lib.sw_smm.argtypes = mm
    lib.sw_dmm.argtypes = mm
    lib.sw_smm_host.argtypes = mm
    lib.sw_sync.argtypes = [_V, _V]
    lib.sw_error_norms.argtypes = [_V, _I, _I, _I, _I, _V, _I, _V, _I, _V, _I, _V, _I, _P(ctypes.c_double), _V]
    lib.sw_mm_batched.argtypes = [_V, _I, _P(sw_problem), _I, _U, _V]
    lib.sw_mm_batched.restype = _I
    lib.sw_profile.argtypes = [_V, _I]
    lib.sw_profile_read.argtypes = [_V, _I, _P(_I), _P(ctypes.c_double)]
    lib.sw_last_tuning.argtypes = [_V, _P(_I), _P(_I), _P(_I), _P(ctypes.c_double), _P(_I)]
    lib.sw_server_start.argtypes = [_V, _P(sw_server_cfg)]
    lib.sw_server_submit.argtypes = [_V, _P(sw_request), _P(ctypes.c_uint64)]
    lib.sw_server_wait.argtypes = [_V, ctypes.c_uint64, ctypes.c_int64]
    lib.sw_server_stop.argtypes = [_V]
    lib.sw_selftest_expired_wait.argtypes = [_V, _V]
    lib.sw_mm_products.argtypes = [_V, _I, _V, _I, _V, _I, _V, _I, _I, _I, _I, _I, _U, _U, _V]
    for name in ("sw_create", "sw_destroy", "sw_mm_workspace_size", "sw_mm_depth", "sw_smm", "sw_dmm",
                 "sw_smm_host", "sw_sync", "sw_error_norms", "sw_profile", "sw_profile_read", "sw_server_start",
                 "sw_server_submit", "sw_server_wait", "sw_server_stop", "sw_selftest_expired_wait",
                 "sw_mm_products"):
        getattr(lib, name).restype = _I
    _lib = lib
    return lib


# ------------------------------------------------------------------ C names
def sw_create(budget: int = 0):
    h = _V()
    st = load().sw_create(ctypes.byref(h), budget)
    if st != SW_OK:
        raise SwError(st, "sw_create failed")
    return h


def sw_destroy(h) -> int:
    return load().sw_destroy(h)


def sw_last_error(h) -> str:
    r = load().sw_last_error(h)
    return r.decode() if r else ""


def sw_mm_workspace_size(m, n, k, cutoff, variant, elem_bytes):
    b = _S()
    st = load().sw_mm_workspace_size(m, n, k, cutoff, variant, elem_bytes, ctypes.byref(b))
    return st, b.value


def sw_mm_depth(m, n, k, cutoff, variant, elem_bytes):
    d = _I()
    st = load().sw_mm_depth(m, n, k, cutoff, variant, elem_bytes, ctypes.byref(d))
    return st, d.value


def sw_smm(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream=None) -> int:
    return load().sw_smm(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream)


def sw_dmm(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream=None) -> int:
    return load().sw_dmm(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream)


def sw_mm_products(h, elem_bytes, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, product_mask, stream=None) -> int:
    return load().sw_mm_products(h, elem_bytes, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, product_mask, stream)


def sw_smm_host(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream=None) -> int:
    return load().sw_smm_host(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream)


def sw_mm_batched(h, count, probs, cutoff, variant, stream=None) -> int:
    """probs: a ctypes array of sw_problem (or a list, converted here)."""
    if not isinstance(probs, ctypes.Array):
        probs = (sw_problem * len(probs))(*probs)
    return load().sw_mm_batched(h, count, probs, cutoff, variant, stream)


def sw_sync(h, stream=None) -> int:
    return load().sw_sync(h, stream)


def sw_error_norms(h, elem_bytes, m, n, k, A, lda, B, ldb, C, ldc, R, ldr, stream=None):
    out = (ctypes.c_double * 3)()
    st = load().sw_error_norms(h, elem_bytes, m, n, k, A, lda, B, ldb, C, ldc, R, ldr, out, stream)
    return st, [out[0], out[1], out[2]]


PROFILE_KINDS = ["gemm_tf32", "gemm_simt", "addsub", "copy_pad", "preadd", "memset", "transpose", "transpose_sq",
                 "split_bf16", "gemm_bf16x3", "batch_copy", "split_tf32", "gemm_tf32x3",
                 "preadd_split"]


def sw_selftest_expired_wait(h, stream=None) -> int:
    """Bounded-wait self-test (see include/swmm.h): SW_ETIMEOUT when a device wait that nothing
    satisfies ends at its bound."""
    return load().sw_selftest_expired_wait(h, stream)


def sw_profile(h, enable: bool) -> int:
    return load().sw_profile(h, 1 if enable else 0)


def sw_profile_read(h):
    """(status, {kind: (launches, total_ms)}) since the last read."""
    n = len(PROFILE_KINDS)
    launches = (ctypes.c_int * n)()
    ms = (ctypes.c_double * n)()
    st = load().sw_profile_read(h, n, launches, ms)
    return st, {PROFILE_KINDS[i]: (launches[i], ms[i]) for i in range(n)}


def sw_last_tuning(h):
    """(status, {"cutoff", "tile_n", "cta_pair", "ms", "candidates"}) of the autotuner's last decision."""
    c, t, pr, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    st = load().sw_last_tuning(h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(pr), ctypes.byref(ms),
                               ctypes.byref(nc))
    return st, {"cutoff": c.value, "tile_n": t.value, "cta_pair": pr.value, "ms": ms.value, "candidates": nc.value}


def sw_server_start(h, cfg: sw_server_cfg | None = None) -> int:
    return load().sw_server_start(h, ctypes.byref(cfg) if cfg is not None else None)


def sw_server_submit(h, req: sw_request):
    """Returns (status, ticket)."""
    t = ctypes.c_uint64(0)
    st = load().sw_server_submit(h, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def sw_server_wait(h, ticket: int, timeout_ns: int = -1) -> int:
    return load().sw_server_wait(h, ticket, timeout_ns)


def sw_server_stop(h) -> int:
    return load().sw_server_stop(h)


def request(A, B, C, cutoff: int = 0, variant: int = SW_ALGO_WINOGRAD) -> sw_request:
    """sw_request for C = A @ B on row-major CUDA tensors (float32 or float64)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    eb = 4 if A.dtype == torch.float32 else 8
    return sw_request(eb, A.data_ptr(), max(A.stride(0), 1), B.data_ptr(), max(B.stride(0), 1), C.data_ptr(),
                      max(C.stride(0), 1), m, n, k, cutoff, variant)


def check(h, status: int) -> None:
    """Raise SwError for a non-OK status, with the handle's last error message."""
    if status != SW_OK:
        raise SwError(status, sw_last_error(h))


# ------------------------------------------------------------------ torch marshalling
def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def mm(h, A, B, cutoff: int = 0, variant: int = SW_ALGO_WINOGRAD, out=None, stream=None, sync: bool = False):
    """C = A @ B for row-major CUDA tensors (float32 -> sw_smm, float64 -> sw_dmm)."""
    import torch
    assert A.is_cuda and B.is_cuda and A.dim() == 2 and B.dim() == 2 and A.dtype == B.dtype
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    assert A.stride(1) == 1 and B.stride(1) == 1
    C = out if out is not None else torch.empty((m, n), dtype=A.dtype, device=A.device)
    fn = sw_smm if A.dtype == torch.float32 else sw_dmm
    st = fn(h, ctypes.c_void_p(A.data_ptr()), max(A.stride(0), 1), ctypes.c_void_p(B.data_ptr()), max(B.stride(0), 1),
            ctypes.c_void_p(C.data_ptr()), max(C.stride(0), 1), m, n, k, cutoff, variant, _stream_ptr(stream))
    check(h, st)
    if sync:
        check(h, sw_sync(h, _stream_ptr(stream)))
    return C


def sw_smm_noalloc(A, lda, B, ldb, C, ldc, m, n, k, stream=None) -> int:
    """The no-allocation FP32 Winograd product (see include/swmm.h): all temporaries live in
    the library's static device array, so callers that cannot allocate device memory can use it."""
    fn = load().sw_smm_noalloc
    if fn.argtypes is None:
        fn.argtypes = [_V, _I, _V, _I, _V, _I, _I, _I, _I, _V]
        fn.restype = _I
    return fn(A, lda, B, ldb, C, ldc, m, n, k, stream)
