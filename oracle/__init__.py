"""FP64 CPU oracle for the Strassen / Strassen-Winograd matrix product.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path never does.
It shares no code with the CUDA path.  The arithmetic lives in ``oracle.c``
(plain C, IEEE binary64, no FMA contraction); this module compiles it with gcc on
first use and wraps it for numpy arrays.

Algorithms (``alg`` argument of :func:`recursive`):
  0 Strassen (Sec. 2.2, Alg. 2)              1 Winograd, BDPZ 22-op form (Sec. 2.3, Alg. 3)
  2 Winograd, Knuth's form (Sec. 2.3)         3 Two-Temp schedule (Sec. 3.3, Table 2)
  4 In-Place schedule (Sec. 3.3, Table 3; square only, overwrites copies of A, B)
Odd sizes: ``mode`` PAD (zero padding to a multiple of 2^L, Sec. 3.1) or PEEL.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

PAD, PEEL = 0, 1
STRASSEN, WINOGRAD, KNUTH, TWO_TEMP, IN_PLACE = 0, 1, 2, 3, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (cached by source hash)."""
    src = open(_SRC, "rb").read()
    tag = hashlib.sha1(src).hexdigest()[:12]
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"liboracle_{tag}.so")
    if force or not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return so


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    L = ctypes.c_long
    lib.orc_naive.argtypes = [L, L, L, dp, L, dp, L, dp, L]
    lib.orc_naive_mt.argtypes = [L, L, L, dp, L, dp, L, dp, L, ctypes.c_int]
    lib.orc_max_threads.restype = ctypes.c_int
    lib.orc_depth.argtypes = [L, L, L, L]
    lib.orc_depth.restype = ctypes.c_int
    lib.orc_cutoff_model.argtypes = [ctypes.c_double] * 3 + [dp, dp]
    lib.orc_recursive.argtypes = [ctypes.c_int, L, L, L, dp, L, dp, L, dp, L, L, ctypes.c_int, dp]
    lib.orc_recursive.restype = ctypes.c_int
    lib.orc_workspace_elems.argtypes = [ctypes.c_int, L, L, L, ctypes.c_int]
    lib.orc_workspace_elems.restype = ctypes.c_double
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_schedule_table.argtypes = [ctypes.c_int, ip]
    lib.orc_recursive_table.argtypes = [ip, ctypes.c_int, L, L, L, dp, dp, dp, L, dp]
    lib.orc_recursive_table.restype = ctypes.c_int
    lib.orc_recursive_products.argtypes = [ctypes.c_int, L, L, L, dp, L, dp, L, dp, L, L, ctypes.c_uint]
    lib.orc_recursive_products.restype = ctypes.c_int
    lib.orc_err_norm.argtypes = [L, L, L, dp, L, dp, L, dp, L, dp, L]
    lib.orc_err_norm.restype = ctypes.c_double
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def naive(A, B) -> np.ndarray:
    """Alg. 1: C = A B, FP64, inner index ascending."""
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.zeros((m, n), np.float64)
    _load().orc_naive(m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(C), max(n, 1))
    return C


def naive_mt(A, B, threads: int = 0) -> np.ndarray:
    """Alg. 1 with rows spread over host threads (same bits as :func:`naive`)."""
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    _, n = B.shape
    C = np.zeros((m, n), np.float64)
    _load().orc_naive_mt(m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(C), max(n, 1), threads)
    return C


def max_threads() -> int:
    return int(_load().orc_max_threads())


def depth(m: int, n: int, k: int, cutoff: int) -> int:
    """Number of recursion levels: halve while min dimension > cutoff (Sec. 3.4)."""
    return int(_load().orc_depth(m, n, k, cutoff))


def cutoff_model(m: float, k: float, n: float):
    """(lhs, rhs) of the Sec. 3.4 inequality built from the op counts M and G."""
    l, r = ctypes.c_double(), ctypes.c_double()
    _load().orc_cutoff_model(m, k, n, ctypes.byref(l), ctypes.byref(r))
    return l.value, r.value


def recursive(alg: int, A, B, cutoff: int, mode: int = PAD, trace: bool = False):
    """Recursive product with the chosen algorithm / schedule, naive below the cutoff.

    Returns C, or (C, trace_vector) when ``trace`` is set: the [0][0] element of
    each top-level intermediate (numbering documented in oracle.c).
    Raises RuntimeError if a schedule's liveness shadow failed.
    """
    A, B = _f64(A).copy(), _f64(B).copy()
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.zeros((m, n), np.float64)
    tv = np.full(32, np.nan)
    rc = _load().orc_recursive(alg, m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(C), max(n, 1),
                               cutoff, mode, _p(tv) if trace else None)
    if rc == 1:
        raise ValueError("bad arguments")
    if rc == 2:
        raise RuntimeError("schedule liveness shadow failed")
    return (C, tv) if trace else C


def recursive_products(alg: int, A, B, cutoff: int, mask: int) -> np.ndarray:
    """The top-level products in `mask` only (bit i = product i+1 of Sec. 2.2 / 2.3; Knuth's form
    in the BDPZ numbering), the others taken as zero: their contribution to C = A B.  Zero padding
    (Sec. 3.1); the depth must be >= 1."""
    A, B = _f64(A).copy(), _f64(B).copy()
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), np.float64)
    rc = _load().orc_recursive_products(alg, m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(C), max(n, 1),
                                        cutoff, mask)
    if rc != 0:
        raise ValueError("bad arguments (algorithm, mask or depth 0)")
    return C


def workspace_elems(sched: int, m: int, n: int, k: int, L: int) -> float:
    """Peak temporary elements: sched 0 = allocating Alg. 3, 1 = two-temp (Table 2)."""
    return float(_load().orc_workspace_elems(sched, m, n, k, L))


def err_norm(C, R, A, B) -> float:
    """max|C - R| / (k * max|A| * max|B|)."""
    C, R, A, B = _f64(C), _f64(R), _f64(A), _f64(B)
    m, n = C.shape
    k = A.shape[1]
    return float(_load().orc_err_norm(m, n, k, _p(C), max(n, 1), _p(R), max(n, 1), _p(A), max(k, 1),
                                      _p(B), max(n, 1)))


def schedule_table(which: int) -> np.ndarray:
    """Table 2 (which=0) or Table 3 (which=1) as a 22 x 5 int array {op, val, dst, v1, v2}."""
    out = np.zeros(22 * 5, np.int32)
    _load().orc_schedule_table(which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out.reshape(22, 5)


def run_table(tab, A, B, cutoff: int, trace: bool = False, two_temp: bool = False):
    """Run a (possibly perturbed) 22-step table: with Table 3's rules (in place, square inputs,
    the default) or, with two_temp=True, Table 2's (temporaries X and Y, any shape).

    Raises RuntimeError when the liveness shadow finds a read of a dead value."""
    tab = np.ascontiguousarray(np.asarray(tab, np.int32).reshape(-1))
    A, B = _f64(A).copy(), _f64(B).copy()
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), np.float64)
    tv = np.full(32, np.nan)
    rc = _load().orc_recursive_table(tab.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), 1 if two_temp else 0,
                                     m, n, k, _p(A), _p(B), _p(C), cutoff, _p(tv) if trace else None)
    if rc == 1:
        raise ValueError("bad table")
    if rc == 2:
        raise RuntimeError("schedule liveness shadow failed")
    return (C, tv) if trace else C
