"""The float bounds of the GPU parity tests (tests/bounds.py) against emulations on the CPU.

TF32: the GPU's TF32 leaves are emulated on the host -- every leaf operand truncated to 10
mantissa bits (the tensor core's reading of an FP32 operand), the operand sums formed in FP32 in
the order of Sec. 2.2 / 2.3, the leaf products and post-additions in FP64 -- and the bound must
cover the emulated error yet stay within 10x of it, at every depth, for both the uniform and the
normal inputs of the configs.  An emulation that keeps three fewer operand bits (a wrong rounding
mode or dropped low-order bits) must exceed the bound.

FP64: the oracle's own FP64 recursions against an extended-precision product: the FP64 bound
covers them within 16x.
"""
import numpy as np
import pytest

import bounds
import oracle
from paper_2309_00628_gb300 import inputs


def _trunc(x, bits=10):
    x = np.ascontiguousarray(x, np.float32)
    mask = np.uint32((0xFFFFFFFF << (23 - bits)) & 0xFFFFFFFF)
    return (x.view(np.uint32) & mask).view(np.float32).astype(np.float64)


def _emulate(A, B, L, algo, bits=10):
    """C = A B with TF32-truncated leaf operands; FP32 operand sums, FP64 products and adds."""
    if L == 0:
        return _trunc(A, bits) @ _trunc(B, bits)
    f = lambda x: x.astype(np.float32)
    h, w, v = A.shape[0] // 2, A.shape[1] // 2, B.shape[1] // 2
    A11, A12, A21, A22 = A[:h, :w], A[:h, w:], A[h:, :w], A[h:, w:]
    B11, B12, B21, B22 = B[:w, :v], B[:w, v:], B[w:, :v], B[w:, v:]
    rec = lambda a, b: _emulate(a, b, L - 1, algo, bits)
    if algo == "winograd":  # the BDPZ form, Sec. 2.3
        S1 = f(A21 + A22); S2 = f(S1 - A11); S3 = f(A11 - A21); S4 = f(A12 - S2)
        T1 = f(B12 - B11); T2 = f(B22 - T1); T3 = f(B22 - B12); T4 = f(T2 - B21)
        P1, P2, P3, P4 = rec(A11, B11), rec(A12, B21), rec(S4, B22), rec(A22, T4)
        P5, P6, P7 = rec(S1, T1), rec(S2, T2), rec(S3, T3)
        U2 = P1 + P6
        U3 = U2 + P7
        C11, C12, C21, C22 = P1 + P2, U2 + P5 + P3, U3 - P4, U3 + P5
    else:  # Strassen, Sec. 2.2
        P1, P2 = rec(f(A11 + A22), f(B11 + B22)), rec(f(A21 + A22), B11)
        P3, P4 = rec(A11, f(B12 - B22)), rec(A22, f(B21 - B11))
        P5, P6, P7 = rec(f(A11 + A12), B22), rec(f(A21 - A11), f(B11 + B12)), rec(f(A12 - A22), f(B21 + B22))
        C11, C12, C21, C22 = P1 + P4 - P5 + P7, P3 + P5, P2 + P4, P1 - P2 + P3 + P6
    return np.block([[C11, C12], [C21, C22]])


def _err(C, A, B):
    R = A.astype(np.float64) @ B.astype(np.float64)
    return float(np.max(np.abs(C - R)) / (A.shape[1] * np.max(np.abs(A)) * np.max(np.abs(B))))


@pytest.mark.parametrize("dist", ["uniform", "normal"])
@pytest.mark.parametrize("algo", ["winograd", "strassen"])
def test_tf32_bound_covers_the_truncation_emulation_within_10x(dist, algo):
    n = 512
    A, B = inputs.pair(n, n, n, dist, seed=3, dtype=np.float32)
    for L in (0, 1, 2, 3):
        err = _err(_emulate(A, B, L, algo), A, B)
        tol = bounds.tol_tf32(n * n, n, L, A, B, algo if L else "naive")
        assert err <= tol <= 10 * err, (L, err, tol)


def test_tf32_bound_catches_three_dropped_bits():
    n = 512
    A, B = inputs.pair(n, n, n, "uniform", seed=4, dtype=np.float32)
    for L in (0, 1, 2):
        err = _err(_emulate(A, B, L, "winograd", bits=7), A, B)
        assert err > bounds.tol_tf32(n * n, n, L, A, B, "winograd" if L else "naive"), L


def test_tf32_bound_applies_the_fixed_bound_where_it_is_tighter():
    A, B = inputs.pair(64, 64, 64, "uniform", seed=5, dtype=np.float32)
    # tiny k: the derived bound exceeds 2e-4, and the fixed bound applies only from k = 4096
    assert bounds.tol_tf32(10 ** 8, 64, 2, A, B) > 2e-4
    assert bounds.tol_tf32(10 ** 8, 4096, 2, np.ones((1, 4096)), np.ones((4096, 1))) == 2e-4


@pytest.mark.parametrize("n,cutoff", [(256, 32), (512, 16)])
def test_fp64_bound_covers_the_oracle_recursions(n, cutoff):
    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float64)
    R = A.astype(np.longdouble) @ B.astype(np.longdouble)
    den = n * np.max(np.abs(A)) * np.max(np.abs(B))
    L = oracle.depth(n, n, n, cutoff)
    for alg, name in ((oracle.WINOGRAD, "winograd"), (oracle.STRASSEN, "strassen"), (oracle.TWO_TEMP, "winograd")):
        C = oracle.recursive(alg, A, B, cutoff)
        err = float(np.max(np.abs(C.astype(np.longdouble) - R)) / den)
        tol = bounds.tol_fp64(C.size, n, L, A, B, name)
        assert err <= tol <= 16 * err, (name, L, err, tol)
    C = oracle.naive(A, B)
    err = float(np.max(np.abs(C.astype(np.longdouble) - R)) / den)
    assert err <= bounds.tol_fp64(C.size, n, 0, A, B, "naive") <= 16 * err
