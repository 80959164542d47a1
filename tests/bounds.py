"""Error bounds of the GPU parity tests, derived from the arithmetic of each leaf kind.

The normalised error of a result is max|C - C_ref| / (k max|A| max|B|) (k the inner
dimension), C_ref the FP64 oracle.  Each bound below models the error of one element of C as a
sum of many small independent rounding contributions, takes its root mean square from the
operands' own second moments (not from max|a||b|, which overstates a product term about 3x on
uniform data), and covers the largest of N compared elements with the Gaussian tail factor
z(N) = sqrt(2 ln 2N).  A fixed safety factor then covers what the model leaves out (tails
heavier than Gaussian, correlations between the operand sums of one level).

Per recursion level the error of one C quadrant is the signed sum of the errors of the products
that feed it (Sec. 2.2 / 2.3).  A product P = S T of two operand sums with n_s and n_t block
terms has n_s n_t times the error variance of a plain block product over the same inner length
k/2, so quadrant q gets R_q = (1/2) sum_{P -> q} n_s n_t times the variance of the undivided
product.  Worst quadrant, per level:
  BDPZ / Knuth (Sec. 2.3):  C12 = P1 + P6 + P5 + P3 -> (1 + 9 + 4 + 4) / 2 = 9
  Strassen (Sec. 2.2):      C11 = P1 + P4 - P5 + P7 -> (4 + 2 + 2 + 4) / 2 = 6
so the RMS of a term-rounding error grows by sqrt(R) per level.

TF32 leaves.  The tensor core reads an FP32 operand as TF32, keeping 10 mantissa bits; we take
the worst case of truncation (round-to-nearest halves every figure below).  An operand x is read
as x (1 + d) with d in (-2^-10, 0]: |E d| <= 2^-11 and E d^2 <= 2^-20 / 3 whatever the mantissa.
A product term a b then errs by a b (mu + xi): the mean mu (|mu| <= 2^-10 for both operands)
adds up coherently to mu * c_ij, i.e. a relative error of the result itself that recursion does
not amplify (every leaf result carries the same mu), while the zero-mean part xi
(E xi^2 <= 2 * 2^-20 / 3) is a random walk over the k terms that grows by sqrt(R) per level.
With rho = sqrt(E a^2 E b^2) / (max|a| max|b|) and c_ij of RMS sqrt(k) E|ab|:
    tol = F z(N) 2^-10 rho sqrt(1 + (2/3) R^L) / sqrt(k) + 2^-20,
F = 2.  The 2^-20 term allows for the FP32 accumulation of the tensor core.  Where the fixed TF32
bound of 2e-4 set for these workloads applies (k >= 4096, L <= 2) the smaller of the two is used.

Compensated leaves (split-BF16 and 3xTF32).  The operand split carries x to a relative error e
(split-BF16: hi = bf16(x), lo = bf16(x - hi) and the dropped lo*lo term give a term error of
RMS below 2^-18; 3xTF32: hi = tf32(x) and lo read as TF32 truncate lo by at most 2^-10 |lo| <=
2^-21 |x|, uniformly, RMS 2^-21 / sqrt(3), the dropped lo*lo term below 2^-22).  These terms
behave like the TF32 ones with 2^-10 replaced by e.  What dominates is the FP32 accumulator:
each MMA adds its partial sum into the accumulator with one rounding of relative size below
u = 2^-23 (a truncating FP32 accumulate; the tensor core's rounding is not
documented, so the worse of truncation and rounding to nearest is assumed), all of one sign in
the worst case.  With n_mma MMAs of depth K per k-step (split-BF16: 3 of K = 16; 3xTF32: 3 of
K = 8) the accumulated error is u n_mma sum_j |D_j| with |D_j| ~ sqrt(2/pi) sqrt(K j) RMS(ab),
which gives u (2/3) sqrt(2/pi) (n_mma / K) sqrt(k) rho (normalised).  Per level the leaf depth
halves and the operand sums grow, a factor sqrt(2 R) / 2^1.5 (1.5 for BDPZ); the leaf results
add in FP32 (rounding to nearest, negligible).
    tol = F [z(N) e rho sqrt(R^L) / sqrt(k) + u (2/3) sqrt(2/pi) (n_mma / K) sqrt(k) rho g^L],
F = 4 (the accumulator model is the loosest part of the derivation).

FP64 (SIMT leaves, every operation rounded to nearest, u = 2^-53).  Rounding to nearest leaves
an error uniform within half an ulp, RMS ulp / sqrt(12) <= u |s| / sqrt(3) for a result s.  A
leaf of inner length k' = k / 2^L accumulates its terms one FMA at a time; the rounding errors
form a random walk over partial sums of RMS sqrt(j) RMS(st), so a leaf result errs by about
(u / sqrt(3)) k' RMS(s) RMS(t) / sqrt(2); over the leaves of the worst quadrant this grows by
sqrt(R / 2) per level.  The operand sums add one rounding each (behaving like a term error).
    tol = F z(N) (u / sqrt(3)) rho (sqrt((R / 2)^L / 2) + sqrt(R^L / k)),  F = 4,
and the fixed FP64 bound 1e-13 is checked as well.

A result may be compared on sampled rows; N is then the number of compared elements.
"""
from __future__ import annotations

import math

import numpy as np

# per-level growth of the worst quadrant's error variance
GROWTH = {"naive": 1.0, "winograd": 9.0, "knuth": 9.0, "strassen": 6.0}


def z_tail(nelem: int) -> float:
    """Gaussian tail factor for the largest of nelem independent errors."""
    return math.sqrt(2.0 * math.log(2.0 * max(int(nelem), 1)))


def rho(A, B) -> float:
    """RMS of a product term over the largest one: sqrt(E a^2 E b^2) / (max|a| max|b|)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    am, bm = float(np.max(np.abs(A))), float(np.max(np.abs(B)))
    if am == 0.0 or bm == 0.0:
        return 0.0
    return math.sqrt(float(np.mean(A * A)) * float(np.mean(B * B))) / (am * bm)


def tol_tf32(nelem: int, k: int, L: int, A, B, algo: str = "winograd") -> float:
    R = GROWTH[algo] if L > 0 else 1.0
    t = 2.0 * z_tail(nelem) * 2.0 ** -10 * rho(A, B) * math.sqrt(1.0 + (2.0 / 3.0) * R ** L) / math.sqrt(k)
    t += 2.0 ** -20
    if k >= 4096 and L <= 2:
        t = min(t, 2e-4)
    return t


def _tol_compensated(nelem, k, L, A, B, algo, e, n_mma, K):
    R = GROWTH[algo] if L > 0 else 1.0
    r = rho(A, B)
    g = math.sqrt(2.0 * R) / 2.0 ** 1.5 if L > 0 else 1.0
    term = z_tail(nelem) * e * r * math.sqrt(R ** L) / math.sqrt(k)
    acc = 2.0 ** -23 * (2.0 / 3.0) * math.sqrt(2.0 / math.pi) * (n_mma / K) * math.sqrt(k) * r * g ** L
    return 4.0 * (term + acc)


def tol_bf16x3(nelem: int, k: int, L: int, A, B, algo: str = "winograd") -> float:
    return _tol_compensated(nelem, k, L, A, B, algo, 2.0 ** -18, 3, 16)


def tol_tf32x3(nelem: int, k: int, L: int, A, B, algo: str = "winograd") -> float:
    return _tol_compensated(nelem, k, L, A, B, algo, 2.0 ** -21 / math.sqrt(3.0), 3, 8)


def tol_fp64(nelem: int, k: int, L: int, A, B, algo: str = "winograd") -> float:
    R = GROWTH[algo] if L > 0 else 1.0
    u = 2.0 ** -53 / math.sqrt(3.0)
    t = 4.0 * z_tail(nelem) * u * rho(A, B) * (math.sqrt((R / 2.0) ** L / 2.0) + math.sqrt(R ** L / k))
    return min(t, 1e-13)
