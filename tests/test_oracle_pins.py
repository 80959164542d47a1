"""Pins for the FP64 CPU oracle, independent of the oracle itself.

Each pin is fixed by the paper or by mathematics, not by re-running the oracle's
own formulas: hand-worked values (tests/golden/worked_2x2.txt, derived from the
formulas of Sec. 2.2 / 2.3), exact rational arithmetic with the classical dot-product
error bound, integer products through numpy's int64 matmul, identity and permutation
matrices, the closed form of the Sec. 3.4 cutoff inequality, Freivalds' identity,
and planted mistakes in copies of Tables 2 and 3 that the liveness shadow must catch.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_2x2.txt")
ALGS = [oracle.STRASSEN, oracle.WINOGRAD, oracle.KNUTH, oracle.TWO_TEMP, oracle.IN_PLACE]
U = 2.0 ** -53


def _golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out[key] = [float(v) for v in vals]
    return out


def _ints(rng, shape, lo=-8, hi=8):
    return rng.integers(lo, hi + 1, size=shape).astype(np.float64)


def _exact_matmul_int(A, B):
    return (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)


# --------------------------------------------------------------------------- 2x2 worked example
def test_worked_2x2_all_forms():
    g = _golden()
    A = np.array(g["A"]).reshape(2, 2)
    B = np.array(g["B"]).reshape(2, 2)
    C = np.array(g["C"]).reshape(2, 2)
    Cs, t = oracle.recursive(oracle.STRASSEN, A, B, cutoff=1, trace=True)
    assert np.array_equal(Cs, C)
    assert t[:7].tolist() == g["strassen_P"]
    for alg in (oracle.WINOGRAD, oracle.TWO_TEMP, oracle.IN_PLACE):
        Cw, t = oracle.recursive(alg, A, B, cutoff=1, trace=True)
        assert np.array_equal(Cw, C), alg
        assert t[8:12].tolist() == g["bdpz_S"], alg
        assert t[12:16].tolist() == g["bdpz_T"], alg
        assert t[16:23].tolist() == g["bdpz_P"], alg
        assert t[23:30].tolist() == g["bdpz_U"], alg
    Ck, t = oracle.recursive(oracle.KNUTH, A, B, cutoff=1, trace=True)
    assert np.array_equal(Ck, C)
    assert t[:3].tolist() == g["knuth_uvw"]
    assert np.array_equal(oracle.naive(A, B), C)


def test_knuth_terms_equal_bdpz_terms():
    # u = P7, v = P5, w = P1 + P6 (Sec. 2.3: the two forms share their products)
    rng = np.random.default_rng(11)
    for _ in range(20):
        A, B = _ints(rng, (2, 2)), _ints(rng, (2, 2))
        _, tk = oracle.recursive(oracle.KNUTH, A, B, 1, trace=True)
        _, tw = oracle.recursive(oracle.WINOGRAD, A, B, 1, trace=True)
        assert tk[0] == tw[22] and tk[1] == tw[20] and tk[2] == tw[16] + tw[21]


@pytest.mark.parametrize("alg", ALGS)
def test_2x2_random_scalars_against_exact(alg):
    # one level on scalars: every form is an exact identity, so the FP64 result
    # must be within a few ulps of the exact rational product
    rng = np.random.default_rng(5 + alg)
    for _ in range(50):
        A, B = rng.uniform(-1, 1, (2, 2)), rng.uniform(-1, 1, (2, 2))
        C = oracle.recursive(alg, A, B, cutoff=1)
        for i in range(2):
            for j in range(2):
                ex = sum(Fraction(A[i, p]) * Fraction(B[p, j]) for p in range(2))
                assert abs(Fraction(C[i, j]) - ex) <= Fraction(64 * U)


# --------------------------------------------------------------------------- naive (Alg. 1)
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 4, 5), (7, 2, 9), (6, 6, 6), (1, 9, 13)])
def test_naive_within_dot_product_bound(m, n, k):
    # |fl(sum) - sum| <= gamma_k sum|a||b|, gamma_k = k u / (1 - k u)
    rng = np.random.default_rng(m * 100 + n * 10 + k)
    A, B = rng.uniform(-1, 1, (m, k)), rng.uniform(-1, 1, (k, n))
    C = oracle.naive(A, B)
    gam = k * U / (1 - k * U)
    for i in range(m):
        for j in range(n):
            ex = sum(Fraction(A[i, p]) * Fraction(B[p, j]) for p in range(k))
            bnd = gam * float(sum(abs(A[i, p] * B[p, j]) for p in range(k)))
            assert abs(float(Fraction(C[i, j]) - ex)) <= bnd * 1.0000001 + 1e-300


def test_naive_integers_match_int64_matmul():
    rng = np.random.default_rng(3)
    for m, n, k in [(17, 9, 33), (64, 64, 64), (1, 100, 7)]:
        A, B = _ints(rng, (m, k)), _ints(rng, (k, n))
        assert np.array_equal(oracle.naive(A, B), _exact_matmul_int(A, B))
        assert np.array_equal(oracle.naive_mt(A, B, 4), _exact_matmul_int(A, B))


def test_naive_mt_same_bits_as_naive():
    rng = np.random.default_rng(4)
    A, B = rng.uniform(-1, 1, (37, 53)), rng.uniform(-1, 1, (53, 29))
    assert np.array_equal(oracle.naive(A, B), oracle.naive_mt(A, B, 3))


# --------------------------------------------------------------------------- recursive forms
SHAPES = [(8, 8, 8), (16, 16, 16), (12, 12, 12), (9, 9, 9), (13, 7, 11), (20, 6, 15), (33, 33, 33)]


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("mode", [oracle.PAD, oracle.PEEL])
def test_integers_bit_exact_all_depths(alg, mode):
    # all intermediates are integers far below 2^53, so every form, schedule,
    # depth and odd-size policy must reproduce the exact product bit for bit
    rng = np.random.default_rng(100 + alg * 3 + mode)
    for m, n, k in SHAPES:
        if alg == oracle.IN_PLACE and not (m == n == k):
            continue
        A, B = _ints(rng, (m, k)), _ints(rng, (k, n))
        ex = _exact_matmul_int(A, B)
        for cutoff in (1, 2, 3, 5, 100):
            C = oracle.recursive(alg, A, B, cutoff, mode)
            assert np.array_equal(C, ex), (alg, mode, m, n, k, cutoff)


@pytest.mark.parametrize("alg", ALGS)
def test_identity_and_permutation_exact(alg):
    rng = np.random.default_rng(7)
    for n in (1, 2, 4, 5, 8, 16, 17):
        B = _ints(rng, (n, n))
        I = np.eye(n)
        P = np.eye(n)[rng.permutation(n)]
        for cutoff in (1, 2, 4):
            assert np.array_equal(oracle.recursive(alg, I, B, cutoff), B)
            assert np.array_equal(oracle.recursive(alg, P, B, cutoff), P.astype(int) @ B)
            assert np.array_equal(oracle.recursive(alg, B, I, cutoff), B)


@pytest.mark.parametrize("alg", ALGS)
def test_float_against_exact_tiny(alg):
    # brute force: exact rational product of the FP64 inputs, tiny sizes, all depths
    rng = np.random.default_rng(50 + alg)
    for n in (2, 3, 4, 6, 8):
        A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
        ex = [[sum(Fraction(A[i, p]) * Fraction(B[p, j]) for p in range(n)) for j in range(n)]
              for i in range(n)]
        for cutoff in (1, 2):
            C = oracle.recursive(alg, A, B, cutoff)
            err = max(abs(float(Fraction(C[i, j]) - ex[i][j])) for i in range(n) for j in range(n))
            # 4^L growth of the operand sums times a dot-product bound, generous constant
            assert err <= 1e3 * n * U


@pytest.mark.parametrize("alg", ALGS)
def test_float_close_to_naive_moderate(alg):
    rng = np.random.default_rng(60 + alg)
    n = 96
    A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
    R = oracle.naive(A, B)
    C = oracle.recursive(alg, A, B, cutoff=8)   # L = 4
    assert oracle.err_norm(C, R, A, B) <= 1e-14


def test_freivalds_identity():
    # C x = A (B x) for a random x; independent of how C was formed
    rng = np.random.default_rng(8)
    m, k, n = 150, 130, 170
    A, B = rng.uniform(-1, 1, (m, k)), rng.uniform(-1, 1, (k, n))
    for alg in (oracle.STRASSEN, oracle.WINOGRAD, oracle.TWO_TEMP):
        for mode in (oracle.PAD, oracle.PEEL):
            C = oracle.recursive(alg, A, B, 16, mode)
            x = rng.uniform(-1, 1, n)
            lhs, rhs = C @ x, A @ (B @ x)
            assert np.max(np.abs(lhs - rhs)) <= 1e-11 * np.max(np.abs(rhs))


def test_in_place_leaves_caller_arrays_alone_and_rejects_rectangles():
    rng = np.random.default_rng(9)
    A, B = _ints(rng, (16, 16)), _ints(rng, (16, 16))
    A0, B0 = A.copy(), B.copy()
    oracle.recursive(oracle.IN_PLACE, A, B, 2)
    assert np.array_equal(A, A0) and np.array_equal(B, B0)
    with pytest.raises(ValueError):
        oracle.recursive(oracle.IN_PLACE, _ints(rng, (8, 4)), _ints(rng, (4, 8)), 2)


# --------------------------------------------------------------------------- schedules (Tables 2, 3)
@pytest.mark.parametrize("which", [0, 1])
def test_tables_traces_match_bdpz(which):
    # every intermediate the schedule produces equals the BDPZ value of the same name
    rng = np.random.default_rng(12)
    A, B = _ints(rng, (2, 2)), _ints(rng, (2, 2))
    _, tw = oracle.recursive(oracle.WINOGRAD, A, B, 1, trace=True)
    _, ts = oracle.recursive(oracle.TWO_TEMP if which == 0 else oracle.IN_PLACE, A, B, 1, trace=True)
    assert np.array_equal(tw[8:30], ts[8:30])


def test_real_tables_pass_the_shadow():
    rng = np.random.default_rng(13)
    A, B = _ints(rng, (16, 16)), _ints(rng, (16, 16))
    assert np.array_equal(oracle.run_table(oracle.schedule_table(1), A, B, 2), _exact_matmul_int(A, B))
    # Table 2 under its own rules (X and Y temporaries), square and rectangular
    for m, n, k in ((16, 16, 16), (16, 8, 32), (8, 32, 16)):
        A, B = _ints(rng, (m, k)), _ints(rng, (k, n))
        assert np.array_equal(oracle.run_table(oracle.schedule_table(0), A, B, 2, two_temp=True),
                              _exact_matmul_int(A, B))


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(14)
    A, B = _ints(rng, (8, 8)), _ints(rng, (8, 8))
    ex = _exact_matmul_int(A, B)
    base = oracle.schedule_table(1)
    caught = 0
    # (a) swap two adjacent steps: a value is read before it is made or after it died
    for i in range(21):
        tab = base.copy()
        tab[[i, i + 1]] = tab[[i + 1, i]]
        try:
            C = oracle.run_table(tab, A, B, 2)
            if not np.array_equal(C, ex):
                caught += 1
        except RuntimeError:
            caught += 1
    assert caught >= 15
    # (b) store step 2's S1 over A22 instead of A21: A22 is still needed by P4
    tab = base.copy()
    tab[1, 2] = 3
    with pytest.raises(RuntimeError):
        oracle.run_table(tab, A, B, 2)
    # (c) flip the sign of U6 = U3 - P4
    tab = base.copy()
    tab[18, 0] = 0
    assert not np.array_equal(oracle.run_table(tab, A, B, 2), ex)


def test_planted_mistakes_in_table2_are_caught():
    # Table 2 (Sec. 3.3) with X and Y: the shadow (or the exact product) catches a reordered step,
    # X or Y overwritten while a value in it is still live, and a flipped sign
    rng = np.random.default_rng(16)
    A, B = _ints(rng, (8, 16)), _ints(rng, (16, 8))
    ex = _exact_matmul_int(A, B)
    base = oracle.schedule_table(0)
    run = lambda t: oracle.run_table(t, A, B, 2, two_temp=True)
    caught = 0
    for i in range(21):  # (a) swap two adjacent steps
        tab = base.copy()
        tab[[i, i + 1]] = tab[[i + 1, i]]
        try:
            if not np.array_equal(run(tab), ex):
                caught += 1
        except RuntimeError:
            caught += 1
    assert caught >= 15
    # (b) S4 = A12 - S2 computed before P6 = S2 T2 reads S2: X is overwritten while S2 is live
    tab = base.copy()
    tab[[8, 9]] = tab[[9, 8]]
    with pytest.raises(RuntimeError):
        run(tab)
    # (c) P1 stored in Y instead of X: T2 in Y is still needed by T4 = T2 - B21
    tab = base.copy()
    assert tab[11, 1] == 16 and tab[11, 2] == 12  # step 12: P1 -> X
    tab[11, 2] = 13
    with pytest.raises(RuntimeError):
        run(tab)
    # (d) the sign of U6 = U3 - P4 flipped
    tab = base.copy()
    assert tab[19, 1] == 28 and tab[19, 0] == 1
    tab[19, 0] = 0
    assert not np.array_equal(run(tab), ex)


# --------------------------------------------------------------------------- top-level product subsets
# C's coefficient of each top-level product, read off the paper's combinations:
# Strassen (Sec. 2.2) C11 = P1+P4-P5+P7, C12 = P3+P5, C21 = P2+P4, C22 = P1+P3-P2+P6;
# BDPZ (Sec. 2.3) C11 = U1 = P1+P2, C12 = U5 = P1+P6+P5+P3, C21 = U6 = P1+P6+P7-P4,
# C22 = U7 = P1+P6+P7+P5.  Rows: products P1..P7; columns: C11, C12, C21, C22.
_COEF = {
    oracle.STRASSEN: [[1, 0, 0, 1], [0, 0, 1, -1], [0, 1, 0, 1], [1, 0, 1, 0], [-1, 1, 0, 0], [0, 0, 0, 1],
                      [1, 0, 0, 0]],
    oracle.WINOGRAD: [[1, 1, 1, 1], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, -1, 0], [0, 1, 0, 1], [0, 1, 1, 1],
                      [0, 0, 1, 1]],
}


def test_single_top_products_on_the_worked_2x2():
    g = _golden()
    A = np.array(g["A"], float).reshape(2, 2)
    B = np.array(g["B"], float).reshape(2, 2)
    for alg, key in ((oracle.STRASSEN, "strassen_P"), (oracle.WINOGRAD, "bdpz_P")):
        for i, P in enumerate(g[key]):
            C = oracle.recursive_products(alg, A, B, 1, 1 << i)
            want = np.array(_COEF[alg][i], float).reshape(2, 2) * P
            assert np.array_equal(C, want), (alg, i)


@pytest.mark.parametrize("alg", [oracle.STRASSEN, oracle.WINOGRAD, oracle.KNUTH])
@pytest.mark.parametrize("m,n,k,cutoff", [(16, 16, 16, 8), (16, 16, 16, 2), (13, 10, 7, 3), (24, 8, 40, 4)])
def test_product_subsets_partition_the_product(alg, m, n, k, cutoff):
    # masks that partition the seven top-level products add up to the exact product, and a union
    # of disjoint masks is the sum of their results (integers: exact)
    rng = np.random.default_rng(17)
    A, B = _ints(rng, (m, k)), _ints(rng, (k, n))
    ex = _exact_matmul_int(A, B)
    assert np.array_equal(oracle.recursive_products(alg, A, B, cutoff, 0x7F), oracle.recursive(alg, A, B, cutoff))
    assert not np.any(oracle.recursive_products(alg, A, B, cutoff, 0))
    for parts in ([0x7F], [0x0F, 0x70], [0x03, 0x1C, 0x60], [1 << i for i in range(7)]):
        tot = sum(oracle.recursive_products(alg, A, B, cutoff, msk) for msk in parts)
        assert np.array_equal(tot, ex), (alg, parts)
    a = oracle.recursive_products(alg, A, B, cutoff, 0x05)
    b = oracle.recursive_products(alg, A, B, cutoff, 0x48)
    assert np.array_equal(a + b, oracle.recursive_products(alg, A, B, cutoff, 0x4D))
    with pytest.raises(ValueError):  # depth 0 has no top-level products
        oracle.recursive_products(alg, A, B, 10 ** 6, 0x7F)


# --------------------------------------------------------------------------- cutoff (Sec. 3.4)
def test_cutoff_model_closed_form():
    # lhs <= rhs  <=>  mkn <= 4(mk + kn + mn); for m = n = k tight at n = 12
    rng = np.random.default_rng(15)
    for _ in range(500):
        m, k, n = (2 * int(v) for v in rng.integers(1, 40, 3))
        lhs, rhs = oracle.cutoff_model(m, k, n)
        assert (lhs <= rhs) == (m * k * n <= 4 * (m * k + k * n + m * n))
    for n in range(2, 40, 2):
        lhs, rhs = oracle.cutoff_model(n, n, n)
        assert (lhs <= rhs) == (n <= 12)
    lhs, rhs = oracle.cutoff_model(12, 12, 12)
    assert lhs == rhs


def test_depth_rule():
    assert oracle.depth(256, 256, 256, 32) == 3       # 256 -> 128 -> 64 -> 32
    assert oracle.depth(16, 16, 16, 12) == 1           # Sec. 3.4: n <= 12 goes naive
    assert oracle.depth(12, 12, 12, 12) == 0
    assert oracle.depth(2, 2, 2, 1) == 1
    assert oracle.depth(8192, 8192, 8192, 1024) == 3
    assert oracle.depth(100, 300, 3000, 32) == 2       # the smallest dimension decides
    assert oracle.depth(33, 33, 33, 32) == 1


def test_workspace_accounting():
    # FP32 bytes at n = 16384: allocating Alg. 3 with 15 temporaries per level, and
    # Table 2's X, Y per level
    n = 16384
    gb = lambda e: e * 4 / 1e9
    assert [round(gb(oracle.workspace_elems(0, n, n, n, L)), 2) for L in (1, 2, 3)] == [4.03, 5.03, 5.28]
    assert [round(gb(oracle.workspace_elems(1, n, n, n, L)), 2) for L in (1, 2, 3)] == [0.54, 0.67, 0.7]
    assert oracle.workspace_elems(1, n, n, n, 20) <= (2 / 3) * n * n


def test_err_norm():
    A = np.array([[2.0, -4.0]])
    B = np.array([[1.0], [0.5]])
    C = np.array([[0.25]])
    R = np.array([[0.0]])
    assert oracle.err_norm(C, R, A, B) == 0.25 / (2 * 4.0 * 1.0)
