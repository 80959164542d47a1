"""GPU parity: every path of libswmm against the FP64 CPU oracle.

Bars (the normalised error is max|C - C_ref| / (k max|A| max|B|)):
  * integer-valued inputs: bit-exact, on sizes where every partial sum the GPU forms is an
    integer below 2^24 (FP32) -- the bound is computed from the depth and value range;
  * float inputs: the bounds of tests/bounds.py, derived from each leaf kind's arithmetic (TF32
    truncation, the compensated splits and the FP32 accumulator, FP64 rounding) with the RMS of
    the product terms, the per-level growth of the worst C quadrant (9 for the Winograd forms,
    6 for Strassen) and the tail factor of the number of compared elements; FP64 results also
    meet the 1e-13 bound, split-BF16 results the 2e-6 bound of FP32-equivalent paths.  Every
    float test also checks the error is far below that of an all-zero result, so a dropped
    product cannot hide under the bound.
With SWMM_ERRLOG set, every float comparison appends "test err tol" to that file.
"""
import ctypes
import os

import numpy as np
import pytest

import bounds
import oracle
from paper_2309_00628_gb300 import inputs, swmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W, S, K = swmm.SW_ALGO_WINOGRAD, swmm.SW_ALGO_STRASSEN, swmm.SW_ALGO_WINOGRAD_KNUTH
FUSED, TWO, INPL, ALLOC = swmm.SW_SCHED_FUSED, swmm.SW_SCHED_TWO_TEMP, swmm.SW_SCHED_IN_PLACE, swmm.SW_SCHED_ALLOC
WT = swmm.SW_LEAF_F64_WTILE


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    hd = swmm.sw_create(0)
    yield hd
    swmm.sw_destroy(hd)


ALGO_NAME = {swmm.SW_ALGO_NAIVE: "naive", W: "winograd", K: "knuth", S: "strassen"}


def _algo(variant):
    return ALGO_NAME[variant & 0xF]


def tol_tf32(C, A, B, L, variant=W):
    return bounds.tol_tf32(np.size(C), A.shape[1], L, A, B, _algo(variant))


def tol_bf16x3(C, A, B, L, variant=W):
    return bounds.tol_bf16x3(np.size(C), A.shape[1], L, A, B, _algo(variant))


def tol_tf32x3(C, A, B, L, variant=W):
    return bounds.tol_tf32x3(np.size(C), A.shape[1], L, A, B, _algo(variant))


def tol_fp64(C, A, B, L, variant=W):
    return bounds.tol_fp64(np.size(C), A.shape[1], L, A, B, _algo(variant))


def check_close(C, R, A, B, tol):
    """Normalised error within tol, and far below the error of returning zeros."""
    err = oracle.err_norm(C, R, A, B)
    zero = oracle.err_norm(np.zeros_like(R), R, A, B)
    log = os.environ.get("SWMM_ERRLOG")
    if log:
        with open(log, "a") as f:
            f.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]} {err:.3e} {tol:.3e}\n")
    assert err <= tol, (err, tol)
    assert err <= 0.3 * zero, (err, zero)
    return err


def run(h, A, B, cutoff, variant, dtype=np.float32, lda_pad=0, clobber_ok=False):
    """C = A B through sw_smm / sw_dmm on device copies of A, B; returns numpy C."""
    m, k = A.shape
    n = B.shape[1]
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    dA = torch.zeros((m, k + lda_pad), dtype=tdt, device="cuda")
    dA[:, :k] = torch.from_numpy(A.astype(dtype))
    dB = torch.from_numpy(B.astype(dtype)).cuda()
    dC = torch.full((m, n), float("nan"), dtype=tdt, device="cuda")
    fn = swmm.sw_smm if dtype == np.float32 else swmm.sw_dmm
    st = fn(h, ctypes.c_void_p(dA.data_ptr()), k + lda_pad, ctypes.c_void_p(dB.data_ptr()), max(n, 1),
            ctypes.c_void_p(dC.data_ptr()), max(n, 1), m, n, k, cutoff, variant, None)
    swmm.check(h, st)
    swmm.check(h, swmm.sw_sync(h, None))
    return dC.cpu().numpy().astype(np.float64)


def depth(h, m, n, k, cutoff, variant, eb):
    st, d = swmm.sw_mm_depth(m, n, k, cutoff, variant, eb)
    assert st == swmm.SW_OK
    return d


def exact_int_safe(lim, k, L, growth=4):
    # worst case |partial sum| of an integer product at depth L: operand sums grow <= growth^L,
    # a leaf sums ceil(k/2^L) nonzero products (padding adds zeros), and a C block receives up
    # to 4^L leaf results
    s = lim * growth ** L
    return s * s * -(-k // 2 ** L) * 4 ** L < 2 ** 24


# ------------------------------------------------------------------ plain product (Alg. 1)
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (128, 256, 32), (300, 500, 200), (129, 257, 33), (1000, 1000, 1000),
                                   (64, 2000, 7), (5, 3, 4000)])
def test_plain_tf32_integers_bit_exact(h, m, n, k):
    A, B = inputs.pair(m, n, k, "int", seed=0, dtype=np.float64)
    C = run(h, A, B, 0, swmm.SW_ALGO_NAIVE)
    assert np.array_equal(C, oracle.naive(A, B))


def test_plain_tf32_float_within_bound_and_deterministic(h):
    m, n, k = 777, 640, 1500
    A, B = inputs.pair(m, n, k, "uniform", seed=3, dtype=np.float32)
    C1 = run(h, A, B, 0, swmm.SW_ALGO_NAIVE)
    C2 = run(h, A, B, 0, swmm.SW_ALGO_NAIVE)
    assert np.array_equal(C1, C2)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    err = check_close(C1, R, A, B, tol_tf32(C1, A, B, 0, swmm.SW_ALGO_NAIVE))
    assert err > 0  # the tensor core really ran at TF32, not FP32


def test_plain_unaligned_leading_dimension(h):
    m, n, k = 70, 90, 61
    A, B = inputs.pair(m, n, k, "int", seed=4, dtype=np.float64)
    C = run(h, A, B, 0, swmm.SW_ALGO_NAIVE, lda_pad=3)
    assert np.array_equal(C, oracle.naive(A, B))


def test_degenerate_sizes(h):
    for m, n, k in [(0, 5, 5), (5, 0, 5), (3, 4, 0)]:
        A, B = np.ones((m, k)), np.ones((k, n))
        for v in (swmm.SW_ALGO_NAIVE, W | FUSED, W | TWO):
            if m == 0 or n == 0:
                continue
            C = run(h, A, B, 1, v)
            assert np.array_equal(C, np.zeros((m, n)))


# ------------------------------------------------------------------ FUSED recursion
@pytest.mark.parametrize("algo", [W, S, K])
@pytest.mark.parametrize("m,n,k,cutoff", [(256, 256, 256, 128), (256, 256, 256, 64), (384, 384, 384, 32),
                                          (300, 260, 200, 64), (97, 131, 203, 40), (512, 128, 1024, 32),
                                          (1024, 1024, 1024, 256)])
def test_fused_integers_bit_exact(h, algo, m, n, k, cutoff):
    v = algo | FUSED
    L = depth(h, m, n, k, cutoff, v, 4)
    assert L >= 1
    lim = 1 if L >= 2 else 4
    assert exact_int_safe(lim, k, L)
    A, B = inputs.pair(m, n, k, "int", seed=L, dtype=np.float64, lim=lim)
    C = run(h, A, B, cutoff, v)
    assert np.array_equal(C, oracle.naive(A, B)), (algo, L)


@pytest.mark.parametrize("algo", [W, S, K])
@pytest.mark.parametrize("L", [1, 2, 3])
def test_fused_float_within_bound(h, algo, L):
    n = 1024
    A, B = inputs.pair(n, n, n, "uniform", seed=10 + L, dtype=np.float32)
    R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
    C = run(h, A, B, n >> L, algo | FUSED)
    assert depth(h, n, n, n, n >> L, algo | FUSED, 4) == L
    check_close(C, R, A, B, tol_tf32(C, A, B, L, algo))


# ------------------------------------------------------------------ materialised schedules
@pytest.mark.parametrize("sched", [TWO, INPL, ALLOC])
@pytest.mark.parametrize("n,cutoff", [(256, 128), (256, 64), (512, 128), (384, 48)])
def test_schedules_integers_bit_exact(h, sched, n, cutoff):
    v = W | sched
    L = depth(h, n, n, n, cutoff, v, 4)
    lim = 1 if L >= 2 else 4
    assert exact_int_safe(lim, n, L)
    A, B = inputs.pair(n, n, n, "int", seed=20 + L, dtype=np.float64, lim=lim)
    C = run(h, A, B, cutoff, v)
    assert np.array_equal(C, oracle.naive(A, B)), (sched, L)


def test_strassen_alloc_integers_bit_exact(h):
    n = 512
    A, B = inputs.pair(n, n, n, "int", seed=30, dtype=np.float64, lim=1)
    C = run(h, A, B, 64, S | ALLOC)
    assert np.array_equal(C, oracle.naive(A, B))


@pytest.mark.parametrize("odd", [swmm.SW_PAD, swmm.SW_PEEL])
@pytest.mark.parametrize("sched", [TWO, ALLOC, INPL])
def test_schedules_odd_sizes(h, odd, sched):
    shapes = [(300, 300, 300)] if sched == INPL else [(300, 260, 200), (97, 131, 203), (260, 100, 300)]
    for m, n, k in shapes:
        A, B = inputs.pair(m, n, k, "int", seed=40, dtype=np.float64, lim=2)
        C = run(h, A, B, 40, W | sched | odd)
        assert np.array_equal(C, oracle.naive(A, B)), (m, n, k, sched, odd)


def test_schedules_float_within_bound(h):
    n = 512
    A, B = inputs.pair(n, n, n, "uniform", seed=50, dtype=np.float32)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    for sched in (TWO, INPL, ALLOC):
        C = run(h, A, B, 64, W | sched)
        L = depth(h, n, n, n, 64, W | sched, 4)
        check_close(C, R, A, B, tol_tf32(C, A, B, L))


# ------------------------------------------------------------------ FP64 path (n = 256, cutoff 32, L = 3)
CONFIG1 = [(swmm.SW_ALGO_NAIVE, FUSED), (S, FUSED), (S, ALLOC), (W, FUSED), (W, TWO), (W, INPL), (W, ALLOC),
           (K, FUSED)]


@pytest.mark.parametrize("algo,sched", CONFIG1)
def test_fp64_n256_cutoff32(h, algo, sched):
    n = 256
    v = algo | sched
    if algo != swmm.SW_ALGO_NAIVE:
        assert depth(h, n, n, n, 32, v, 8) == 3
    Ai, Bi = inputs.pair(n, n, n, "int", seed=0, dtype=np.float64)
    assert np.array_equal(run(h, Ai, Bi, 32, v, dtype=np.float64), oracle.naive(Ai, Bi))
    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float64)
    C = run(h, A, B, 32, v, dtype=np.float64)
    check_close(C, oracle.naive(A, B), A, B, tol_fp64(C, A, B, 0 if algo == swmm.SW_ALGO_NAIVE else 3, v))


@pytest.mark.parametrize("odd", [swmm.SW_PAD, swmm.SW_PEEL])
def test_fp64_odd_sizes(h, odd):
    for m, n, k in [(255, 257, 129), (33, 65, 17)]:
        A, B = inputs.pair(m, n, k, "uniform", seed=1, dtype=np.float64)
        R = oracle.naive(A, B)
        for v in (W | FUSED, W | TWO, S | ALLOC):
            C = run(h, A, B, 16, v | odd, dtype=np.float64)
            check_close(C, R, A, B, tol_fp64(C, A, B, depth(h, m, n, k, 16, v | odd, 8), v))


@pytest.mark.parametrize("algo", [W, S])
@pytest.mark.parametrize("m,n,k,cutoff,L", [(2048, 2048, 2048, 16, 4), (2048, 2080, 2064, 40, 4), (2050, 2048, 2052, 40, 4)])
def test_fp64_fused_deeper_than_three(h, algo, m, n, k, cutoff, L):
    # FP64 FUSED past three levels: Table 2 (BDPZ) / Alg. 2 (Strassen) steps above a fused
    # three-level bottom; with and without the tile-step leaf
    for leaf in ((0, WT) if algo == W else (0,)):
        v = algo | FUSED | leaf
        assert depth(h, m, n, k, cutoff, v, 8) == L
        Ai, Bi = inputs.pair(m, n, k, "int", seed=8, dtype=np.float64)
        assert np.array_equal(run(h, Ai, Bi, cutoff, v, dtype=np.float64), oracle.naive_mt(Ai, Bi)), v
        A, B = inputs.pair(m, n, k, "uniform", seed=9, dtype=np.float64)
        C = run(h, A, B, cutoff, v, dtype=np.float64)
        check_close(C, oracle.naive_mt(A, B), A, B, tol_fp64(C, A, B, L + (1 if leaf else 0), v))


# ------------------------------------------------------------------ FP64 leaves with a Winograd step per tile


@pytest.mark.parametrize("algo,sched", [(W, FUSED), (W, TWO), (W, INPL), (W, ALLOC), (K, FUSED)])
def test_fp64_wtile_n256_cutoff32(h, algo, sched):
    # every 64 x 64 leaf tile takes one more Winograd step, its operand sums in shared memory
    n = 256
    v = algo | sched | WT
    assert depth(h, n, n, n, 32, v, 8) == 3
    Ai, Bi = inputs.pair(n, n, n, "int", seed=0, dtype=np.float64)
    assert np.array_equal(run(h, Ai, Bi, 32, v, dtype=np.float64), oracle.naive(Ai, Bi))
    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float64)
    C = run(h, A, B, 32, v, dtype=np.float64)
    check_close(C, oracle.naive(A, B), A, B, tol_fp64(C, A, B, 3 + 1, v))  # + the in-tile step


@pytest.mark.parametrize("cutoff", [1 << 20, 40])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 16), (63, 65, 17), (300, 260, 100), (129, 257, 33),
                                   (5, 3, 4000), (1000, 1000, 1000)])
def test_fp64_wtile_shapes(h, m, n, k, cutoff):
    # depth 0 (one leaf) and deeper; ragged tiles and blocks, k not a multiple of the 16-deep block
    Ai, Bi = inputs.pair(m, n, k, "int", seed=5, dtype=np.float64)
    Ri = oracle.naive(Ai, Bi)
    A, B = inputs.pair(m, n, k, "uniform", seed=6, dtype=np.float64)
    R = oracle.naive(A, B)
    for v in (W | FUSED | WT, W | TWO | WT | swmm.SW_PEEL, K | FUSED | WT):
        assert np.array_equal(run(h, Ai, Bi, cutoff, v, dtype=np.float64), Ri), (m, n, k, cutoff, v)
        C = run(h, A, B, cutoff, v, dtype=np.float64)
        check_close(C, R, A, B, tol_fp64(C, A, B, depth(h, m, n, k, cutoff, v, 8) + 1, v))


def test_fp64_wtile_is_its_own_leaf(h):
    # the tile step rounds differently from the plain leaf (so the Winograd-step kernel ran), and
    # both sit well inside the FP64 bound
    m, n, k = 300, 260, 100
    A, B = inputs.pair(m, n, k, "uniform", seed=7, dtype=np.float64)
    R = oracle.naive(A, B)
    C0 = run(h, A, B, 1 << 20, W | FUSED, dtype=np.float64)
    C1 = run(h, A, B, 1 << 20, W | FUSED | WT, dtype=np.float64)
    assert not np.array_equal(C0, C1)
    check_close(C0, R, A, B, tol_fp64(C0, A, B, 0))
    check_close(C1, R, A, B, tol_fp64(C1, A, B, 1))


# ------------------------------------------------------------------ host entry point, norms, errors
def test_host_entry_point_matches_device_path(h):
    m, n, k = 500, 300, 700
    A, B = inputs.pair(m, n, k, "uniform", seed=60, dtype=np.float32)
    C = np.zeros((m, n), np.float32)
    st = swmm.sw_smm_host(h, A.ctypes.data_as(ctypes.c_void_p), k, B.ctypes.data_as(ctypes.c_void_p), n,
                          C.ctypes.data_as(ctypes.c_void_p), n, m, n, k, 256, W | FUSED, None)
    swmm.check(h, st)
    Cd = run(h, A, B, 256, W | FUSED)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    check_close(C.astype(np.float64), R, A, B, tol_tf32(C, A, B, 1))
    assert np.max(np.abs(C - Cd)) <= 1e-3


@pytest.mark.parametrize("algo", [W, K, swmm.SW_ALGO_NAIVE])
def test_host_entry_point_row_panels(h, algo):
    # a large host-operand product moves A and C in row panels (copies overlap the panel
    # products); each panel runs at the whole product's depth, the last panel lower
    m, n, k, cutoff = 4500, 2000, 1500, 400
    v = algo | FUSED
    L = depth(h, m, n, k, cutoff, v, 4)
    assert L == (0 if algo == swmm.SW_ALGO_NAIVE else 2)
    assert exact_int_safe(2, k, L)
    for kind in ("int", "uniform"):
        A, B = inputs.pair(m, n, k, kind, seed=62, dtype=np.float32, **({"lim": 2} if kind == "int" else {}))
        hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
        hC = torch.full((m, n), float("nan")).pin_memory()
        st = swmm.sw_smm_host(h, ctypes.c_void_p(hA.data_ptr()), k, ctypes.c_void_p(hB.data_ptr()), n,
                              ctypes.c_void_p(hC.data_ptr()), n, m, n, k, cutoff, v, None)
        swmm.check(h, st)
        C = hC.numpy().astype(np.float64)
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        if kind == "int":
            assert np.array_equal(C, R)
        else:
            check_close(C, R, A, B, tol_tf32(C, A, B, L, algo))


def test_error_norms_match_numpy(h):
    m, n, k = 300, 200, 100
    A, B = inputs.pair(m, n, k, "uniform", seed=61, dtype=np.float32)
    C = (A.astype(np.float64) @ B.astype(np.float64)).astype(np.float32)
    R = A.astype(np.float64) @ B.astype(np.float64) + 1e-3
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    dR = torch.from_numpy(R).cuda()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st, out = swmm.sw_error_norms(h, 4, m, n, k, p(dA), k, p(dB), n, p(dC), n, p(dR), n, None)
    swmm.check(h, st)
    assert out[0] == pytest.approx(np.max(np.abs(C - R)), rel=1e-12)
    assert out[1] == np.max(np.abs(A)) and out[2] == np.max(np.abs(B))


def test_argument_errors(h):
    lib = swmm.load()
    assert lib.sw_smm(h, None, 4, None, 4, None, 4, 4, 4, 4, 1, 0, None) == swmm.SW_EINVAL
    d = torch.zeros(64, device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    assert lib.sw_smm(h, p, 2, p, 4, p, 4, 4, 4, 4, 1, 0, None) == swmm.SW_EINVAL
    assert lib.sw_smm(h, p, 8, p, 4, p, 4, 4, 4, 8, 1, W | INPL, None) == swmm.SW_EUNSUPPORTED
    assert "m == n == k" in swmm.sw_last_error(h)
    assert swmm.sw_sync(h, None) == swmm.SW_OK


# ------------------------------------------------------------------ full size (n = 8192), sampled rows
@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_full_size_sampled_rows(h, L):
    n = 8192
    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float32)
    v = swmm.SW_ALGO_NAIVE if L == 0 else W | FUSED
    cutoff = n >> L if L else 0
    if L:
        assert depth(h, n, n, n, cutoff, v, 4) == L
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = swmm.mm(h, dA, dB, cutoff, v, sync=True)
    rows = np.random.Generator(np.random.PCG64(99)).choice(n, 8, replace=False)
    R = oracle.naive_mt(A[rows].astype(np.float64), B.astype(np.float64))
    Cr = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    check_close(Cr, R, A, B, tol_tf32(Cr, A, B, L, v))


@pytest.mark.parametrize("algo,L,leaf", [(S, 1, "tf32"), (S, 2, "tf32"), (K, 1, "tf32"), (K, 2, "tf32"),
                                         (W, 1, "bf16x3")])
def test_full_size_variants_sampled_rows(h, algo, L, leaf):
    # the bench's other n = 8192 rows: Strassen and Knuth-form Winograd FUSED with TF32 leaves, and
    # Winograd L1 with split-BF16 leaves, on the headline's operands
    n = 8192
    A, B = inputs.pair(n, n, n, "uniform", seed=0, dtype=np.float32)
    v = algo | FUSED | (swmm.SW_LEAF_BF16X3 if leaf == "bf16x3" else 0)
    cutoff = n >> L
    assert depth(h, n, n, n, cutoff, v, 4) == L
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = swmm.mm(h, dA, dB, cutoff, v, sync=True)
    rows = np.random.Generator(np.random.PCG64(97)).choice(n, 8, replace=False)
    R = oracle.naive_mt(A[rows].astype(np.float64), B.astype(np.float64))
    Cr = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    tol = tol_bf16x3(Cr, A, B, L, v) if leaf == "bf16x3" else tol_tf32(Cr, A, B, L, v)
    check_close(Cr, R, A, B, tol)
    del dA, dB, C


@pytest.mark.parametrize("sched", [TWO, FUSED])
def test_bf16x3_n16384_normal_depth1_sampled_rows(h, sched):
    # config 3's other rows: split-BF16 leaves at n = 16384 on N(0, 1) operands, one level, with
    # the Table 2 schedule and with the fused one; the FP32-accuracy bound 2e-6 holds
    n, cutoff = 16384, 8192
    v = W | sched | swmm.SW_LEAF_BF16X3
    assert depth(h, n, n, n, cutoff, v, 4) == 1
    A, B = inputs.pair(n, n, n, "normal", seed=0, dtype=np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = swmm.mm(h, dA, dB, cutoff, v, sync=True)
    rows = np.random.Generator(np.random.PCG64(96)).choice(n, 6, replace=False)
    R = oracle.naive_mt(A[rows].astype(np.float64), B.astype(np.float64))
    Cr = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    check_close(Cr, R, A, B, min(2e-6, tol_bf16x3(Cr, A, B, 1)))
    del dA, dB, C


# ------------------------------------------------------------------ split-BF16 leaves (hi*hi + hi*lo + lo*hi)
# hi = bf16(x), lo = bf16(x - hi) carry x to a relative 2^-16, and the dropped lo*lo term is below
# 2^-16 |a b|: each product term errs by < 3 * 2^-16 |a||b|, so the same Hoeffding argument as
# for TF32 gives 8 * 3 * 2^-16 * 3^L / sqrt(k) (normalised), 40x tighter than TF32.
BF = swmm.SW_LEAF_BF16X3


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 500, 200), (1000, 1000, 1000), (129, 257, 33)])
def test_bf16x3_plain_integers_bit_exact(h, m, n, k):
    A, B = inputs.pair(m, n, k, "int", seed=70, dtype=np.float64)
    assert np.array_equal(run(h, A, B, 0, swmm.SW_ALGO_NAIVE | BF), oracle.naive(A, B))


def test_bf16x3_plain_float_far_tighter_than_tf32(h):
    m, n, k = 777, 640, 1500
    A, B = inputs.pair(m, n, k, "uniform", seed=71, dtype=np.float32)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    e_bf = check_close(run(h, A, B, 0, swmm.SW_ALGO_NAIVE | BF), R, A, B, tol_bf16x3(R, A, B, 0))
    e_tf = check_close(run(h, A, B, 0, swmm.SW_ALGO_NAIVE), R, A, B, tol_tf32(R, A, B, 0))
    assert e_bf < e_tf / 16, (e_bf, e_tf)


@pytest.mark.parametrize("algo,sched", [(W, FUSED), (W, TWO), (W, INPL), (W, ALLOC), (S, FUSED), (S, ALLOC)])
def test_bf16x3_recursive(h, algo, sched):
    # (Tables 2 and 3 are Winograd schedules: Strassen runs FUSED and allocating only)
    n, cutoff = 512, 128  # L = 2
    v = algo | sched | BF
    L = depth(h, n, n, n, cutoff, v, 4)
    assert L == 2
    Ai, Bi = inputs.pair(n, n, n, "int", seed=72, dtype=np.float64, lim=1)
    assert np.array_equal(run(h, Ai, Bi, cutoff, v), oracle.naive(Ai, Bi))
    A, B = inputs.pair(n, n, n, "uniform", seed=73, dtype=np.float32)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    # (at k = 512 and depth 2 the split leaves' own error, not the accumulator, dominates: the
    # normalised error exceeds the 2e-6 of the n = 16384 configuration, which the test below checks)
    check_close(run(h, A, B, cutoff, v), R, A, B, tol_bf16x3(R, A, B, L, algo))


def test_bf16x3_odd_sizes_fused_and_two_temp(h):
    for m, n, k in [(300, 260, 200), (97, 131, 203)]:
        A, B = inputs.pair(m, n, k, "int", seed=74, dtype=np.float64, lim=2)
        for v in (W | FUSED | BF, W | TWO | BF | swmm.SW_PAD, W | TWO | BF | swmm.SW_PEEL):
            assert np.array_equal(run(h, A, B, 40, v), oracle.naive(A, B)), (m, n, k, v)


def test_bf16x3_two_temp_n16384_normal_sampled_rows(h):
    # the split-BF16 low-allocation configuration: n = 16384, N(0,1), Table 2 schedule, depth 2
    n, cutoff = 16384, 4096
    v = W | TWO | BF
    assert depth(h, n, n, n, cutoff, v, 4) == 2
    st, ws = swmm.sw_mm_workspace_size(n, n, n, cutoff, v, 4)
    assert st == swmm.SW_OK
    A, B = inputs.pair(n, n, n, "normal", seed=0, dtype=np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = swmm.mm(h, dA, dB, cutoff, v, sync=True)
    rows = np.random.Generator(np.random.PCG64(98)).choice(n, 6, replace=False)
    R = oracle.naive_mt(A[rows].astype(np.float64), B.astype(np.float64))
    Cr = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    check_close(Cr, R, A, B, min(2e-6, tol_bf16x3(Cr, A, B, 2)))
    del dA, dB, C
    torch.cuda.empty_cache()


@pytest.mark.parametrize("sched", [TWO, INPL, ALLOC])
def test_ragged_leaf_widths_do_not_spill_into_neighbours(h, sched):
    # leaf widths that are not a multiple of 4 FP32 elements (here 18 and 10): each C quadrant must
    # only be written inside its own columns
    for n, cutoff in ((36, 18), (40, 16)):
        A, B = inputs.pair(n, n, n, "int", seed=75, dtype=np.float64, lim=2)
        C = run(h, A, B, cutoff, W | sched | BF)
        assert np.array_equal(C, oracle.naive(A, B)), (n, sched)


# ------------------------------------------------------------------ autotuner (cutoff <= 0)
def test_autotuned_depth_is_timed_exact_and_reused(h):
    # n = 4096: depths 0, 1, 2 keep TF32 leaves of >= 1024, so the first call times three plans;
    # integers in [-1, 1] keep every partial sum an exact integer at all three depths
    n = 4096
    assert exact_int_safe(1, n, 2)
    A, B = inputs.pair(n, n, n, "int", seed=5, dtype=np.float32, lim=1)
    R = A.astype(np.float64) @ B.astype(np.float64)  # integer sums below 2^53: exact in FP64
    v = W | FUSED
    C = run(h, A, B, 0, v)
    assert np.array_equal(C, R)
    st, t = swmm.sw_last_tuning(h)
    assert st == swmm.SW_OK
    assert t["candidates"] == 3 and t["cutoff"] in (4096, 2048, 1024) and t["ms"] > 0, t
    # the decision is kept: a second call plans nothing new and gives the same bits
    C2 = run(h, A, B, 0, v)
    assert np.array_equal(C2, R)
    st, t2 = swmm.sw_last_tuning(h)
    assert st == swmm.SW_OK and t2 == t


# ------------------------------------------------------------------ Knuth's form of Winograd
def test_knuth_and_bdpz_errors_agree_by_depth(h):
    # the same seven products with differently grouped operand sums: at every depth both forms
    # stay within the TF32 bound and within a factor 2 of each other
    n = 1024
    A, B = inputs.pair(n, n, n, "uniform", seed=60, dtype=np.float32)
    R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
    for L in (1, 2, 3):
        ew = check_close(run(h, A, B, n >> L, W | FUSED), R, A, B, tol_tf32(R, A, B, L, W))
        ek = check_close(run(h, A, B, n >> L, K | FUSED), R, A, B, tol_tf32(R, A, B, L, K))
        assert 0.5 <= ek / ew <= 2.0, (L, ek, ew)


def test_knuth_fp64_matches_oracle_knuth_recursion(h):
    # FP64, n = 256, cutoff 32 (depth 3): the GPU's Knuth form against the oracle's own Knuth
    # recursion (Sec. 2.3 as written) and the plain product
    n = 256
    A, B = inputs.pair(n, n, n, "uniform", seed=61, dtype=np.float64)
    C = run(h, A, B, 32, K | FUSED, dtype=np.float64)
    check_close(C, oracle.recursive(oracle.KNUTH, A, B, 32), A, B, tol_fp64(C, A, B, 3, K))
    check_close(C, oracle.naive(A, B), A, B, tol_fp64(C, A, B, 3, K))


def test_knuth_only_in_fused_schedule(h):
    A, B = inputs.pair(64, 64, 64, "int", seed=62, dtype=np.float32, lim=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty(64, 64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    for sched in (TWO, INPL, ALLOC):
        st = swmm.sw_smm(h, p(dA), 64, p(dB), 64, p(dC), 64, 64, 64, 64, 16, K | sched, None)
        assert st == swmm.SW_EUNSUPPORTED, sched


# ------------------------------------------------------------------ compensated TF32 leaves (3 TF32 products)
# hi = tf32(x) (nearest) leaves |x - hi| <= 2^-11 |x|; lo = x - hi is read by the tensor core as
# TF32 (10 mantissa bits), so hi + lo carries x to 2^-21 relative; the dropped lo*lo term is below
# 2^-22 |a b|.  Each product term errs by < 2^-19 |a||b|: the Hoeffding argument gives
# 8 * 2^-19 * 3^L / sqrt(k), plus the same FP32-accumulation floor 2^-20 as the split-BF16 bound.
X3 = swmm.SW_LEAF_TF32X3


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (300, 500, 200), (1000, 1000, 1000), (129, 257, 33)])
def test_tf32x3_plain_integers_bit_exact(h, m, n, k):
    A, B = inputs.pair(m, n, k, "int", seed=80, dtype=np.float64)
    assert np.array_equal(run(h, A, B, 0, swmm.SW_ALGO_NAIVE | X3), oracle.naive(A, B))


def test_tf32x3_plain_float_far_tighter_than_tf32(h):
    # both compensated forms end at the FP32-accumulation floor of the tensor core (the operand
    # split of TF32X3 is finer, but it issues two accumulator updates per 16-deep k-step where
    # split-BF16 issues one): within a factor 4 of each other, and 16x tighter than plain TF32
    m, n, k = 777, 640, 1500
    A, B = inputs.pair(m, n, k, "uniform", seed=81, dtype=np.float32)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    e_x3 = check_close(run(h, A, B, 0, swmm.SW_ALGO_NAIVE | X3), R, A, B, tol_tf32x3(R, A, B, 0))
    e_bf = check_close(run(h, A, B, 0, swmm.SW_ALGO_NAIVE | BF), R, A, B, tol_bf16x3(R, A, B, 0))
    e_tf = check_close(run(h, A, B, 0, swmm.SW_ALGO_NAIVE), R, A, B, tol_tf32(R, A, B, 0))
    assert e_x3 < e_tf / 16 and e_x3 < 4 * e_bf, (e_x3, e_bf, e_tf)


@pytest.mark.parametrize("algo,sched", [(W, FUSED), (W, TWO), (W, INPL), (W, ALLOC), (S, FUSED), (S, ALLOC),
                                        (K, FUSED)])
def test_tf32x3_recursive(h, algo, sched):
    n, cutoff = 512, 128  # L = 2
    v = algo | sched | X3
    L = depth(h, n, n, n, cutoff, v, 4)
    assert L == 2
    Ai, Bi = inputs.pair(n, n, n, "int", seed=82, dtype=np.float64, lim=1)
    assert np.array_equal(run(h, Ai, Bi, cutoff, v), oracle.naive(Ai, Bi))
    A, B = inputs.pair(n, n, n, "uniform", seed=83, dtype=np.float32)
    R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
    check_close(run(h, A, B, cutoff, v), R, A, B, tol_tf32x3(R, A, B, L, algo))


def test_tf32x3_odd_sizes(h):
    for m, n, k in [(300, 260, 200), (97, 131, 203)]:
        A, B = inputs.pair(m, n, k, "int", seed=84, dtype=np.float64, lim=2)
        for v in (W | FUSED | X3, W | TWO | X3 | swmm.SW_PAD, W | TWO | X3 | swmm.SW_PEEL):
            assert np.array_equal(run(h, A, B, 40, v), oracle.naive(A, B)), (m, n, k, v)


# ------------------------------------------------------------------ depth-1 accumulation chains
@pytest.mark.parametrize("leaf", [swmm.SW_LEAF_TF32, swmm.SW_LEAF_BF16X3])
@pytest.mark.parametrize("algo", [W, K])
@pytest.mark.parametrize("m,n,k", [(1024, 1024, 1024), (1000, 1500, 700), (2304, 520, 300), (3000, 2900, 2000),
                                   (600, 9000, 520)])
def test_fused_depth1_wide_quadrants_integers_bit_exact(h, leaf, algo, m, n, k):
    # depth-1 leaf launches with the products of a tile position summed in tensor memory (TF32:
    # CTA pairs, quadrants wider than 128 columns; split-BF16: single CTAs), stores before
    # reduce-adds; odd position counts leave unpaired chains and balanced per-unit sequences
    cutoff = min(m, n, k) - 1
    v = algo | FUSED | leaf
    assert depth(h, m, n, k, cutoff, v, 4) == 1
    assert exact_int_safe(4, k, 1)
    A, B = inputs.pair(m, n, k, "int", seed=90, dtype=np.float64, lim=4)
    assert np.array_equal(run(h, A, B, cutoff, v), oracle.naive(A, B)), (algo, m, n, k)


@pytest.mark.parametrize("leaf", [swmm.SW_LEAF_TF32, swmm.SW_LEAF_BF16X3])
def test_ordered_depth1_graph_replay_integers_bit_exact(h, leaf):
    # a depth-1 product whose C blocks take a store then reduce-adds (ordering counters) captured
    # once into a CUDA graph and replayed on new data in the same buffers: every replay orders its
    # adds after its own stores (the launch epoch lives on the device, not in the captured args)
    # (large enough that the product keeps its ordered stores: at least one store job per unit)
    m, n, k = 8192, 8192, 1024
    cutoff = 1000
    v = W | FUSED | leaf
    assert depth(h, m, n, k, cutoff, v, 4) == 1
    rows = np.sort(np.random.Generator(np.random.PCG64(94)).choice(m, 24, replace=False))
    dA = torch.zeros((m, k), dtype=torch.float32, device="cuda")
    dB = torch.zeros((k, n), dtype=torch.float32, device="cuda")
    dC = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    args = (ctypes.c_void_p(dA.data_ptr()), k, ctypes.c_void_p(dB.data_ptr()), n, ctypes.c_void_p(dC.data_ptr()), n,
            m, n, k, cutoff, v)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        # plan once outside the capture (the plan's upload is not capturable)
        swmm.check(h, swmm.sw_smm(h, *args, ctypes.c_void_p(side.cuda_stream)))
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = swmm.sw_smm(h, *args, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    swmm.check(h, st)
    for seed in (91, 92, 93):
        A, B = inputs.pair(m, n, k, "int", seed=seed, dtype=np.float64, lim=4)
        dA.copy_(torch.from_numpy(A.astype(np.float32)))
        dB.copy_(torch.from_numpy(B.astype(np.float32)))
        dC.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        swmm.check(h, swmm.sw_sync(h, None))
        got = dC[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        assert np.array_equal(got, oracle.naive_mt(A[rows], B)), seed
        assert not torch.isnan(dC).any()



@pytest.mark.parametrize("leaf", [swmm.SW_LEAF_TF32, swmm.SW_LEAF_BF16X3])
@pytest.mark.parametrize("algo", [W, K])
@pytest.mark.parametrize("m,n,k,ordered", [(8192, 8192, 1024, True), (8192, 8192, 8192, True),
                                           (2048, 2048, 2048, False), (1500, 1000, 700, False)])
def test_depth1_ordered_and_unordered_paths_integers_bit_exact(h, leaf, algo, m, n, k, ordered):
    # depth-1 products with enough first-writer jobs for every unit keep ordered stores and
    # accumulation chains (no zeroing of C); smaller ones zero C and reduce-add every product
    # (TF32 n = 8192, k = 1024: 256-wide tiles, two accumulators; k = 8192: 512-wide, one)
    cutoff = min(m, n, k) - 1
    v = algo | FUSED | leaf
    assert depth(h, m, n, k, cutoff, v, 4) == 1
    lim = 4 if k <= 4096 else 2
    assert exact_int_safe(lim, k, 1)
    A, B = inputs.pair(m, n, k, "int", seed=95, dtype=np.float64, lim=lim)
    dA, dB = torch.from_numpy(A.astype(np.float32)).cuda(), torch.from_numpy(B.astype(np.float32)).cuda()
    dC = torch.full((m, n), float("nan"), device="cuda")
    swmm.check(h, swmm.sw_profile(h, True))
    swmm.sw_profile_read(h)
    swmm.mm(h, dA, dB, cutoff, v, out=dC, sync=True)
    _, prof = swmm.sw_profile_read(h)
    swmm.check(h, swmm.sw_profile(h, False))
    assert (prof["memset"][0] == 0) == ordered, prof["memset"]
    rows = np.sort(np.random.Generator(np.random.PCG64(96)).choice(m, 16, replace=False))
    got = dC[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.array_equal(got, oracle.naive_mt(A[rows], B))
    assert not torch.isnan(dC).any()


@pytest.mark.parametrize("algo,cutoff", [(W, 23200), (swmm.SW_ALGO_NAIVE, 0)])
def test_max_size_past_2_31_elements_sampled_entries(h, algo, cutoff):
    # 46400 x 46400 operands hold 2.15e9 elements each, past 2^31: the operand-sum pass, the
    # tensor maps and the epilogue index them in 64 bits.  Integer inputs in [-2, 2] keep every
    # partial sum exact; sampled rows x sampled columns (first, last, block edges, random) of C
    # are compared bit-exactly with the oracle on the matching slices of A and B.
    n = 46400
    if torch.cuda.mem_get_info()[0] < 64e9:
        pytest.skip("needs 64 GB of free device memory")
    v = algo | FUSED
    L = depth(h, n, n, n, cutoff, v, 4)
    assert L == (1 if algo == W else 0) and exact_int_safe(2, n, L)
    g = torch.Generator(device="cuda")
    g.manual_seed(96)
    dA = torch.randint(-2, 3, (n, n), generator=g, device="cuda", dtype=torch.float32)
    dB = torch.randint(-2, 3, (n, n), generator=g, device="cuda", dtype=torch.float32)
    dC = torch.full((n, n), float("nan"), device="cuda")
    st = swmm.sw_smm(h, ctypes.c_void_p(dA.data_ptr()), n, ctypes.c_void_p(dB.data_ptr()), n,
                     ctypes.c_void_p(dC.data_ptr()), n, n, n, n, cutoff, v, None)
    swmm.check(h, st)
    swmm.check(h, swmm.sw_sync(h, None))
    rng = np.random.Generator(np.random.PCG64(97))
    idx = np.unique(np.concatenate([[0, 1, n // 2 - 1, n // 2, n - 2, n - 1], rng.choice(n, 10, replace=False)]))
    ti = torch.from_numpy(idx).cuda()
    Ar = dA[ti].double().cpu().numpy()
    Bc = dB[:, ti].double().cpu().numpy()
    Cs = dC[ti][:, ti].double().cpu().numpy()
    del dA, dB, dC
    torch.cuda.empty_cache()
    assert np.array_equal(Cs, oracle.naive(Ar, Bc))


def test_expired_device_wait_reports_timeout_and_the_handle_stays_usable(h):
    # failure detection without a fault: a reduce-add whose ordering counter nothing advances
    # waits until its bound, the kernel records the expiry and finishes, sw_sync reports it
    assert swmm.sw_selftest_expired_wait(h, None) == swmm.SW_ETIMEOUT
    assert "expired" in swmm.sw_last_error(h)
    assert swmm.sw_sync(h, None) == swmm.SW_OK  # the error word was consumed
    A, B = inputs.pair(300, 260, 520, "int", seed=98, dtype=np.float64, lim=4)
    assert np.array_equal(run(h, A, B, 200, W | FUSED), oracle.naive(A, B))


@pytest.mark.parametrize("ldc_pad", [12, 5])
@pytest.mark.parametrize("variant,cutoff,dtype", [(W | FUSED, 300, np.float32), (W | FUSED, 120, np.float32),
                                                  (swmm.SW_ALGO_NAIVE, 0, np.float32),
                                                  (W | FUSED | swmm.SW_LEAF_BF16X3, 300, np.float32),
                                                  (W | TWO, 200, np.float32), (W | FUSED, 60, np.float64)])
def test_output_stays_inside_its_view(h, ldc_pad, variant, cutoff, dtype):
    # canary bands: C is a view inside a larger buffer (rows above and below, columns on both
    # sides; ldc_pad 12 keeps 16-byte rows, 5 does not); every element outside the view keeps
    # its sentinel and the view holds the exact product (integer inputs)
    m, n, k = 520, 600, 460
    L = depth(h, m, n, k, cutoff, variant, 4 if dtype == np.float32 else 8)
    assert dtype == np.float64 or exact_int_safe(2, k, L)
    A, B = inputs.pair(m, n, k, "int", seed=99, dtype=np.float64, lim=2)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    dA = torch.from_numpy(A.astype(dtype)).cuda()
    dB = torch.from_numpy(B.astype(dtype)).cuda()
    ldc, top, left, bottom = n + ldc_pad, 3, 4, 5
    sentinel = -12345.0
    buf = torch.full((top + m + bottom, ldc), sentinel, dtype=tdt, device="cuda")
    view = buf[top:top + m, left:left + n]
    fn = swmm.sw_smm if dtype == np.float32 else swmm.sw_dmm
    st = fn(h, ctypes.c_void_p(dA.data_ptr()), k, ctypes.c_void_p(dB.data_ptr()), n, ctypes.c_void_p(view.data_ptr()),
            ldc, m, n, k, cutoff, variant, None)
    swmm.check(h, st)
    swmm.check(h, swmm.sw_sync(h, None))
    out = buf.cpu().numpy().astype(np.float64)
    inside = np.zeros(out.shape, bool)
    inside[top:top + m, left:left + n] = True
    assert np.all(out[~inside] == sentinel)
    assert np.array_equal(out[top:top + m, left:left + n], oracle.naive(A, B))
