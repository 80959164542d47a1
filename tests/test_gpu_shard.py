"""sw_mm_products, the per-rank computation of the split of the top recursion level.

Ranks are emulated one after another on the one GPU (ranks whose kernels waited on each other
must not share a GPU; these do not wait on each other): the partial result of every mask equals
the oracle's contribution of the same top-level products (bit-exact on integer inputs, with the
block split the library uses), and the partials of the masks of 2, 3 and 7 ranks add up to the
exact product; on float inputs the summed partials stay within the TF32 / FP64 bounds of the
parity tests.
"""
import ctypes

import numpy as np
import pytest

import bounds
import oracle
from paper_2309_00628_gb300 import inputs, shard, swmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W, S, K = swmm.SW_ALGO_WINOGRAD, swmm.SW_ALGO_STRASSEN, swmm.SW_ALGO_WINOGRAD_KNUTH
ORC = {W: oracle.WINOGRAD, S: oracle.STRASSEN, K: oracle.KNUTH}
NAME = {W: "winograd", S: "strassen", K: "knuth"}


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    hd = swmm.sw_create(0)
    yield hd
    swmm.sw_destroy(hd)


def partial(h, A, B, cutoff, variant, mask):
    return shard.gpu_partial(h, A, B, cutoff, variant, mask)


# shapes whose leaf blocks need no rounding (FP32 leaf blocks have k / 2^L a multiple of 32 and
# n / 2^L a multiple of 4), so the library splits the top level where the oracle's padding does
@pytest.mark.parametrize("algo", [W, S, K])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("m,n,k,cutoff", [(512, 512, 512, 256), (300, 256, 512, 64), (512, 384, 256, 40)])
def test_partials_match_the_oracle_and_add_up(h, algo, dtype, m, n, k, cutoff):
    eb = 4 if dtype == np.float32 else 8
    v = algo | swmm.SW_SCHED_FUSED
    st, L = swmm.sw_mm_depth(m, n, k, cutoff, v, eb)
    assert st == swmm.SW_OK and 1 <= L <= 3
    lim = 1 if L >= 2 else 2
    A, B = inputs.pair(m, n, k, "int", seed=31, dtype=dtype, lim=lim)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ex = oracle.naive(A64, B64)
    for world in (2, 3, 7):
        tot = torch.zeros((m, n), dtype=dA.dtype, device="cuda")
        for mask in shard.product_masks(world):
            C = partial(h, dA, dB, cutoff, v, mask)
            tot += C
            if world == 7:  # one product per rank
                want = oracle.recursive_products(ORC[algo], A64, B64, cutoff, mask)
                assert np.array_equal(C.double().cpu().numpy(), want), (world, mask)
        torch.cuda.synchronize()
        assert np.array_equal(tot.double().cpu().numpy(), ex), world


@pytest.mark.parametrize("algo", [W, S])
def test_partials_add_up_within_the_float_bounds(h, algo):
    n, cutoff = 1024, 256  # depth 2
    v = algo | swmm.SW_SCHED_FUSED
    for dtype, bound in ((np.float32, bounds.tol_tf32), (np.float64, bounds.tol_fp64)):
        A, B = inputs.pair(n, n, n, "uniform", seed=32, dtype=dtype)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        tot = sum(partial(h, dA, dB, cutoff, v, mk) for mk in shard.product_masks(3))
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        err = oracle.err_norm(tot.double().cpu().numpy(), R, A, B)
        assert err <= bound(n * n, n, 2, A, B, NAME[algo]), (dtype, err)


def test_split_bf16_partials_add_up(h):
    n, cutoff = 512, 256
    v = W | swmm.SW_SCHED_FUSED | swmm.SW_LEAF_BF16X3
    A, B = inputs.pair(n, n, n, "int", seed=33, dtype=np.float32, lim=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    tot = sum(partial(h, dA, dB, cutoff, v, mk) for mk in shard.product_masks(2))
    assert np.array_equal(tot.double().cpu().numpy(), oracle.naive(A.astype(np.float64), B.astype(np.float64)))


def test_product_subset_argument_errors(h):
    d = torch.zeros((64, 64), device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    call = lambda v, cutoff, mask, eb=4: swmm.sw_mm_products(h, eb, p, 64, p, 64, p, 64, 64, 64, 64, cutoff, v, mask)
    assert call(W | swmm.SW_SCHED_FUSED, 32, 0x80) == swmm.SW_EINVAL
    assert call(W | swmm.SW_SCHED_FUSED, 32, 1, eb=2) == swmm.SW_EINVAL
    assert call(swmm.SW_ALGO_NAIVE, 32, 1) == swmm.SW_EUNSUPPORTED
    assert call(W | swmm.SW_SCHED_TWO_TEMP, 32, 1) == swmm.SW_EUNSUPPORTED
    assert call(W | swmm.SW_SCHED_FUSED, 1000, 1) == swmm.SW_EUNSUPPORTED  # depth 0
    assert swmm.sw_sync(h, None) == swmm.SW_OK
