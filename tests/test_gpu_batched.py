"""Batched products (sw_mm_batched): many independent FP32 products in one grouped launch.

Each result must equal the FP64 oracle bit for bit on integer inputs, equal its solo sw_smm run,
survive graph replay with new data in the same buffers, and (512-problem workload) satisfy
Freivalds' identity C x = A (B x) in FP64 within the TF32 bound.
"""
import ctypes

import numpy as np
import pytest

import bounds
import oracle
from paper_2309_00628_gb300 import inputs, swmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
W = swmm.SW_ALGO_WINOGRAD


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    hd = swmm.sw_create(0)
    yield hd
    swmm.sw_destroy(hd)


def make_batch(shapes, dist, seed, lim=4, pad_lda=False):
    """Device operands for each (m, n, k); returns (problem array, host A/B list, device tensors)."""
    probs, host, keep = [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = inputs.pair(m, n, k, dist, seed=seed + 2 * i, dtype=np.float32, lim=lim)
        lda = k + (3 if (pad_lda and i % 2) else 0)
        dA = torch.zeros((max(m, 1), max(lda, 1)), dtype=torch.float32, device="cuda")
        if m and k:
            dA[:m, :k] = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(B).cuda() if k and n else torch.zeros(1, device="cuda")
        dC = torch.full((max(m, 1), max(n, 1)), float("nan"), dtype=torch.float32, device="cuda")
        probs.append(swmm.sw_problem(dA.data_ptr(), max(lda, 1), dB.data_ptr(), max(n, 1), dC.data_ptr(), max(n, 1),
                                     m, n, k))
        host.append((A, B))
        keep.append((dA, dB, dC))
    return (swmm.sw_problem * len(probs))(*probs), host, keep


def run_batch(h, probs, cutoff, variant=W | swmm.SW_SCHED_FUSED):
    swmm.check(h, swmm.sw_mm_batched(h, len(probs), probs, cutoff, variant, None))
    swmm.check(h, swmm.sw_sync(h, None))


SHAPES = [(128, 256, 32), (97, 131, 203), (300, 500, 200), (1, 1, 1), (64, 2000, 7), (515, 77, 1030),
          (256, 256, 256), (0, 5, 5), (5, 0, 5), (33, 45, 1), (700, 700, 700), (129, 257, 33)]


@pytest.mark.parametrize("cutoff", [100000, 128])
def test_batched_integers_bit_exact(h, cutoff):
    probs, host, keep = make_batch(SHAPES, "int", seed=0, lim=2, pad_lda=True)
    run_batch(h, probs, cutoff)
    for (A, B), (dA, dB, dC), (m, n, k) in zip(host, keep, SHAPES):
        if m == 0 or n == 0:
            continue
        C = dC[:m, :n].double().cpu().numpy()
        assert np.array_equal(C, oracle.naive(A.astype(np.float64), B.astype(np.float64))), (m, n, k, cutoff)


_FORM_SCRIPT = r"""
import sys
import numpy as np, torch
sys.path[:0] = [sys.argv[1], sys.argv[1] + "/tests"]
import oracle
from paper_2309_00628_gb300 import inputs, swmm
from test_gpu_batched import SHAPES, make_batch, run_batch
swmm.load()
h = swmm.sw_create(0)
for cutoff in (100000, 128):
    probs, host, keep = make_batch(SHAPES, "int", seed=5, lim=2, pad_lda=True)
    run_batch(h, probs, cutoff)
    for (A, B), (dA, dB, dC), (m, n, k) in zip(host, keep, SHAPES):
        if m and n:
            C = dC[:m, :n].double().cpu().numpy()
            assert np.array_equal(C, oracle.naive(A.astype(np.float64), B.astype(np.float64))), (m, n, k, cutoff)
    run_batch(h, probs, cutoff)  # the captured graph once more: the in-launch pack counters advance
    for (A, B), (dA, dB, dC), (m, n, k) in zip(host, keep, SHAPES):
        if m and n:
            assert np.array_equal(dC[:m, :n].double().cpu().numpy(),
                                  oracle.naive(A.astype(np.float64), B.astype(np.float64))), (m, n, k, cutoff)
swmm.sw_destroy(h)
print("forms ok")
"""


@pytest.mark.parametrize("form", ["cta", "pair", "pack"])
def test_batched_forms_integers_bit_exact(form):
    # each form of the grouped launch (one CTA per tile; CTA pairs with a packing launch before
    # the GEMM; CTA pairs packing inside the GEMM launch), selected per process, on integer batches
    # with unaligned leading dimensions, flat (cutoff 100000) and recursive (cutoff 128)
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SWMM_BATCH_FORM=form)
    r = subprocess.run([sys.executable, "-c", _FORM_SCRIPT, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "forms ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_batched_equals_solo_runs_and_replays(h):
    shapes = [(300, 500, 200), (129, 257, 33), (700, 700, 700), (97, 131, 203)]
    probs, host, keep = make_batch(shapes, "uniform", seed=10)
    run_batch(h, probs, 0)
    first = [dC[:m, :n].clone() for (dA, dB, dC), (m, n, k) in zip(keep, shapes)]
    for (dA, dB, dC), (m, n, k), c0 in zip(keep, shapes, first):
        solo = swmm.mm(h, dA[:m, :k].contiguous(), dB, 0, swmm.SW_ALGO_NAIVE, sync=True)
        assert torch.equal(solo, c0), (m, n, k)
    # replay the captured graph on new data in the same buffers
    for (dA, dB, dC), (m, n, k) in zip(keep, shapes):
        dA.mul_(-2.0)
    run_batch(h, probs, 0)
    for (dA, dB, dC), (m, n, k), c0 in zip(keep, shapes, first):
        assert torch.equal(dC[:m, :n], -2.0 * c0), (m, n, k)


def test_batched_512_uneven_products(h):
    # 512 products, m, n, k each round(exp(U(ln 96, ln 3000))), entries uniform[-1, 1]
    shapes = inputs.batched_shapes(512, seed=2)
    g = torch.Generator(device="cuda")
    g.manual_seed(2)
    probs, keep = [], []
    for (m, n, k) in shapes:
        dA = torch.rand((m, k), generator=g, device="cuda") * 2 - 1
        dB = torch.rand((k, n), generator=g, device="cuda") * 2 - 1
        dC = torch.empty((m, n), device="cuda")
        probs.append(swmm.sw_problem(dA.data_ptr(), k, dB.data_ptr(), n, dC.data_ptr(), n, m, n, k))
        keep.append((dA, dB, dC))
    arr = (swmm.sw_problem * len(probs))(*probs)
    run_batch(h, arr, 0)
    # the first call with cutoff 0 timed the grouped launch's shapes and cutoffs on this list
    st, t = swmm.sw_last_tuning(h)
    assert st == swmm.SW_OK
    assert t["candidates"] == 5 and t["tile_n"] in (128, 256) and t["cta_pair"] in (0, 1, 2) and t["ms"] > 0, t
    rng = np.random.Generator(np.random.PCG64(3))
    worst = 0.0
    for i, ((dA, dB, dC), (m, n, k)) in enumerate(zip(keep, shapes)):
        A, B, C = (t.double().cpu().numpy() for t in (dA, dB, dC))
        x = rng.uniform(-1, 1, n)
        err = np.max(np.abs(C @ x - A @ (B @ x))) / (n * k * np.max(np.abs(A)) * np.max(np.abs(B)))
        worst = max(worst, err)
        if i < 6:  # exact oracle rows on a few products
            rows = rng.choice(m, min(m, 4), replace=False)
            R = oracle.naive(A[rows], B)
            st, L = swmm.sw_mm_depth(m, n, k, t["cutoff"], swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, 4)
            assert st == swmm.SW_OK
            assert oracle.err_norm(C[rows], R, A, B) <= bounds.tol_tf32(R.size, k, L, A, B)
    assert worst <= 8 * 2.0 ** -9 / np.sqrt(96), worst
