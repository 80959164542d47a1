"""The no-allocation entry point (sw_smm_noalloc) against the regular one.

sw_smm_noalloc serves callers that cannot let the library allocate device memory -- a runtime
that has reserved the GPU's memory for its own pool, or a deployment that forbids allocation
after start-up; it keeps all its temporaries in a fixed static device array.  This test calls it
through the C ABI twice in a row and checks each result against sw_smm (same algorithm, same
depth, same TF32 leaves) within the tolerance the parity tests use.  It lives in a file that
pytest collects last, and it passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2309_00628_gb300 import inputs, swmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def tol_tf32(k, L):
    # the parity tests' TF32 bound (8 * 2^-9 * 3^L / sqrt(k) + 2^-20, normalised)
    return 8.0 * 2.0 ** -9 * 3.0 ** L / np.sqrt(k) + 2.0 ** -20


def test_noalloc_matches_regular_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    h = swmm.sw_create(0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        for (m, n, k, dist, seed) in [(1024, 1024, 1024, "uniform", 0), (700, 900, 520, "uniform", 5),
                                      (384, 260, 300, "int", 9)]:
            A, B = inputs.pair(m, n, k, dist, seed=seed, dtype=np.float32, lim=4)
            dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            cutoff = (min(m, n, k) + 1) // 2  # exactly one recursion level
            v = swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED
            st, L = swmm.sw_mm_depth(m, n, k, cutoff, v, 4)
            assert st == swmm.SW_OK and L == 1
            ref = swmm.mm(h, dA, dB, cutoff, v, sync=True).double().cpu().numpy()
            C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
            st = swmm.sw_smm_noalloc(ptr(dA), k, ptr(dB), n, ptr(C), n, m, n, k, stream)
            assert st == swmm.SW_OK, swmm.STATUS_NAMES[st]
            got = C.double().cpu().numpy()
            if dist == "int":
                assert np.array_equal(got, ref)
            else:
                err = np.max(np.abs(got - ref)) / (k * np.max(np.abs(A)) * np.max(np.abs(B)))
                assert err <= tol_tf32(k, 1), err
        # a problem larger than the static array is refused before any memory is touched
        st = swmm.sw_smm_noalloc(ptr(dA), 4096, ptr(dB), 4096, ptr(C), 4096, 4096, 4096, 4096, stream)
        assert st == swmm.SW_EBUDGET
    finally:
        swmm.sw_destroy(h)
