"""The no-allocation entry point (sw_smm_noalloc) against the regular one and the oracle.

sw_smm_noalloc is for callers that cannot let this library allocate device memory: a runtime
that reserved nearly all of the GPU's memory for its own pool at start-up (a library cudaMalloc
would fail or fragment it), or a deployment that forbids device allocation after initialisation.
It keeps every temporary in a fixed static device array.  These tests call it through the C ABI
twice in a row per problem and check each result against sw_smm (the same one-level Winograd
product with TF32 leaves) and against the FP64 oracle, with the TF32 bound the parity tests use
(bit-exact on integer inputs); they check that a call after the first takes no device memory,
and, in a fresh process, that the array's memory is taken by the first call (lazy module
loading) and by nothing after it.  The file is collected last, and it passes alone in a fresh
process as well as after the other tests.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bounds
import oracle
from paper_2309_00628_gb300 import inputs, swmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W1 = swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(dA, dB, C, m, n, k):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return swmm.sw_smm_noalloc(_ptr(dA), k, _ptr(dB), n, _ptr(C), n, m, n, k, stream)


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    hd = swmm.sw_create(0)
    yield hd
    swmm.sw_destroy(hd)


def test_noalloc_two_calls_match_sw_smm_and_the_oracle(h):
    for (m, n, k, dist, seed) in [(1024, 1024, 1024, "uniform", 0), (700, 900, 520, "uniform", 5),
                                  (384, 260, 300, "int", 9)]:
        A, B = inputs.pair(m, n, k, dist, seed=seed, dtype=np.float32, lim=4)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        cutoff = (min(m, n, k) + 1) // 2  # exactly one recursion level
        st, L = swmm.sw_mm_depth(m, n, k, cutoff, W1, 4)
        assert st == swmm.SW_OK and L == 1
        ref = swmm.mm(h, dA, dB, cutoff, W1, sync=True).double().cpu().numpy()  # the regular entry point
        R = oracle.naive(A.astype(np.float64), B.astype(np.float64))
        tol = bounds.tol_tf32(m * n, k, 1, A, B)
        got = []
        for call in range(2):
            C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
            st = _noalloc(dA, dB, C, m, n, k)
            assert st == swmm.SW_OK, (call, swmm.STATUS_NAMES[st])
            got.append(C.double().cpu().numpy())
            if dist == "int":
                assert np.array_equal(got[-1], R) and np.array_equal(got[-1], ref), call
            else:
                assert oracle.err_norm(got[-1], ref, A, B) <= tol, call
                assert oracle.err_norm(got[-1], R, A, B) <= tol, call
        if dist == "int":
            assert np.array_equal(got[0], got[1])  # the shared scratch left nothing behind
    # a problem larger than the static array is refused before any memory is touched
    C = torch.zeros(1, device="cuda")
    st = _noalloc(dA, dB, C, 4096, 4096, 4096)
    assert st == swmm.SW_EBUDGET


def test_noalloc_takes_no_device_memory_after_its_first_call(h):
    m = n = k = 512
    A, B = inputs.pair(m, n, k, "int", seed=11, dtype=np.float32, lim=4)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    assert _noalloc(dA, dB, C, m, n, k) == swmm.SW_OK  # first call on this device in this process, or not
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _noalloc(dA, dB, C, m, n, k) == swmm.SW_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, free0 - free1
    assert np.array_equal(C.double().cpu().numpy(), oracle.naive(A.astype(np.float64), B.astype(np.float64)))


_FRESH = r"""
import ctypes, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2309_00628_gb300 import inputs, swmm
swmm.load()
m = n = k = 512
A, B = inputs.pair(m, n, k, "int", seed=12, dtype=np.float32, lim=4)
dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
C = torch.empty((m, n), dtype=torch.float32, device="cuda")
s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
call = lambda: swmm.sw_smm_noalloc(ctypes.c_void_p(dA.data_ptr()), k, ctypes.c_void_p(dB.data_ptr()), n,
                                   ctypes.c_void_p(C.data_ptr()), n, m, n, k, s)
torch.cuda.synchronize()
free = [torch.cuda.mem_get_info()[0]]
st = [call()]
torch.cuda.synchronize()
free.append(torch.cuda.mem_get_info()[0])
st.append(call())
torch.cuda.synchronize()
free.append(torch.cuda.mem_get_info()[0])
print(json.dumps({"free": free, "status": st, "C": C.double().cpu().numpy().tolist()}))
"""


def test_noalloc_in_a_fresh_process():
    # with lazy module loading (CUDA's default) the first call places the static array (and the
    # code of the kernels it uses) in device memory; the second call takes nothing
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    f0, f1, f2 = out["free"]
    assert out["status"] == [swmm.SW_OK, swmm.SW_OK]
    assert f0 - f1 >= swmm.SW_NOALLOC_SCRATCH_BYTES, (f0, f1)  # the array arrives with the first call
    assert f2 == f1, (f1, f2)                                      # ... and nothing after it
    A, B = inputs.pair(512, 512, 512, "int", seed=12, dtype=np.float64, lim=4)
    assert np.array_equal(np.array(out["C"]), oracle.naive(A, B))
