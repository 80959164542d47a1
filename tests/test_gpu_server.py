"""Serving loop (sw_server_*): products of mixed shape, precision and schedule admitted together.

Integer-valued inputs keep every partial sum an exact integer, so each served result must equal
the FP64 oracle bit for bit whatever order the resident loop adds tile contributions in.  Float
inputs must meet the TF32 bound (NAIVE products: bit-identical to their solo sw_smm result, one
STORE per tile in the same k order).  Also: a request larger than the arena is refused with
SW_EBUDGET, a zero-length wait on unfinished work returns SW_ETIMEOUT and keeps the ticket, several
host threads may submit at once, and stop drains what is queued.
"""
import ctypes
import threading

import numpy as np
import pytest

import bounds
import oracle
from paper_2309_00628_gb300 import inputs, swmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

W, S, N = swmm.SW_ALGO_WINOGRAD, swmm.SW_ALGO_STRASSEN, swmm.SW_ALGO_NAIVE
FUSED, TWO, INPL = swmm.SW_SCHED_FUSED, swmm.SW_SCHED_TWO_TEMP, swmm.SW_SCHED_IN_PLACE
BF = swmm.SW_LEAF_BF16X3


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    swmm.load(build_if_missing=True)
    hd = swmm.sw_create(0)
    yield hd
    swmm.sw_destroy(hd)


@pytest.fixture
def srv(h):
    cfg = swmm.sw_server_cfg(0, 32, 8 << 30, 5000)
    swmm.check(h, swmm.sw_server_start(h, cfg))
    yield h
    swmm.check(h, swmm.sw_server_stop(h))


ALGO_NAME = {0: "naive", 1: "strassen", 2: "winograd", 3: "knuth"}


def device_problem(m, n, k, dist, seed, eb=4, lim=2):
    dt, tdt = (np.float32, torch.float32) if eb == 4 else (np.float64, torch.float64)
    A, B = inputs.pair(m, n, k, dist, seed=seed, dtype=dt, lim=lim)
    dA = torch.from_numpy(A).cuda() if m and k else torch.zeros((max(m, 1), max(k, 1)), dtype=tdt, device="cuda")
    dB = torch.from_numpy(B).cuda() if k and n else torch.zeros((max(k, 1), max(n, 1)), dtype=tdt, device="cuda")
    dC = torch.full((max(m, 1), max(n, 1)), float("nan"), dtype=tdt, device="cuda")
    return A, B, dA, dB, dC


def req(dA, dB, dC, m, n, k, eb, cutoff, variant):
    return swmm.sw_request(eb, dA.data_ptr(), max(k, 1), dB.data_ptr(), max(n, 1), dC.data_ptr(), max(n, 1), m, n,
                           k, cutoff, variant)


# (m, n, k, elem_bytes, cutoff, variant): resident NAIVE / FUSED products, an unaligned A (packed
# on a side stream), FP64 and split-BF16 requests (whole plan on a side stream), the step-by-step
# schedules (pads and peels included), and the empty cases
MIX = [
    (512, 512, 512, 4, 0, N),
    (1024, 768, 1024, 4, 256, W | FUSED),
    (1024, 1024, 1024, 4, 512, S | FUSED),
    (515, 77, 1030, 4, 128, W | FUSED),
    (300, 500, 200, 8, 64, W | FUSED),
    (640, 640, 640, 4, 256, W | TWO),
    (512, 512, 512, 4, 256, W | FUSED | BF),
    (257, 300, 129, 4, 64, W | TWO),
    (260, 260, 260, 4, 64, W | TWO | swmm.SW_PEEL),
    (512, 512, 512, 4, 128, W | INPL),
    (0, 5, 5, 4, 0, W),
    (5, 5, 0, 4, 0, W),
    (2048, 2048, 2048, 4, 1024, W | FUSED),
    (128, 256, 32, 4, 0, W),
    (96, 4096, 64, 4, 0, N),
    (1536, 1024, 512, 4, 256, W | FUSED),
]


def test_server_mix_integers_bit_exact(srv):
    h = srv
    probs = []
    for i, (m, n, k, eb, cutoff, var) in enumerate(MIX):
        A, B, dA, dB, dC = device_problem(m, n, k, "int", seed=100 + 2 * i, eb=eb)
        probs.append((A, B, dA, dB, dC, req(dA, dB, dC, m, n, k, eb, cutoff, var)))
    torch.cuda.synchronize()
    tickets = []
    for p in probs:
        st, t = swmm.sw_server_submit(h, p[5])
        swmm.check(h, st)
        tickets.append(t)
    for t in tickets:
        swmm.check(h, swmm.sw_server_wait(h, t, 120 * 10 ** 9))
    for (m, n, k, eb, cutoff, var), (A, B, dA, dB, dC, _) in zip(MIX, probs):
        if m == 0 or n == 0:
            continue
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        C = dC[:m, :n].cpu().numpy().astype(np.float64)
        assert np.array_equal(C, R), ((m, n, k, eb, cutoff, hex(var)), np.abs(C - R).max())


def test_server_mix_floats(srv, h):
    """Float inputs: the TF32 / FP64 bounds of the parity tests, and NAIVE results identical to solo sw_smm."""
    cases = [(512, 512, 512, 4, 0, N), (1024, 768, 1024, 4, 256, W | FUSED), (2048, 2048, 2048, 4, 1024, S | FUSED),
             (300, 500, 200, 8, 64, W | FUSED), (640, 384, 896, 4, 0, N), (1000, 1000, 1000, 4, 256, W | TWO)]
    probs = []
    for i, (m, n, k, eb, cutoff, var) in enumerate(cases):
        A, B, dA, dB, dC = device_problem(m, n, k, "uniform", seed=300 + 2 * i, eb=eb)
        probs.append((A, B, dA, dB, dC, req(dA, dB, dC, m, n, k, eb, cutoff, var)))
    torch.cuda.synchronize()
    tickets = []
    for p in probs:
        st, t = swmm.sw_server_submit(srv, p[5])
        swmm.check(srv, st)
        tickets.append(t)
    for t in tickets:
        swmm.check(srv, swmm.sw_server_wait(srv, t, 120 * 10 ** 9))
    for (m, n, k, eb, cutoff, var), (A, B, dA, dB, dC, _) in zip(cases, probs):
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        C = dC.cpu().numpy().astype(np.float64)
        st, L = swmm.sw_mm_depth(m, n, k, cutoff, var, eb)
        err = oracle.err_norm(C, R, A, B)
        zero = oracle.err_norm(np.zeros_like(R), R, A, B)
        bound = bounds.tol_fp64 if eb == 8 else bounds.tol_tf32
        tol = bound(C.size, k, L, A, B, ALGO_NAME[var & 0xF])
        assert err <= tol and err <= 0.3 * zero, ((m, n, k, cutoff, hex(var)), err, tol)
        if var == N and eb == 4:
            solo = torch.full_like(dC, float("nan"))
            fn = swmm.sw_smm
            swmm.check(h, fn(h, ctypes.c_void_p(dA.data_ptr()), k, ctypes.c_void_p(dB.data_ptr()), n,
                             ctypes.c_void_p(solo.data_ptr()), n, m, n, k, cutoff, var, None))
            swmm.check(h, swmm.sw_sync(h, None))
            assert torch.equal(solo, dC), (m, n, k)


def test_server_long_requests_beside_short_ones(srv):
    """Requests estimated at 2 ms of work or more have their ops enqueued by the launcher thread
    (deep FP64 plans hold thousands of kernels); two such FP64 products run beside short FP32 and
    FP64 ones, every result bit-exact against the oracle on integer inputs."""
    cases = [(1280, 1280, 1280, 8, 0, W | FUSED), (512, 512, 512, 4, 0, N), (300, 500, 200, 8, 64, W | FUSED),
             (1536, 1152, 1280, 8, 0, W | FUSED), (1024, 768, 1024, 4, 256, W | FUSED), (640, 640, 640, 4, 0, W)]
    for (m, n, k, eb, cutoff, var) in cases[:1] + cases[3:4]:
        assert 2.0 * m * n * k / 1.5e9 >= 2.0  # long by the server's estimate (FP64 at 1.5 TFLOP/s)
    probs = []
    for i, (m, n, k, eb, cutoff, var) in enumerate(cases):
        A, B, dA, dB, dC = device_problem(m, n, k, "int", seed=500 + 2 * i, eb=eb, lim=1)
        probs.append((A, B, dA, dB, dC, req(dA, dB, dC, m, n, k, eb, cutoff, var)))
    torch.cuda.synchronize()
    tickets = []
    for p in probs:
        st, t = swmm.sw_server_submit(srv, p[5])
        swmm.check(srv, st)
        tickets.append(t)
    for t in tickets:
        swmm.check(srv, swmm.sw_server_wait(srv, t, -1))
    for (m, n, k, eb, cutoff, var), (A, B, dA, dB, dC, _) in zip(cases, probs):
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        assert np.array_equal(dC[:m, :n].cpu().numpy().astype(np.float64), R), (m, n, k, eb, hex(var))


def test_server_budget_and_timeout(h):
    cfg = swmm.sw_server_cfg(0, 8, 64 << 20, 2000)
    swmm.check(h, swmm.sw_server_start(h, cfg))
    try:
        # the operand sums alone need 512 MiB: more than the arena
        m = n = k = 8192
        big = swmm.sw_request(4, 1 << 20, k, 1 << 20, n, 1 << 20, n, m, n, k, 4096, W | FUSED)
        st, _ = swmm.sw_server_submit(h, big)
        assert st == swmm.SW_EBUDGET, swmm.sw_last_error(h)
        # a request that fits still runs; a zero wait right after submit finds it unfinished
        m = n = k = 1024
        A, B, dA, dB, dC = device_problem(m, n, k, "int", seed=7)
        torch.cuda.synchronize()
        st, t = swmm.sw_server_submit(h, req(dA, dB, dC, m, n, k, 4, 512, W | FUSED))
        swmm.check(h, st)
        assert swmm.sw_server_wait(h, t, 0) == swmm.SW_ETIMEOUT
        swmm.check(h, swmm.sw_server_wait(h, t, 60 * 10 ** 9))
        assert swmm.sw_server_wait(h, t, 0) == swmm.SW_EINVAL  # collected
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), R)
        # bad arguments are refused at submit
        bad = swmm.sw_request(4, 0, 16, 0, 16, 0, 16, 16, 16, 16, 0, W)
        assert swmm.sw_server_submit(h, bad)[0] == swmm.SW_EINVAL
    finally:
        swmm.check(h, swmm.sw_server_stop(h))
    assert swmm.sw_server_stop(h) == swmm.SW_EINVAL  # not running any more


def test_server_threads_and_drain(h):
    """Four host threads submit and wait at once; then a batch is left to stop(), which drains it."""
    swmm.check(h, swmm.sw_server_start(h, None))
    shapes = [(256 + 128 * (i % 5), 512, 256 + 64 * (i % 3)) for i in range(24)]
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        A, B, dA, dB, dC = device_problem(m, n, k, "int", seed=500 + 2 * i)
        probs.append((A, B, dA, dB, dC, req(dA, dB, dC, m, n, k, 4, 128, W | FUSED)))
    torch.cuda.synchronize()
    errors = []

    def worker(part):
        try:
            ts = []
            for p in part:
                st, t = swmm.sw_server_submit(h, p[5])
                assert st == swmm.SW_OK
                ts.append(t)
            for t in ts:
                assert swmm.sw_server_wait(h, t, 60 * 10 ** 9) == swmm.SW_OK
        except AssertionError as e:  # reported by the main thread
            errors.append(e)

    ths = [threading.Thread(target=worker, args=(probs[j::4],)) for j in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errors, (errors, swmm.sw_last_error(h))
    for A, B, dA, dB, dC, _ in probs:
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), R)
    # drain on stop: nobody waits for these tickets
    for _, _, _, _, dC, _ in probs:
        dC.fill_(float("nan"))
    torch.cuda.synchronize()
    for p in probs:
        swmm.check(h, swmm.sw_server_submit(h, p[5])[0])
    swmm.check(h, swmm.sw_server_stop(h))
    for A, B, dA, dB, dC, _ in probs:
        R = oracle.naive_mt(A.astype(np.float64), B.astype(np.float64))
        assert np.array_equal(dC.cpu().numpy().astype(np.float64), R)
