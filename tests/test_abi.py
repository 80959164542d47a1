"""CPU tests of the C-ABI library: it loads, exports every symbol include/swmm.h
declares, and its host-side planning logic (depth rule, workspace accounting,
argument checks) agrees with the oracle's counting.  No GPU is touched."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2309_00628_gb300 import build, swmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swmm.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return swmm.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:sw_status|const char \*|void)\s*\**\s*(sw_\w+)\s*\(", text, re.M)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("sw_create", "sw_destroy", "sw_smm", "sw_dmm", "sw_smm_host", "sw_sync", "sw_mm_workspace_size",
              "sw_last_error"):
        assert s in syms


def test_binding_constants_match_the_header():
    text = open(HEADER).read()
    defines = dict(re.findall(r"^#define (SW_\w+) (.+)$", text, re.M))
    for name, val in defines.items():
        if name in ("SW_PROFILE_KINDS",) or not hasattr(swmm, name):
            continue
        assert getattr(swmm, name) == eval(val.replace("u", "").replace("(32 << 20)", "33554432")), name
    assert swmm.SW_NOALLOC_SCRATCH_BYTES == 32 << 20 and "(32u << 20)" in defines["SW_NOALLOC_SCRATCH_BYTES"]


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(swmm.library_path())
    missing = [s for s in declared_symbols() if not hasattr(so, s)]
    assert not missing, missing


@pytest.mark.parametrize("m,n,k,cutoff", [(256, 256, 256, 32), (16, 16, 16, 12), (100, 300, 3000, 32),
                                          (33, 33, 33, 32), (8192, 8192, 8192, 1024), (5, 7, 9, 1)])
def test_depth_rule_matches_oracle(lib, m, n, k, cutoff):
    for v in (swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_TWO_TEMP, swmm.SW_ALGO_STRASSEN | swmm.SW_SCHED_ALLOC):
        st, d = swmm.sw_mm_depth(m, n, k, cutoff, v, 8)
        assert st == swmm.SW_OK and d == oracle.depth(m, n, k, cutoff)
    st, d = swmm.sw_mm_depth(m, n, k, cutoff, swmm.SW_ALGO_NAIVE, 4)
    assert d == 0


def test_fused_depth_is_capped_at_three(lib):
    st, d = swmm.sw_mm_depth(4096, 4096, 4096, 32, swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, 4)
    assert st == swmm.SW_OK and d == 3


@pytest.mark.parametrize("m,n,k,want", [(8192, 8192, 8192, 6), (4096, 4096, 4096, 5), (4100, 4100, 4100, 5),
                                        (4098, 4096, 4096, 4), (4097, 4096, 4096, 3), (2048, 2080, 2064, 4),
                                        (1040, 1056, 1024, 3)])
def test_fused_fp64_depth_grows_by_exact_halvings(lib, m, n, k, want):
    # FP64 Strassen / BDPZ products go past three fused levels by one Table 2 / Alg. 2 level per
    # exact halving of m, n and k while the fused bottom keeps a smallest side >= 1024; Knuth's
    # form and FP32 stay at three
    F = swmm.SW_SCHED_FUSED
    for a in (swmm.SW_ALGO_WINOGRAD, swmm.SW_ALGO_STRASSEN):
        assert swmm.sw_mm_depth(m, n, k, 8, a | F, 8) == (swmm.SW_OK, want)
    assert swmm.sw_mm_depth(m, n, k, 8, swmm.SW_ALGO_WINOGRAD_KNUTH | F, 8) == (swmm.SW_OK, 3)
    assert swmm.sw_mm_depth(m, n, k, 8, swmm.SW_ALGO_WINOGRAD | F, 4) == (swmm.SW_OK, 3)
    # the FP64 static default (cutoff <= 0) keeps leaves of more than 128
    assert swmm.sw_mm_depth(4096, 4096, 4096, 0, swmm.SW_ALGO_WINOGRAD | F, 8) == (swmm.SW_OK, 5)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_workspace_matches_schedule_counts(lib, L):
    n = 16384
    cutoff = n >> L  # halve exactly L times
    for sched, which in ((swmm.SW_SCHED_ALLOC, 0), (swmm.SW_SCHED_TWO_TEMP, 1)):
        # FP64: exactly the schedule's temporaries
        st, b = swmm.sw_mm_workspace_size(n, n, n, cutoff, swmm.SW_ALGO_WINOGRAD | sched, 8)
        assert st == swmm.SW_OK
        assert b == pytest.approx(oracle.workspace_elems(which, n, n, n, L) * 8, rel=1e-3)
        # FP32: the same temporaries (the TF32 tensor cores read B as stored: no B^T copy)
        st, b = swmm.sw_mm_workspace_size(n, n, n, cutoff, swmm.SW_ALGO_WINOGRAD | sched, 4)
        assert st == swmm.SW_OK
        assert b == pytest.approx(oracle.workspace_elems(which, n, n, n, L) * 4, rel=1e-3)
    for eb in (4, 8):  # in place: temporaries live in A, B, C
        st, b = swmm.sw_mm_workspace_size(n, n, n, cutoff, swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_IN_PLACE, eb)
        assert st == swmm.SW_OK and b == 0


def test_fused_workspace_counts_materialised_sums(lib):
    # Winograd: 7^L - 3^L leaf operands per side are sums (the rest are plain blocks)
    n = 8192
    for L in (1, 2, 3):
        st, b = swmm.sw_mm_workspace_size(n, n, n, n >> L, swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED, 4)
        blk = (n >> L) ** 2 * 4
        assert st == swmm.SW_OK
        assert b == pytest.approx(2 * (7 ** L - 3 ** L) * blk, rel=1e-3)


def test_argument_errors_without_gpu(lib):
    st, _ = swmm.sw_mm_workspace_size(-1, 4, 4, 1, 0, 4)
    assert st == swmm.SW_EINVAL
    st, _ = swmm.sw_mm_workspace_size(4, 4, 4, 1, 0, 3)
    assert st == swmm.SW_EINVAL
    st, _ = swmm.sw_mm_workspace_size(8, 8, 8, 1, swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_IN_PLACE, 4)
    assert st == swmm.SW_OK
    st, _ = swmm.sw_mm_workspace_size(8, 4, 8, 1, swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_IN_PLACE, 4)
    assert st == swmm.SW_EUNSUPPORTED
    st, _ = swmm.sw_mm_workspace_size(8, 8, 8, 1, swmm.SW_ALGO_STRASSEN | swmm.SW_SCHED_TWO_TEMP, 4)
    assert st == swmm.SW_EUNSUPPORTED
    assert swmm.load().sw_smm(None, None, 1, None, 1, None, 1, 1, 1, 1, 1, 0, None) == swmm.SW_EINVAL
    # the Winograd-step FP64 leaf: FP64 entries with the Winograd algorithms only
    wt = swmm.SW_LEAF_F64_WTILE
    assert swmm.sw_mm_workspace_size(64, 64, 64, 16, swmm.SW_ALGO_WINOGRAD | wt, 4)[0] == swmm.SW_EINVAL
    assert swmm.sw_mm_workspace_size(64, 64, 64, 16, swmm.SW_ALGO_NAIVE | wt, 8)[0] == swmm.SW_EUNSUPPORTED
    assert swmm.sw_mm_workspace_size(64, 64, 64, 16, swmm.SW_ALGO_STRASSEN | wt, 8)[0] == swmm.SW_EUNSUPPORTED
    assert swmm.sw_mm_workspace_size(64, 64, 64, 16, swmm.SW_ALGO_WINOGRAD | 0x4000, 8)[0] == swmm.SW_EINVAL
    for v in (swmm.SW_ALGO_WINOGRAD, swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_TWO_TEMP,
              swmm.SW_ALGO_WINOGRAD_KNUTH):
        assert swmm.sw_mm_workspace_size(256, 256, 256, 32, v | wt, 8) == swmm.sw_mm_workspace_size(256, 256, 256,
                                                                                                    32, v, 8)


@pytest.mark.parametrize("n,cutoff,top", [(4096, 256, 1), (4096, 128, 2), (8192, 128, 3)])
def test_deep_fp64_fused_workspace_is_table2_plus_one_bottom(lib, n, cutoff, top):
    # a deep FP64 FUSED product holds the Table 2 temporaries X, Y of its top levels (each
    # (n / 2^l)^2 FP64 at level l) plus the sum slots of one fused three-level bottom at a time
    v = swmm.SW_ALGO_WINOGRAD | swmm.SW_SCHED_FUSED
    assert swmm.sw_mm_depth(n, n, n, cutoff, v, 8) == (swmm.SW_OK, 3 + top)
    st, total = swmm.sw_mm_workspace_size(n, n, n, cutoff, v, 8)
    assert st == swmm.SW_OK
    s = n >> top
    st, bottom = swmm.sw_mm_workspace_size(s, s, s, s // 8, v, 8)
    assert st == swmm.SW_OK
    xy = sum(2 * (n >> l) ** 2 * 8 for l in range(1, top + 1))
    assert total == xy + bottom, (total, xy, bottom)
