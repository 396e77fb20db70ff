"""The allocation-free curve-order entry point, for callers that cannot call
cudaMalloc (stream capture, externally pooled device memory, latency-critical
code).  It must return exactly what the allocating path returns: the Hilbert
keys by lexicographic id and the curve-order permutation, bit for bit.

Collected last on purpose (file name), so a run that stops at the first failure
has already run every other test.
"""
import ctypes as C

import pytest
import torch

from paper_2110_11211_gb300 import _lib

pytestmark = pytest.mark.gpu

CASES = [((10, 5, 3), 128, 1.0), ((5, 4, 3, 3, 2, 2), 256, 0.25)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11211_gb300.build import build
    build()


def noalloc_curve(levels):
    L = _lib.lib()
    n = 1
    for l in levels:
        n *= (1 << l) - 1
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    lv = (C.c_int * len(levels))(*levels)
    rc = L.sfcdd_curve_order_noalloc(lv, len(levels), keys.data_ptr(), perm.data_ptr(),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, keys, perm


def test_two_calls_in_a_row_match_the_allocating_path():
    from paper_2110_11211_gb300.solver import Solver
    got = [noalloc_curve(levels) for levels, _, _ in CASES]   # two calls, shared scratch
    for (levels, P, gamma), (rc, keys, perm) in zip(CASES, got):
        assert rc == 0
        with Solver(levels, P, gamma, variant="coarse_only", q=1) as s:
            ref_keys, ref_perm = s.curve()
        assert torch.equal(keys, ref_keys)
        assert torch.equal(perm, ref_perm)


def test_rejects_grids_beyond_the_scratch_limit():
    rc, _, _ = noalloc_curve((10, 10))      # 1,046,529 points > 262,144
    assert rc == -1


def test_rejects_oversized_levels_before_counting_points():
    # d * max l > 64 -> KEY_OVERFLOW; sum l > 31 -> UNSUPPORTED; both before the
    # point count is formed (no overflow for levels up to 30 on every axis)
    for levels, code in [((30,) * 6, -2), ((30, 30), -9), ((16, 16), -9)]:
        rc, _, _ = noalloc_curve_args(levels)
        assert rc == code, (levels, rc)


def noalloc_curve_args(levels):
    L = _lib.lib()
    keys = torch.empty(1, dtype=torch.int64, device="cuda")
    perm = torch.empty(1, dtype=torch.int32, device="cuda")
    lv = (C.c_int * len(levels))(*levels)
    rc = L.sfcdd_curve_order_noalloc(lv, len(levels), keys.data_ptr(), perm.data_ptr(),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, keys, perm
