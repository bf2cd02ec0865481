"""The allocation-free forward entry point (hrc_fluence_noalloc).

It serves callers that cannot call cudaMalloc (an engine-owned memory
budget, a host framework that must own every device allocation, a plugin
forbidden to allocate after start-up): every intermediate level lives in a
fixed device array inside the library.  This file is collected last so a
run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, assert_fp32, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the fp32 parity tolerance used by the other forward tests


def _reference(e, s):
    from paper_2505_02041_gb300 import HRC
    C, H, W = e.shape
    h = HRC(W, H, C)
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    h.close()
    return F


def _noalloc(lib, e, s, stream):
    from paper_2505_02041_gb300 import _lib
    C, H, W = e.shape
    ed, sd = to_dev(e), to_dev(s)
    out = torch.full((C, H, W), float("nan"), device="cuda")
    st = lib.hrc_fluence_noalloc(W, H, C, ed.data_ptr(), sd.data_ptr(), out.data_ptr(), ctypes.c_void_p(stream))
    assert st == _lib.HRC_OK, _lib.hrc_last_error()
    assert lib.hrc_noalloc_sync(ctypes.c_void_p(stream)) == _lib.HRC_OK, _lib.hrc_last_error()
    return out.cpu().numpy()


def test_noalloc_matches_context_entry_two_calls():
    require_gpu()
    from paper_2505_02041_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row share the scratch; the largest accepted grid
    # (128 x 128, C = 4: the layout must fill the fixed array exactly) and
    # the smallest (1 x 1) included
    for (W, H, C, seed) in [(128, 96, 3, 0), (64, 64, 1, 1), (128, 128, 4, 2), (1, 1, 1, 3)]:
        e, s = scenes.random_scene(W, H, C, seed)
        F = _noalloc(lib, e, s, stream)
        assert np.all(np.isfinite(F))
        assert_fp32(F, _reference(e, s))
        assert_fp32(F, oracle.fluence(e, s))


def test_noalloc_copy_wait_timeout_is_reported():
    """A copy wait of the no-alloc path that gives up is reported by
    hrc_noalloc_sync (the path's own status word, not a context's); the
    next call computes correctly again."""
    require_gpu()
    from paper_2505_02041_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    e, s = scenes.random_scene(128, 96, 2, 4)          # W a multiple of 4: the trace stages by TMA
    ed, sd = to_dev(e), to_dev(s)
    out = torch.zeros((2, 96, 128), device="cuda")
    assert lib.hrc_noalloc_debug_wait(16, 1_000_000) == _lib.HRC_OK
    try:
        st = lib.hrc_fluence_noalloc(128, 96, 2, ed.data_ptr(), sd.data_ptr(), out.data_ptr(),
                                     ctypes.c_void_p(stream))
        assert st == _lib.HRC_OK
        assert lib.hrc_noalloc_sync(ctypes.c_void_p(stream)) == _lib.HRC_ETIMEOUT
    finally:
        assert lib.hrc_noalloc_debug_wait(0, 0) == _lib.HRC_OK
    F = _noalloc(lib, e, s, stream)
    assert_fp32(F, oracle.fluence(e, s))


def test_noalloc_rejects_oversize_grid():
    require_gpu()
    from paper_2505_02041_gb300 import _lib
    lib = _lib.load()
    e = torch.zeros((1, 8, 129), device="cuda")
    s = torch.zeros((8, 129), device="cuda")
    out = torch.zeros((1, 8, 129), device="cuda")
    st = lib.hrc_fluence_noalloc(129, 8, 1, e.data_ptr(), s.data_ptr(), out.data_ptr(), None)
    assert st == _lib.HRC_EINVAL
    assert "128" in _lib.hrc_last_error()
