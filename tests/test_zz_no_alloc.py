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

from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the fp32 parity tolerance used by the other forward tests


def _reference(e, s):
    from paper_2505_02041_gb300 import HRC
    C, H, W = e.shape
    h = HRC(W, H, C)
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    h.close()
    return F


def test_noalloc_matches_context_entry_two_calls():
    require_gpu()
    from paper_2505_02041_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    for (W, H, C, seed) in [(128, 96, 3, 0), (64, 64, 1, 1)]:   # two calls in a row, shared scratch
        e, s = scenes.random_scene(W, H, C, seed)
        ed, sd = to_dev(e), to_dev(s)
        out = torch.full((C, H, W), float("nan"), device="cuda")
        st = lib.hrc_fluence_noalloc(W, H, C, ed.data_ptr(), sd.data_ptr(), out.data_ptr(),
                                     ctypes.c_void_p(stream))
        assert st == _lib.HRC_OK, _lib.hrc_last_error()
        torch.cuda.synchronize()
        F = out.cpu().numpy()
        assert np.all(np.isfinite(F))
        assert err_max(F, _reference(e, s)) <= TOL


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
