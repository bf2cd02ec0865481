"""Helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def err_max(F, Fref):
    """max |F - Fref| / max |Fref| (0 when both vanish)."""
    F = np.asarray(F, np.float64)
    Fref = np.asarray(Fref, np.float64)
    den = np.max(np.abs(Fref))
    num = np.max(np.abs(F - Fref))
    return num / den if den > 0 else num


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()
