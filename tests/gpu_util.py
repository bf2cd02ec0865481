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


def pixel_rel(F, Fref, floor=1e-3):
    """Largest relative error |F - Fref| / |Fref| over the pixels whose
    reference value is at least `floor` times the largest (the pixels that
    carry visible fluence)."""
    F = np.asarray(F, np.float64)
    Fref = np.asarray(Fref, np.float64)
    lit = (np.abs(Fref) >= floor * np.max(np.abs(Fref))) & (Fref != 0)
    if not lit.any():
        return 0.0
    return float(np.max(np.abs(F - Fref)[lit] / np.abs(Fref)[lit]))


def assert_fp32(F, Fref, tol=1e-4, rel=1e-5, msg=""):
    """The fp32 forward bounds: err_max <= 1e-4 and, pixel by pixel, a
    relative error <= 1e-5 wherever the fluence is at least 1e-3 of its
    maximum (so that a shadowed pixel cannot hide a large relative error
    behind the global normalisation)."""
    em, pr = err_max(F, Fref), pixel_rel(F, Fref)
    assert em <= tol and pr <= rel, f"{msg} err_max {em:.3e} (<= {tol}), pixel-relative {pr:.3e} (<= {rel})"
