"""Cross blur (Sec. 4.2, Eq. 21 with opacity rejection): the CUDA path
through the C ABI against the FP64 oracle's blurred fluence and its adjoint.

The kept set of each pixel is an integer decision taken from floating
point (|a_m - a_c| <= threshold, a = 1 - exp(-sigma)); the GPU takes it in
the path's precision, the oracle in FP64.  Each fixture states the smallest
distance of any neighbour pair from the threshold in FP64: where it exceeds
1e-6 (fp32 rounding of a is below 1e-7) the two sides take the same
decisions and every pixel is compared; pixels with a pair closer than that
are checked to lie between the two outcomes instead.

Tolerances: as for the unblurred fluence (fp32: max |diff| / max |ref|
<= 1e-4; fp64: 1e-10), since the blur is a convex combination.
"""
import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, to_dev, torch

pytestmark = pytest.mark.gpu


def pair_margins(s, thr):
    """Per pixel: the smallest | |a_m - a_c| - thr | over its in-grid
    neighbours m (inf without neighbours)."""
    a = 1.0 - np.exp(-np.asarray(s, np.float64))
    H, W = a.shape
    m = np.full((H, W), np.inf)
    if W > 1:
        d = np.abs(np.abs(a[:, 1:] - a[:, :-1]) - thr)
        m[:, 1:] = np.minimum(m[:, 1:], d)
        m[:, :-1] = np.minimum(m[:, :-1], d)
    if H > 1:
        d = np.abs(np.abs(a[1:, :] - a[:-1, :]) - thr)
        m[1:, :] = np.minimum(m[1:, :], d)
        m[:-1, :] = np.minimum(m[:-1, :], d)
    return m


def check_blurred(Fg, e, s, thr, tol):
    """Compare the GPU's blurred fluence with the oracle's; near-tie pixels
    must lie between the outcomes of keeping and dropping their tie pairs."""
    Fr = oracle.fluence_blurred(e, s, thr)
    tie = pair_margins(s, thr) < 1e-6
    scale = np.max(np.abs(Fr))
    diff = np.abs(Fg - Fr)
    diff[:, tie] = 0.0
    assert (np.max(diff) / scale if scale > 0 else np.max(diff)) <= tol
    if np.any(tie):
        F0 = oracle.fluence(e, s)
        lo = oracle.cross_blur(F0, s, max(thr - 1e-6, 0.0))
        hi = oracle.cross_blur(F0, s, min(thr + 1e-6, 1.0))
        a, b = np.minimum(lo, hi), np.maximum(lo, hi)
        assert np.all(Fg[:, tie] >= a[:, tie] - tol * scale) and np.all(Fg[:, tie] <= b[:, tie] + tol * scale)


@pytest.mark.parametrize("W,H,C,seed,thr", [
    (16, 16, 1, 0, 0.5), (37, 23, 2, 1, 0.5), (5, 7, 1, 2, 0.5), (1, 6, 1, 3, 0.5), (6, 1, 1, 3, 0.5),
    (2, 2, 3, 4, 0.5), (64, 48, 3, 5, 0.5), (100, 100, 4, 6, 0.5), (33, 65, 1, 8, 0.5),
    (64, 48, 3, 5, 0.1), (64, 48, 3, 5, 1.0), (64, 48, 3, 5, 0.0),
])
def test_blurred_forward_fp32_vs_oracle(W, H, C, seed, thr):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    h = HRC(W, H, C)
    h.set_cross_blur(True, thr)
    assert h.cross_blur == (True, pytest.approx(thr))
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    check_blurred(F, e, s, thr, 1e-4)


def test_blurred_forward_disks64_and_toggle():
    """The 64^2 scene (emitters in vacuum, opaque boxes: every opacity pair
    is 0 or 1 apart), blurred, then with the blur switched off again: the
    unblurred fluence is bit-identical to a context that never blurred."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.scene_by_name("disks64")
    C, H, W = e.shape
    h = HRC(W, H, C)
    ed, sd = to_dev(e), to_dev(s)
    F0 = h.forward(ed, sd).clone()
    h.set_cross_blur(True)
    Fb = h.forward(ed, sd).cpu().numpy()
    check_blurred(Fb, e, s, 0.5, 1e-4)
    h.set_cross_blur(False)
    assert torch.equal(h.forward(ed, sd), F0)


@pytest.mark.parametrize("W,H,C,seed", [(16, 16, 1, 0), (37, 23, 2, 1), (5, 7, 1, 2)])
def test_blurred_forward_fp64_vs_oracle(W, H, C, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    h = HRC(W, H, C, 0, "fp64")
    h.set_cross_blur(True)
    F = h.forward(to_dev(e, torch.float64), to_dev(s, torch.float64)).cpu().numpy()
    check_blurred(F, e.astype(np.float64), s.astype(np.float64), 0.5, 1e-10)


@pytest.mark.parametrize("W,H,C,seed,prec,tol", [
    (16, 16, 1, 0, "fp32", 1e-4), (37, 23, 2, 1, "fp32", 1e-4), (64, 48, 3, 5, "fp32", 1e-4),
    (6, 1, 1, 3, "fp32", 1e-4), (37, 23, 2, 1, "fp64", 1e-10),
])
def test_blurred_backward_vs_oracle(W, H, C, seed, prec, tol):
    """dL/de and dL/dsigma of sum(gF * blurred F) against the oracle (whose
    fixtures keep every pair at least 1e-5 from the threshold, so both sides
    hold the same kept sets)."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    assert np.min(pair_margins(s, 0.5)) > 1e-5
    dt = torch.float64 if prec == "fp64" else torch.float32
    gF = scenes.rng(3000 + seed).normal(size=e.shape)
    h = HRC(W, H, C, 0, prec)
    h.set_cross_blur(True)
    h.forward(to_dev(e, dt), to_dev(s, dt))
    ge, gs = h.backward(to_dev(gF, dt))
    ge_r, gs_r = oracle.fluence_blurred_adjoint(e, s, gF if prec == "fp64" else gF.astype(np.float32))
    assert err_max(ge.cpu().numpy(), ge_r) <= tol
    assert err_max(gs.cpu().numpy(), gs_r) <= tol


def test_blurred_backward_fp64_central_differences():
    """GPU FP64 adjoint of the blurred fluence against central differences
    of the GPU FP64 forward (h = 1e-3): e exactly (F is linear in e), sigma
    at pixels whose pairs sit at least 1e-2 from the threshold."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(48, 40, 2, 9)
    e = e.astype(np.float64)
    s = s.astype(np.float64)
    gF = scenes.rng(9).normal(size=e.shape)
    h = HRC(48, 40, 2, 0, "fp64")
    h.set_cross_blur(True)
    ed, sd, gd = to_dev(e), to_dev(s), to_dev(gF)
    h.forward(ed, sd)
    ge, gs = (t.cpu().numpy() for t in h.backward(gd))

    def loss(ee, ss):
        return float(torch.sum(gd * h.forward(ee, ss)))

    marg = pair_margins(s, 0.5)
    pix = scenes.rng(10).integers(0, [40, 48], size=(24, 2))
    hs = 1e-3
    checked = 0
    for (y, x) in pix:
        ep, em = ed.clone(), ed.clone()
        ep[1, y, x] += hs
        em[1, y, x] -= hs
        fd = (loss(ep, sd) - loss(em, sd)) / (2 * hs)
        assert abs(fd - ge[1, y, x]) <= 1e-8 * max(1.0, abs(fd))
        if marg[y, x] < 1e-2:
            continue
        sp, sm = sd.clone(), sd.clone()
        sp[y, x] += hs
        sm[y, x] -= hs
        fd = (loss(ed, sp) - loss(ed, sm)) / (2 * hs)
        assert abs(fd - gs[y, x]) <= 1e-5 * max(1.0, abs(fd))
        checked += 1
    assert checked >= 12


def test_blurred_autograd_and_host_entry():
    """The autograd function and the host-buffer entry apply the blur too."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, fluence
    e, s = scenes.random_scene(40, 30, 2, 11)
    assert np.min(pair_margins(s, 0.5)) > 1e-5
    h = HRC(40, 30, 2)
    h.set_cross_blur(True)
    et = to_dev(e).requires_grad_(True)
    st = to_dev(s).requires_grad_(True)
    w = torch.randn((2, 30, 40), device="cuda")
    (fluence(h, et, st) * w).sum().backward()
    ge_r, gs_r = oracle.fluence_blurred_adjoint(e, s, w.cpu().numpy())
    assert err_max(et.grad.cpu().numpy(), ge_r) <= 1e-4
    assert err_max(st.grad.cpu().numpy(), gs_r) <= 1e-4
    Fh = h.forward_host(torch.from_numpy(e.copy()), torch.from_numpy(s.copy()))
    check_blurred(Fh.numpy(), e, s, 0.5, 1e-4)


def test_blurred_full_size_workload():
    """The 1024^2 three-channel workload with the blur, in the autotuned
    launch configuration, against the oracle at every pixel."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.scene_by_name("volumetric1024")
    C, H, W = e.shape
    h = HRC(W, H, C)
    h.autotune()
    h.set_cross_blur(True)
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    check_blurred(F, e, s, 0.5, 1e-4)


def test_cross_blur_argument_errors():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, BatchedHRC, _lib
    h = HRC(8, 8, 1)
    for en, th in ((2, 0.5), (-1, 0.5), (1, -0.1), (1, 1.5), (1, float("nan"))):
        assert _lib.load().hrc_set_cross_blur(h.ctx, en, th) == _lib.HRC_EINVAL
    assert h.cross_blur == (False, pytest.approx(0.5))
    b = BatchedHRC([(8, 8), (4, 4)], 1)
    with pytest.raises(_lib.HRCError) as ex:
        _lib.hrc_set_cross_blur(b.ctx, True, 0.5)
    assert ex.value.status == _lib.HRC_EINVAL
