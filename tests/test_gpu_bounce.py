"""Multiple bounces (Sec. 4.2: the output fluence fed back as a scattering
source, e_{k+1} = e + albedo * sigma * F_k / (2 pi)): the CUDA path through
the C ABI against the FP64 oracle's iteration and its adjoint, the
uniform-medium closed form, and FP64 central differences.

Tolerances: fp32 max |diff| / max |ref| <= 1e-4 for the fluence and every
gradient (as for one bounce: each bounce is one more pass of the same
kernels on a source of the same scale); fp64 <= 1e-10.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, assert_fp32, to_dev, torch

pytestmark = pytest.mark.gpu


def _albedo(shape, seed):
    return scenes.rng(seed).uniform(0.0, 0.9, size=shape).astype(np.float32)


@pytest.mark.parametrize("W,H,C,K,seed", [
    (16, 16, 1, 1, 0), (37, 23, 2, 2, 1), (5, 7, 1, 3, 2), (1, 6, 1, 2, 3), (64, 48, 3, 6, 5),
    (100, 100, 4, 2, 6), (33, 65, 1, 0, 8),
])
def test_bounces_forward_fp32_vs_oracle(W, H, C, K, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    a = _albedo(e.shape, 50 + seed)
    h = HRC(W, H, C)
    h.reserve_bounces(6)
    F = h.forward_bounces(to_dev(e), to_dev(s), to_dev(a), K).cpu().numpy()
    assert_fp32(F, oracle.fluence_bounces(e, s, a, K))


def test_bounces_uniform_medium_closed_form():
    """Deep inside a thick uniform medium (sigma = 50, 64^2): K bounces give
    2 pi c (1 - rho^(K+1)) / (1 - rho) (the partial Neumann sum of the
    transfer solution with scattering), independently of the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    X, sg, c, rho = 64, 50.0, 1.3, 0.7
    h = HRC(X, X, 1)
    h.reserve_bounces(6)
    e = torch.full((1, X, X), sg * c, device="cuda")
    s = torch.full((X, X), sg, device="cuda")
    a = torch.full((1, X, X), rho, device="cuda")
    for K in (0, 1, 3, 6):
        F = h.forward_bounces(e, s, a, K).cpu().numpy()
        want = 2 * math.pi * c * (1 - rho ** (K + 1)) / (1 - rho)
        assert np.max(np.abs(F[0, 28:36, 28:36] - want)) <= 1e-5 * want, K


@pytest.mark.parametrize("W,H,C,K,seed", [(16, 16, 1, 1, 0), (37, 23, 2, 2, 1)])
def test_bounces_forward_fp64_vs_oracle(W, H, C, K, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = (x.astype(np.float64) for x in scenes.random_scene(W, H, C, seed))
    a = _albedo(e.shape, 60 + seed).astype(np.float64)
    h = HRC(W, H, C, 0, "fp64")
    h.reserve_bounces(K)
    F = h.forward_bounces(to_dev(e), to_dev(s), to_dev(a), K).cpu().numpy()
    assert err_max(F, oracle.fluence_bounces(e, s, a, K)) <= 1e-10


@pytest.mark.parametrize("W,H,C,K,seed,prec,tol", [
    (16, 16, 1, 1, 0, "fp32", 1e-4), (37, 23, 2, 2, 1, "fp32", 1e-4), (64, 48, 3, 3, 5, "fp32", 1e-4),
    (1, 6, 1, 2, 3, "fp32", 1e-4), (20, 12, 2, 0, 4, "fp32", 1e-4), (37, 23, 2, 2, 1, "fp64", 1e-10),
])
def test_bounces_backward_vs_oracle(W, H, C, K, seed, prec, tol):
    """dL/de, dL/dsigma, dL/dalbedo; two backward calls in a row (the second
    recomputes the last bounce's levels, which the first overwrote)."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    a = _albedo(e.shape, 70 + seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp64":
        e, s, a = (x.astype(np.float64) for x in (e, s, a))
    g1 = scenes.rng(80 + seed).normal(size=e.shape)
    g2 = scenes.rng(90 + seed).normal(size=e.shape)
    if prec == "fp32":
        g1, g2 = g1.astype(np.float32), g2.astype(np.float32)
    h = HRC(W, H, C, 0, prec)
    h.reserve_bounces(4)
    h.forward_bounces(to_dev(e, dt), to_dev(s, dt), to_dev(a, dt), K)
    for g in (g1, g2):
        ge, gs, ga = (t.cpu().numpy() for t in h.backward_bounces(to_dev(g, dt)))
        re, rs, ra = oracle.fluence_bounces_adjoint(e, s, a, g, K)
        assert err_max(ge, re) <= tol
        assert err_max(gs, rs) <= tol
        if K > 0:
            assert err_max(ga, ra) <= tol
        else:
            assert not np.any(ga)


def test_bounces_with_cross_blur_vs_oracle():
    """Every bounce blurred (the fixture keeps every opacity pair at least
    1e-4 from the threshold): forward and backward."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(37, 23, 2, 1)
    a = _albedo(e.shape, 71)
    g = scenes.rng(81).normal(size=e.shape).astype(np.float32)
    h = HRC(37, 23, 2)
    h.reserve_bounces(2)
    h.set_cross_blur(True)
    F = h.forward_bounces(to_dev(e), to_dev(s), to_dev(a), 2).cpu().numpy()
    assert_fp32(F, oracle.fluence_bounces(e, s, a, 2, blur=0.5))
    ge, gs, ga = (t.cpu().numpy() for t in h.backward_bounces(to_dev(g)))
    re, rs, ra = oracle.fluence_bounces_adjoint(e, s, a, g, 2, blur=0.5)
    assert err_max(ge, re) <= 1e-4 and err_max(gs, rs) <= 1e-4 and err_max(ga, ra) <= 1e-4


def test_bounces_fp64_central_differences():
    """GPU FP64 adjoint against central differences of the GPU FP64 bounce
    forward (h = 1e-4) in e, sigma and albedo."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = (x.astype(np.float64) for x in scenes.random_scene(30, 26, 2, 12))
    a = _albedo(e.shape, 13).astype(np.float64)
    g = scenes.rng(14).normal(size=e.shape)
    K = 3
    h = HRC(30, 26, 2, 0, "fp64")
    h.reserve_bounces(K)
    ed, sd, ad, gd = to_dev(e), to_dev(s), to_dev(a), to_dev(g)
    h.forward_bounces(ed, sd, ad, K)
    ge, gs, ga = (t.cpu().numpy() for t in h.backward_bounces(gd))

    def loss(ee, ss, aa):
        return float(torch.sum(gd * h.forward_bounces(ee, ss, aa, K)))

    hs = 1e-4
    for (y, x) in scenes.rng(15).integers(0, [26, 30], size=(8, 2)):
        for which, got in (("e", ge[1, y, x]), ("s", gs[y, x]), ("a", ga[0, y, x])):
            p = [ed.clone(), sd.clone(), ad.clone()]
            m = [ed.clone(), sd.clone(), ad.clone()]
            if which == "e":
                p[0][1, y, x] += hs
                m[0][1, y, x] -= hs
            elif which == "s":
                p[1][y, x] += hs
                m[1][y, x] -= hs
            else:
                p[2][0, y, x] += hs
                m[2][0, y, x] -= hs
            fd = (loss(*p) - loss(*m)) / (2 * hs)
            assert abs(fd - got) <= 1e-6 * max(1.0, abs(fd)), (which, y, x, fd, got)


def test_bounces_autograd_function():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, fluence_bounces
    e, s = scenes.random_scene(40, 30, 2, 16)
    a = _albedo(e.shape, 17)
    h = HRC(40, 30, 2)
    h.reserve_bounces(2)
    et, st, at = (to_dev(x).requires_grad_(True) for x in (e, s, a))
    w = torch.randn((2, 30, 40), device="cuda")
    (fluence_bounces(h, et, st, at, 2) * w).sum().backward()
    re, rs, ra = oracle.fluence_bounces_adjoint(e, s, a, w.cpu().numpy(), 2)
    assert err_max(et.grad.cpu().numpy(), re) <= 1e-4
    assert err_max(st.grad.cpu().numpy(), rs) <= 1e-4
    assert err_max(at.grad.cpu().numpy(), ra) <= 1e-4


@pytest.mark.parametrize("W,H", [(64, 48), (37, 23)])
def test_bounce_source_elementwise(W, H):
    """hrc_bounce_source (one bounce per frame) on the 4-wide (W H % 4 == 0)
    and scalar paths."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, 3, 18)
    a = _albedo(e.shape, 19)
    F = scenes.rng(20).uniform(0, 10, size=e.shape).astype(np.float32)
    h = HRC(W, H, 3)
    out = h.bounce_source(to_dev(e), to_dev(s), to_dev(a), to_dev(F)).cpu().numpy()
    ref = oracle.bounce_source(e.astype(np.float64), s.astype(np.float64), a.astype(np.float64), F.astype(np.float64))
    assert np.max(np.abs(out - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_bounce_state_and_argument_errors():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(8, 8, 1, 21)
    a = _albedo(e.shape, 22)
    ed, sd, ad = to_dev(e), to_dev(s), to_dev(a)
    h = HRC(8, 8, 1)
    out = torch.empty_like(ed)
    with pytest.raises(_lib.HRCError) as ex:                 # no reservation
        _lib.hrc_fluence_bounces(h.ctx, ed, sd, ad, 1, out)
    assert ex.value.status == _lib.HRC_ESTATE
    h.reserve_bounces(2)
    with pytest.raises(_lib.HRCError) as ex:                 # more than reserved
        _lib.hrc_fluence_bounces(h.ctx, ed, sd, ad, 3, out)
    assert ex.value.status == _lib.HRC_EINVAL
    g = torch.ones_like(ed)
    with pytest.raises(_lib.HRCError) as ex:                 # no bounce forward yet
        h.backward_bounces(g)
    assert ex.value.status == _lib.HRC_ESTATE
    h.forward_bounces(ed, sd, ad, 2)
    with pytest.raises(_lib.HRCError) as ex:                 # plain backward after a bounce forward
        _lib.hrc_fluence_backward(h.ctx, g, torch.empty_like(ed), torch.empty_like(sd))
    assert ex.value.status == _lib.HRC_ESTATE
    h.forward(ed, sd)
    with pytest.raises(_lib.HRCError) as ex:                 # bounce backward after a plain forward
        h.backward_bounces(g)
    assert ex.value.status == _lib.HRC_ESTATE


def test_bounces_full_size_workload():
    """The 1024^2 three-channel workload with six bounces (the count of the
    paper's Fig. 14), albedo 0.5 everywhere, against the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.scene_by_name("volumetric1024")
    C, H, W = e.shape
    a = np.full(e.shape, 0.5, np.float32)
    h = HRC(W, H, C)
    h.autotune()
    h.reserve_bounces(6)
    F = h.forward_bounces(to_dev(e), to_dev(s), to_dev(a), 6).cpu().numpy()
    assert_fp32(F, oracle.fluence_bounces(e, s, a, 6))
