"""Adjoint parity: CUDA backward (through the C ABI) vs the FP64 oracle's
adjoint, and the GPU FP64 instance vs FP64 central differences.

Tolerances:
  * fp32 GPU adjoint vs FP64 oracle adjoint: max |diff| / max |grad| <= 1e-4
  * fp64 GPU adjoint vs FP64 oracle adjoint: <= 1e-10
  * fp64 GPU adjoint vs central differences (h = 1e-3): e-gradient <= 1e-7
    relative (F is linear in e), sigma-gradient <= 1e-5 relative (O(h^2)).
"""
import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, to_dev, torch

pytestmark = pytest.mark.gpu


def _gpu_grads(e, s, gF, precision="fp32", cascades=0):
    from paper_2505_02041_gb300 import HRC
    C, H, W = e.shape
    h = HRC(W, H, C, cascades, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    ed, sd = to_dev(e, dt), to_dev(s, dt)
    h.forward(ed, sd)
    ge, gs = h.backward(to_dev(gF, dt))
    torch.cuda.synchronize()
    return ge.cpu().numpy(), gs.cpu().numpy()


@pytest.mark.parametrize("W,H,C,casc,seed", [
    (16, 16, 1, 0, 0), (37, 23, 2, 0, 1), (5, 7, 1, 0, 2), (1, 6, 1, 0, 3), (2, 2, 3, 0, 4),
    (64, 48, 3, 0, 5), (100, 100, 4, 0, 6), (64, 64, 1, 3, 7), (33, 65, 1, 0, 8),
])
def test_backward_fp32_vs_oracle(W, H, C, casc, seed):
    require_gpu()
    e, s = scenes.random_scene(W, H, C, seed)
    gF = scenes.rng(1000 + seed).normal(size=e.shape).astype(np.float32)
    ge, gs = _gpu_grads(e, s, gF, "fp32", casc)
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF, casc)
    assert err_max(ge, ge_r) <= 1e-4
    assert err_max(gs, gs_r) <= 1e-4


def test_backward_fp32_disks64_scene():
    require_gpu()
    e, s = scenes.scene_by_name("disks64")
    gF = scenes.rng(5).normal(size=e.shape).astype(np.float32)
    ge, gs = _gpu_grads(e, s, gF)
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF)
    assert err_max(ge, ge_r) <= 1e-4
    assert err_max(gs, gs_r) <= 1e-4


@pytest.mark.parametrize("W,H,C,seed", [(16, 16, 1, 0), (37, 23, 2, 1), (64, 48, 3, 2)])
def test_backward_fp64_vs_oracle(W, H, C, seed):
    require_gpu()
    e, s = scenes.random_scene(W, H, C, seed)
    gF = scenes.rng(2000 + seed).normal(size=e.shape)
    ge, gs = _gpu_grads(e.astype(np.float64), s.astype(np.float64), gF, "fp64")
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF)
    assert err_max(ge, ge_r) <= 1e-10
    assert err_max(gs, gs_r) <= 1e-10


def test_backward_fp64_central_differences_256():
    """Differentiable HRC on 256x256, C=1, the whole batch of 16 scenes
    (seeds 100+b, fog/disks/rectangles with C=1): loss ||F(e, s) - F_target||^2
    with F_target from a hidden scene (seed 1000+b); the backward recomputes
    every cascade level from the inputs (hrc_set_backward_recompute); adjoint
    vs FP64 central differences (h = 1e-3) at 64 seeded pixels per scene."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    h = HRC(256, 256, 1, 0, "fp64")
    h.set_backward_recompute(True)
    pix = scenes.rng(7).integers(0, 256, size=(64, 2))
    for b in range(16):
        e, s = scenes.scene_disks_rects_fog(256, 256, 1, 100 + b)
        et, _ = scenes.scene_disks_rects_fog(256, 256, 1, 1000 + b)
        ed, sd = to_dev(e, torch.float64), to_dev(s, torch.float64)
        Ft = h.forward(to_dev(et, torch.float64), sd).clone()
        F = h.forward(ed, sd)
        gF = 2.0 * (F - Ft)
        ge, gs = h.backward(gF.contiguous(), ed, sd)
        ge, gs = ge.cpu().numpy(), gs.cpu().numpy()

        hstep = 1e-3
        eps = np.finfo(np.float64).eps

        def central(ep, sp, em, sm):
            """(loss(+) - loss(-)) / 2h formed pixel by pixel as
            sum (F+ - F-)(F+ + F- - 2 F_t) / 2h, which avoids cancelling two
            large sums; with the rounding floor of that form."""
            Fp = h.forward(ep, sp).clone()
            Fm = h.forward(em, sm)
            fd = float(torch.sum((Fp - Fm) * (Fp + Fm - 2 * Ft))) / (2 * hstep)
            floor = 64 * eps * float(torch.sum((Fp.abs() + Fm.abs()) * (Fp + Fm - 2 * Ft).abs())) / (2 * hstep)
            return fd, floor

        for (y, x) in pix:
            ep, em = ed.clone(), ed.clone()
            ep[0, y, x] += hstep
            em[0, y, x] -= hstep
            fd, floor = central(ep, sd, em, sd)
            assert abs(fd - ge[0, y, x]) <= 1e-7 * abs(fd) + floor, (b, y, x, fd, ge[0, y, x], floor)
            sp, sm = sd.clone(), sd.clone()
            sp[y, x] += hstep
            sm[y, x] -= hstep
            fd, floor = central(ed, sp, ed, sm)
            assert abs(fd - gs[y, x]) <= 1e-5 * abs(fd) + floor, (b, y, x, fd, gs[y, x], floor)


def test_autograd_function_matches_abi():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, fluence
    e, s = scenes.random_scene(40, 30, 2, 9)
    h = HRC(40, 30, 2)
    et = to_dev(e).requires_grad_(True)
    st = to_dev(s).requires_grad_(True)
    w = torch.randn((2, 30, 40), device="cuda")
    (fluence(h, et, st) * w).sum().backward()
    ge_r, gs_r = oracle.fluence_adjoint(e, s, w.cpu().numpy())
    assert err_max(et.grad.cpu().numpy(), ge_r) <= 1e-4
    assert err_max(st.grad.cpu().numpy(), gs_r) <= 1e-4


def test_backward_before_forward_is_a_state_error():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    h = HRC(8, 8, 1)
    g = torch.zeros((1, 8, 8), device="cuda")
    with pytest.raises(_lib.HRCError) as ex:
        h.backward(g)
    assert ex.value.status == _lib.HRC_ESTATE


def test_backward_reuses_levels_and_tracks_in_place_changes():
    """The backward reads the levels the forward left in the context: two
    backward calls in a row (another dL/dF, no forward between) each match
    the oracle, and an input modified in place since the forward makes the
    Python binding run the forward again, so the gradient is the one at the
    new inputs."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(45, 38, 2, 21)
    g1 = scenes.rng(31).normal(size=e.shape).astype(np.float32)
    g2 = scenes.rng(32).normal(size=e.shape).astype(np.float32)
    h = HRC(45, 38, 2)
    ed, sd = to_dev(e), to_dev(s)
    h.forward(ed, sd)
    for g in (g1, g2):
        ge, gs = h.backward(to_dev(g))
        ge_r, gs_r = oracle.fluence_adjoint(e, s, g)
        assert err_max(ge.cpu().numpy(), ge_r) <= 1e-4
        assert err_max(gs.cpu().numpy(), gs_r) <= 1e-4
    sd.mul_(1.7)                       # in place: same storage, new version
    ge, gs = h.backward(to_dev(g1), ed, sd)
    ge_r, gs_r = oracle.fluence_adjoint(e, s * np.float32(1.7), g1)
    assert err_max(ge.cpu().numpy(), ge_r) <= 1e-4
    assert err_max(gs.cpu().numpy(), gs_r) <= 1e-4


@pytest.mark.parametrize("W,H,C,seed", [(37, 23, 2, 41), (64, 64, 3, 42)])
def test_backward_recompute_mode(W, H, C, seed):
    """With hrc_set_backward_recompute the backward recomputes every level from
    the inputs: it matches the oracle adjoint and the level-reading backward,
    and, relying on no forward-time storage, it differentiates at the
    borrowed inputs' current contents even after they changed in place
    (called through the C ABI, so no forward runs in between)."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(W, H, C, seed)
    gF = scenes.rng(seed + 100).normal(size=e.shape).astype(np.float32)
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF)
    h = HRC(W, H, C)
    ed, sd, gd = to_dev(e), to_dev(s), to_dev(gF)
    h.forward(ed, sd)
    ge0, gs0 = (t.cpu().numpy() for t in h.backward(gd))
    h.set_backward_recompute(True)
    ge1, gs1 = (t.cpu().numpy() for t in h.backward(gd))
    assert err_max(ge1, ge_r) <= 1e-4 and err_max(gs1, gs_r) <= 1e-4
    assert np.max(np.abs(ge1 - ge0)) <= 1e-6 * np.max(np.abs(ge0))
    assert np.max(np.abs(gs1 - gs0)) <= 1e-6 * np.max(np.abs(gs0))
    sd.mul_(1.7)
    ge2 = torch.empty_like(ed)
    gs2 = torch.empty_like(sd)
    _lib.hrc_fluence_backward(h.ctx, gd, ge2, gs2)
    ge_r2, gs_r2 = oracle.fluence_adjoint(e, s * np.float32(1.7), gF)
    assert err_max(ge2.cpu().numpy(), ge_r2) <= 1e-4 and err_max(gs2.cpu().numpy(), gs_r2) <= 1e-4
