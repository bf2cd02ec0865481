"""End-to-end use of the adjoint and the optional steps.

* Inverse rendering: recover the emission of a scene from its blurred
  fluence (the paper's full Lighting with the Eq. 21 blur) by gradient
  descent through the autograd function, on the GPU path alone; the fluence
  is linear in e, so the loss must fall by orders of magnitude.
* The optional steps in the reduced-precision storage modes, against the
  FP64 oracle within the bounds stated for those modes.
"""
import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, to_dev, torch

pytestmark = pytest.mark.gpu


def test_inverse_rendering_recovers_emission():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, fluence
    e_true, s = scenes.random_scene(48, 40, 2, 300)
    h = HRC(48, 40, 2)
    h.set_cross_blur(True)
    sd = to_dev(s)
    target = fluence(h, to_dev(e_true), sd).detach().clone()
    e = torch.full_like(target, float(e_true.mean())).requires_grad_(True)
    opt = torch.optim.Adam([e], lr=0.05)
    sched = torch.optim.lr_scheduler.StepLR(opt, step_size=100, gamma=0.3)
    losses = []
    for _ in range(300):
        opt.zero_grad()
        loss = torch.mean((fluence(h, e, sd) - target) ** 2)
        loss.backward()
        opt.step()
        sched.step()
        with torch.no_grad():
            e.clamp_(min=0.0)
        losses.append(loss.item())
    # a hundredfold drop: well past what a wrong gradient (sign, scale or
    # missing blur transpose) would allow on this linear least-squares problem
    assert losses[-1] <= 1e-2 * losses[0], (losses[0], losses[-1])
    # the recovered emission reproduces the target fluence (the oracle agrees)
    F = oracle.fluence_blurred(e.detach().cpu().numpy(), s)
    assert err_max(F, target.cpu().numpy()) <= 5e-2


@pytest.mark.parametrize("prec,tol", [("fp16", 1e-3), ("bf16", 6e-3)])
def test_optional_steps_in_reduced_precision(prec, tol):
    """Cross blur, two bounces and per-channel extinction with fp16 / bf16
    interval storage, forward against the FP64 oracle within the modes'
    stated bounds, and the bounce adjoint within four times those."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(37, 23, 2, 1)
    a = scenes.rng(301).uniform(0, 0.9, size=e.shape).astype(np.float32)
    g = scenes.rng(302).normal(size=e.shape).astype(np.float32)
    h = HRC(37, 23, 2, 0, prec)
    h.set_cross_blur(True)
    assert err_max(h.forward(to_dev(e), to_dev(s)).cpu().numpy(), oracle.fluence_blurred(e, s)) <= tol
    h.reserve_bounces(2)
    F = h.forward_bounces(to_dev(e), to_dev(s), to_dev(a), 2).cpu().numpy()
    assert err_max(F, oracle.fluence_bounces(e, s, a, 2, blur=0.5)) <= tol
    ge, gs, ga = (t.cpu().numpy() for t in h.backward_bounces(to_dev(g)))
    re, rs, ra = oracle.fluence_bounces_adjoint(e, s, a, g, 2, blur=0.5)
    assert err_max(ge, re) <= 4 * tol and err_max(ga, ra) <= 4 * tol and err_max(gs, rs) <= 4 * tol
    h.set_cross_blur(False)
    S = np.stack([s, np.float32(1.3) * s]).astype(np.float32)
    h.set_channel_extinction(True)
    assert err_max(h.forward(to_dev(e), to_dev(S)).cpu().numpy(), oracle.fluence(e, S)) <= tol
