"""Per-channel extinction (sigma_t[C][H][W]): the CUDA path through the C
ABI against the FP64 oracle, with every feature that reads the extinction
(cross blur, bounces, environment map), forward and backward, staged and
unstaged channel planes (W H a multiple of 4 or not), and against the
shared-extinction path when the channels are equal.

Tolerances as for one shared extinction: fp32 max |diff| / max |ref|
<= 1e-4, fp64 <= 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, assert_fp32, to_dev, torch

pytestmark = pytest.mark.gpu


def _sigmas(e, s, seed):
    """Channel c: the scene's extinction scaled by a seeded factor, plus a
    seeded fog, so that the channels differ everywhere."""
    g = scenes.rng(seed)
    C = e.shape[0]
    return np.stack([s * g.uniform(0.3, 2.0) + g.uniform(0, 0.3, size=s.shape).astype(np.float32)
                     for _ in range(C)]).astype(np.float32)


@pytest.mark.parametrize("W,H,C,seed", [
    (16, 16, 3, 0), (37, 23, 2, 1), (5, 7, 1, 2), (1, 6, 2, 3), (64, 48, 3, 5), (100, 100, 4, 6), (33, 65, 3, 8),
])
def test_per_channel_forward_fp32_vs_oracle(W, H, C, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    S = _sigmas(e, s, 200 + seed)
    h = HRC(W, H, C)
    h.set_channel_extinction(True)
    F = h.forward(to_dev(e), to_dev(S)).cpu().numpy()
    assert_fp32(F, oracle.fluence(e, S))


def test_equal_channels_match_shared_extinction():
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(70, 50, 3, 9)
    h0 = HRC(70, 50, 3)
    F0 = h0.forward(to_dev(e), to_dev(s)).cpu().numpy()
    h = HRC(70, 50, 3)
    h.set_channel_extinction(True)
    F = h.forward(to_dev(e), to_dev(np.stack([s] * 3))).cpu().numpy()
    assert err_max(F, F0) <= 1e-6


@pytest.mark.parametrize("W,H,C,seed", [(16, 16, 2, 0), (37, 23, 3, 1)])
def test_per_channel_fp64_forward_and_backward(W, H, C, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = (x.astype(np.float64) for x in scenes.random_scene(W, H, C, seed))
    S = _sigmas(e, s, 210 + seed).astype(np.float64)
    g = scenes.rng(220 + seed).normal(size=e.shape)
    h = HRC(W, H, C, 0, "fp64")
    h.set_channel_extinction(True)
    F = h.forward(to_dev(e), to_dev(S)).cpu().numpy()
    assert err_max(F, oracle.fluence(e, S)) <= 1e-10
    ge, gs = (t.cpu().numpy() for t in h.backward(to_dev(g)))
    re, rs = oracle.fluence_adjoint(e, S, g)
    assert gs.shape == (C, H, W)
    assert err_max(ge, re) <= 1e-10 and err_max(gs, rs) <= 1e-10


@pytest.mark.parametrize("W,H,C,seed", [(16, 16, 3, 0), (37, 23, 2, 1), (64, 48, 3, 5)])
def test_per_channel_backward_fp32_vs_oracle(W, H, C, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    S = _sigmas(e, s, 230 + seed)
    g = scenes.rng(240 + seed).normal(size=e.shape).astype(np.float32)
    re, rs = oracle.fluence_adjoint(e, S, g)
    h = HRC(W, H, C)
    h.set_channel_extinction(True)
    for rc in (False, True):
        h.set_backward_recompute(rc)
        h.forward(to_dev(e), to_dev(S))
        ge, gs = (t.cpu().numpy() for t in h.backward(to_dev(g)))
        assert err_max(ge, re) <= 1e-4 and err_max(gs, rs) <= 1e-4, rc


def test_per_channel_with_blur_bounces_and_map():
    """The cross blur (channel c tests sigma_c), two bounces (source with
    sigma_c) and an environment map (row c for channel c), forward and
    backward, against the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    W, H, C = 37, 23, 2
    e, s = scenes.random_scene(W, H, C, 1)
    S = np.stack([s, np.float32(1.3) * s]).astype(np.float32)   # every opacity pair >= 6e-4 from the blur threshold
    a = scenes.rng(250).uniform(0, 0.9, size=e.shape).astype(np.float32)
    g = scenes.rng(251).normal(size=e.shape).astype(np.float32)
    env = scenes.rng(252).uniform(0, 2, size=(C, 12)).astype(np.float32)
    h = HRC(W, H, C)
    h.set_channel_extinction(True)
    h.set_cross_blur(True)
    h.reserve_bounces(2)
    F = h.forward_bounces(to_dev(e), to_dev(S), to_dev(a), 2).cpu().numpy()
    assert_fp32(F, oracle.fluence_bounces(e, S, a, 2, blur=0.5))
    ge, gs, ga = (t.cpu().numpy() for t in h.backward_bounces(to_dev(g)))
    re, rs, ra = oracle.fluence_bounces_adjoint(e, S, a, g, 2, blur=0.5)
    assert err_max(ge, re) <= 1e-4 and err_max(gs, rs) <= 1e-4 and err_max(ga, ra) <= 1e-4
    h.set_cross_blur(False)
    S2 = _sigmas(e, s, 253)
    h.set_environment(to_dev(env))
    F = h.forward(to_dev(e), to_dev(S2)).cpu().numpy()
    assert_fp32(F, oracle.fluence(e, S2, env=env))
    out = h.bounce_source(to_dev(e), to_dev(S2), to_dev(a), to_dev(F)).cpu().numpy()
    ref = oracle.bounce_source(e.astype(np.float64), S2.astype(np.float64), a.astype(np.float64), F.astype(np.float64))
    assert np.max(np.abs(out - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_per_channel_host_entry_autotune_and_level_export():
    require_gpu()
    from paper_2505_02041_gb300 import HRC, _lib
    e, s = scenes.random_scene(70, 50, 3, 16)
    S = _sigmas(e, s, 260)
    h = HRC(70, 50, 3)
    h.set_channel_extinction(True)
    h.autotune()
    Fh = h.forward_host(torch.from_numpy(e.copy()), torch.from_numpy(S.copy())).numpy()
    assert_fp32(Fh, oracle.fluence(e, S))
    with pytest.raises(_lib.HRCError) as ex:
        h.level(0, "T", 0)
    assert ex.value.status == _lib.HRC_ESTATE


def test_per_channel_full_size_workload():
    """The 1024^2 three-channel workload with a different extinction per
    channel, against the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.scene_by_name("volumetric1024")
    C, H, W = e.shape
    S = np.stack([s, 0.5 * s, 2.0 * s]).astype(np.float32)
    h = HRC(W, H, C)
    h.set_channel_extinction(True)
    h.autotune()
    F = h.forward(to_dev(e), to_dev(S)).cpu().numpy()
    assert_fp32(F, oracle.fluence(e, S))
