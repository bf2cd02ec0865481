"""Environment map (footnote 1 of Sec. 4.2: R_N looked up along v_N(i), and
out-of-grid R lookups as the recursion continued through vacuum): the CUDA
path through the C ABI against the FP64 oracle, in every launch
configuration, forward and backward, plus the one-sided-light check that
fixes the look-direction convention without the oracle.

Tolerances as for the fluence without a map: fp32 max |diff| / max |ref|
<= 1e-4, fp64 <= 1e-10.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes
from gpu_util import require_gpu, err_max, assert_fp32, to_dev, torch

pytestmark = pytest.mark.gpu


def _env(C, M, seed):
    return scenes.rng(seed).uniform(0.0, 2.0, size=(C, M)).astype(np.float32)


@pytest.mark.parametrize("W,H,C,casc,M,seed", [
    (16, 16, 1, 0, 8, 0), (37, 23, 2, 0, 64, 1), (5, 7, 1, 0, 1, 2), (1, 6, 1, 0, 5, 3), (6, 1, 1, 0, 5, 3),
    (2, 2, 3, 0, 16, 4), (64, 48, 3, 0, 256, 5), (100, 100, 4, 0, 33, 6), (64, 64, 1, 3, 16, 7), (33, 65, 2, 0, 7, 8),
])
def test_env_forward_fp32_vs_oracle(W, H, C, casc, M, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    env = _env(C, M, 100 + seed)
    h = HRC(W, H, C, casc)
    h.set_environment(to_dev(env))
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    assert_fp32(F, oracle.fluence(e, s, casc, env=env))


def test_env_every_launch_configuration():
    """Schedules, merge-up groups, block widths, grid orders and both
    merge-down variants (per-thread loads, bulk-copy staging) read the map
    at the same out-of-range places: each matches the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(300, 260, 3, 14)
    env = _env(3, 48, 15)
    Fr = oracle.fluence(e, s, env=env)
    h = HRC(300, 260, 3)
    h.set_environment(to_dev(env))
    ed, sd = to_dev(e), to_dev(s)
    for cfg in [(0, 1, 128, 0, 0), (1, 2, 64, 1, 0), (0, 4, 256, 1, 1), (1, 4, 512, 0, 1), (0, 2, 64, 0, 1)]:
        h.set_launch_config(*cfg)
        F = h.forward(ed, sd).cpu().numpy()
        assert_fp32(F, Fr, msg=cfg)


@pytest.mark.parametrize("W,H,C,seed", [(16, 16, 1, 0), (37, 23, 2, 1)])
def test_env_forward_fp64_vs_oracle(W, H, C, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = (x.astype(np.float64) for x in scenes.random_scene(W, H, C, seed))
    env = _env(C, 24, 110 + seed)
    h = HRC(W, H, C, 0, "fp64")
    h.set_environment(to_dev(env))
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    assert err_max(F, oracle.fluence(e, s, env=env)) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("fp16", 1e-3), ("bf16", 6e-3)])
def test_env_reduced_precision(prec, tol):
    """The map in the reduced-precision storage modes (the same bounds as
    their fluence without a map)."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(64, 48, 3, 5)
    env = _env(3, 32, 120)
    h = HRC(64, 48, 3, 0, prec)
    h.set_environment(to_dev(env))
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    assert err_max(F, oracle.fluence(e, s, env=env)) <= tol


@pytest.mark.parametrize("W,H,C,seed,prec,tol", [
    (16, 16, 1, 0, "fp32", 1e-4), (37, 23, 2, 1, "fp32", 1e-4), (64, 48, 3, 5, "fp32", 1e-4),
    (1, 6, 1, 3, "fp32", 1e-4), (37, 23, 2, 1, "fp64", 1e-10),
])
def test_env_backward_vs_oracle(W, H, C, seed, prec, tol):
    """dL/de and dL/dsigma with the map (it adds T-gradient terms wherever a
    merge reads an out-of-grid R), reading the forward's levels and
    recomputing them."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    env = _env(C, 40, 130 + seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = scenes.rng(140 + seed).normal(size=e.shape)
    if prec == "fp32":
        g = g.astype(np.float32)
    else:
        e, s = e.astype(np.float64), s.astype(np.float64)
    re, rs = oracle.fluence_adjoint(e, s, g, env=env)
    h = HRC(W, H, C, 0, prec)
    h.set_environment(to_dev(env))
    ed, sd = to_dev(e, dt), to_dev(s, dt)
    for rc in (False, True):
        h.set_backward_recompute(rc)
        h.forward(ed, sd)
        ge, gs = (t.cpu().numpy() for t in h.backward(to_dev(g, dt)))
        assert err_max(ge, re) <= tol and err_max(gs, rs) <= tol, rc


@pytest.mark.parametrize("axis", ["+x", "-x", "+y", "-y"])
def test_env_light_from_one_side(axis):
    """A cos^8 lobe of light from `axis` onto a 64^2 grid whose far half is
    opaque: lit pixels see the lobe's integral 35 pi / 128 (within 2 %, the
    cone quadrature), pixels inside the wall nothing; independent of the
    oracle, this fixes the look direction of every frame."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    X, M = 64, 512
    ang = {"+x": 0.0, "+y": math.pi / 2, "-x": math.pi, "-y": 3 * math.pi / 2}[axis]
    th = 2 * math.pi * (np.arange(M) + 0.5) / M
    c = np.cos(th - ang)
    env = (np.where(c > 0, c, 0.0) ** 8).astype(np.float32)
    s = np.zeros((X, X), np.float32)
    h2 = X // 2
    sl = {"+x": (slice(None), slice(0, h2)), "-x": (slice(None), slice(h2, X)),
          "+y": (slice(0, h2), slice(None)), "-y": (slice(h2, X), slice(None))}[axis]
    s[sl] = 1e3
    lit = {"+x": (slice(None), slice(h2 + 8, X)), "-x": (slice(None), slice(0, h2 - 8)),
           "+y": (slice(h2 + 8, X), slice(None)), "-y": (slice(0, h2 - 8), slice(None))}[axis]
    dark = {"+x": (slice(4, X - 4), slice(4, h2 - 4)), "-x": (slice(4, X - 4), slice(h2 + 4, X - 4)),
            "+y": (slice(4, h2 - 4), slice(4, X - 4)), "-y": (slice(h2 + 4, X - 4), slice(4, X - 4))}[axis]
    h = HRC(X, X, 1)
    h.set_environment(to_dev(env))
    F = h.forward(torch.zeros((1, X, X), device="cuda"), to_dev(s)).cpu().numpy()[0]
    want = 35 * math.pi / 128
    assert np.max(np.abs(F[lit] - want)) <= 0.02 * want
    assert np.max(np.abs(F[dark])) <= 1e-5


def test_env_removed_and_host_entry():
    """Removing the map restores the map-free fluence bit for bit; the host
    entry point sees the map."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(70, 50, 3, 16)
    env = _env(3, 20, 17)
    h = HRC(70, 50, 3)
    ed, sd = to_dev(e), to_dev(s)
    F0 = h.forward(ed, sd).clone()
    h.set_environment(to_dev(env))
    Fh = h.forward_host(torch.from_numpy(e.copy()), torch.from_numpy(s.copy())).numpy()
    assert_fp32(Fh, oracle.fluence(e, s, env=env))
    h.set_environment(None)
    assert torch.equal(h.forward(ed, sd), F0)


def test_env_full_size_workload():
    """The 1024^2 three-channel workload under a sky-like map (bright above,
    dim below), autotuned launch configuration, against the oracle."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.scene_by_name("volumetric1024")
    C, H, W = e.shape
    th = 2 * math.pi * (np.arange(256) + 0.5) / 256
    env = np.stack([1.0 + 0.8 * np.sin(th + 0.3 * k) for k in range(C)]).astype(np.float32)
    h = HRC(W, H, C)
    h.autotune()
    h.set_environment(to_dev(env))
    F = h.forward(to_dev(e), to_dev(s)).cpu().numpy()
    assert_fp32(F, oracle.fluence(e, s, env=env))


# ---------------------------------------------------------------------------
# Top-level radiance supplied by the caller (hrc_set_top_radiance): R_N of
# every cone of every frame given directly, e.g. from cone tracing.
# ---------------------------------------------------------------------------
def _top(W, H, C, seed):
    K = 1
    while K < max(W, H):
        K *= 2
    return scenes.rng(seed).uniform(0.0, 1.0, size=(4, K, C)).astype(np.float32)


@pytest.mark.parametrize("W,H,C,seed", [(16, 16, 1, 0), (37, 23, 2, 1), (20, 6, 3, 2), (1, 6, 1, 3), (64, 48, 3, 4)])
def test_top_radiance_forward_and_backward_vs_oracle(W, H, C, seed):
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(W, H, C, seed)
    top = _top(W, H, C, 200 + seed)
    h = HRC(W, H, C)
    h.set_top_radiance(to_dev(top))
    ed, sd = to_dev(e), to_dev(s)
    for cfg in [(0, 1, 128, 0, 0), (1, 4, 64, 1, 1), (0, 4, 128, 0, 2)]:
        h.set_launch_config(*cfg)
        F = h.forward(ed, sd).cpu().numpy()
        assert_fp32(F, oracle.fluence(e, s, top=top), msg=cfg)
    gF = scenes.rng(300 + seed).normal(size=e.shape).astype(np.float32)
    ge, gs = h.backward(to_dev(gF))
    ge_r, gs_r = oracle.fluence_adjoint(e, s, gF, top=top)
    assert err_max(ge.cpu().numpy(), ge_r) <= 1e-4 and err_max(gs.cpu().numpy(), gs_r) <= 1e-4


def test_top_radiance_from_a_map_equals_the_map():
    """A table built from a map (the cone's arc times the map along the
    cone's middle direction) gives the map's fluence."""
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    from test_oracle_top_pins import top_from_map
    e, s = scenes.random_scene(48, 40, 2, 5)
    env = _env(2, 32, 6)
    h = HRC(48, 40, 2)
    ed, sd = to_dev(e), to_dev(s)
    h.set_environment(to_dev(env))
    Fm = h.forward(ed, sd).cpu().numpy()
    h.set_top_radiance(to_dev(top_from_map(env.astype(np.float64), 48, 40).astype(np.float32)))
    Ft = h.forward(ed, sd).cpu().numpy()
    assert_fp32(Ft, Fm)
    h.set_top_radiance(None)
    assert_fp32(h.forward(ed, sd).cpu().numpy(), oracle.fluence(e, s))


def test_top_radiance_with_per_channel_extinction():
    require_gpu()
    from paper_2505_02041_gb300 import HRC
    e, s = scenes.random_scene(33, 21, 3, 7)
    S = np.stack([s, 0.5 * s, 2.0 * s]).astype(np.float32)
    top = _top(33, 21, 3, 8)
    h = HRC(33, 21, 3)
    h.set_channel_extinction(True)
    h.set_top_radiance(to_dev(top))
    F = h.forward(to_dev(e), to_dev(S)).cpu().numpy()
    assert_fp32(F, oracle.fluence(e, S, top=top))
