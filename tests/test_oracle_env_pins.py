"""Pins of the oracle's environment map (footnote 1 of Sec. 4.2: R_N from
a map looked up along v_N(i), no occluders outside the grid).

Reading: env[c][m] is the radiance seen along the image-space look angle
theta_m = 2 pi (m + 1/2) / M (from +x towards +y, i.e. down the rows),
linearly interpolated; R_N(p, i) = A_N(i) env(direction of v_N(i)); an
out-of-grid R lookup at a lower level returns the sum over its level-N
descendants.  What pins it independently:
  * the recursive formulation, which has no table for out-of-grid lookups
    but simply continues the recursion outside the grid through vacuum,
    agrees with the array form (this is what makes the descendant sums
    exact, as C3 makes the zero lookups exact without a map);
  * in vacuum a uniform map E0 gives F = 2 pi E0 everywhere (the arcs of a
    quadrant sum to pi / 2);
  * light from one side behind an opaque half-plane: pixels on the lit side
    see the integral of the map over its lobe, pixels behind the wall
    nothing; this fixes the look-direction convention in x and in y;
  * linearity in (e, env), and central differences of the adjoint.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import recursive
from paper_2505_02041_gb300 import scenes


def lobe_env(M, axis_angle, power=8):
    """cos^power of the angle to axis_angle (zero beyond 90 degrees)."""
    th = 2 * math.pi * (np.arange(M) + 0.5) / M
    c = np.cos(th - axis_angle)
    return np.where(c > 0, c, 0.0) ** power


LOBE_INTEGRAL = 35 * math.pi / 128   # integral of cos^8 over (-pi/2, pi/2)


@pytest.mark.parametrize("W,H,C,casc,seed", [
    (12, 10, 1, 0, 77), (7, 13, 2, 0, 78), (3, 9, 1, 0, 79), (16, 16, 1, 3, 80), (1, 5, 1, 0, 81), (9, 1, 1, 0, 82),
])
def test_array_form_equals_recursive_form_with_env(W, H, C, casc, seed):
    e, s = scenes.random_scene(W, H, C, seed)
    env = scenes.rng(seed).uniform(0, 2, size=(C, 24))
    Fa = oracle.fluence(e, s, casc, env=env)
    Fr = recursive.fluence(e, s, casc, env=env)
    assert np.max(np.abs(Fa - Fr)) <= 1e-12 * max(1.0, np.max(np.abs(Fr)))


@pytest.mark.parametrize("W,H", [(16, 16), (21, 9), (1, 1), (2, 7)])
def test_uniform_map_in_vacuum_gives_2pi(W, H):
    F = oracle.fluence(np.zeros((2, H, W)), np.zeros((H, W)), env=np.array([[1.7] * 8, [0.3] * 8]))
    assert np.max(np.abs(F[0] - 2 * math.pi * 1.7)) <= 1e-13
    assert np.max(np.abs(F[1] - 2 * math.pi * 0.3)) <= 1e-13


@pytest.mark.parametrize("axis", ["+x", "-x", "+y", "-y"])
def test_light_from_one_side_behind_an_opaque_half(axis):
    """A lobe of light from direction `axis`; the half of a 64^2 grid on the
    side the light comes from is vacuum, the other half opaque (sigma =
    1e3).  Lit-side pixels at least 8 px from the wall see the lobe's
    integral (HRC's cone quadrature, within 2 %); pixels inside the wall,
    4 px or more from every grid edge, see nothing (at the grid edge the +1
    offset puts a pixel's probe outside, where the map is unobstructed).  A mirrored or transposed direction convention fails both."""
    X = 64
    ang = {"+x": 0.0, "+y": math.pi / 2, "-x": math.pi, "-y": 3 * math.pi / 2}[axis]
    s = np.zeros((X, X))
    lit = np.zeros((X, X), bool)
    dark = np.zeros((X, X), bool)
    h = X // 2
    if axis == "+x":
        s[:, :h] = 1e3
        lit[:, h + 8:] = True
        dark[4:X - 4, 4:h - 4] = True
    elif axis == "-x":
        s[:, h:] = 1e3
        lit[:, :h - 8] = True
        dark[4:X - 4, h + 4:X - 4] = True
    elif axis == "+y":
        s[:h, :] = 1e3
        lit[h + 8:, :] = True
        dark[4:h - 4, 4:X - 4] = True
    else:
        s[h:, :] = 1e3
        lit[:h - 8, :] = True
        dark[h + 4:X - 4, 4:X - 4] = True
    F = oracle.fluence(np.zeros((1, X, X)), s, env=lobe_env(512, ang)[None])[0]
    assert np.max(np.abs(F[lit] - LOBE_INTEGRAL)) <= 0.02 * LOBE_INTEGRAL
    assert np.max(np.abs(F[dark])) <= 1e-6


def test_linear_in_emission_and_map():
    e, s = (x.astype(np.float64) for x in scenes.random_scene(14, 11, 2, 5))
    env = scenes.rng(6).uniform(0, 1, size=(2, 16))
    F = oracle.fluence(e, s, env=env)
    assert np.max(np.abs(F - oracle.fluence(e, s) - oracle.fluence(np.zeros_like(e), s, env=env))) <= 1e-12 * np.max(F)
    assert np.max(np.abs(oracle.fluence(2.5 * e, s, env=2.5 * env) - 2.5 * F)) <= 1e-12 * np.max(F)


def test_adjoint_with_env_matches_central_differences():
    e, s = (x.astype(np.float64) for x in scenes.random_scene(12, 10, 2, 7))
    env = scenes.rng(8).uniform(0.5, 2, size=(2, 20))
    gF = scenes.rng(9).normal(size=e.shape)
    ge, gs = oracle.fluence_adjoint(e, s, gF, env=env)
    loss = lambda ee, ss: float(np.sum(gF * oracle.fluence(ee, ss, env=env)))
    h = 1e-4
    for (y, x) in [(2, 3), (5, 5), (7, 9), (0, 11), (9, 0)]:
        sp, sm = s.copy(), s.copy()
        sp[y, x] += h
        sm[y, x] -= h
        fd = (loss(e, sp) - loss(e, sm)) / (2 * h)
        assert abs(fd - gs[y, x]) <= 1e-6 * max(1.0, abs(fd))
        ep, em = e.copy(), e.copy()
        ep[0, y, x] += h
        em[0, y, x] -= h
        fd = (loss(ep, s) - loss(em, s)) / (2 * h)
        assert abs(fd - ge[0, y, x]) <= 1e-9 * max(1.0, abs(fd))
