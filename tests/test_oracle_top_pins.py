"""Pins of the oracle's caller-supplied top-level radiance (footnote 1 of
Sec. 4.2: offscreen light enters as R_N, which some other method -- a map,
cone tracing -- may compute).  The table top[q][j][c] holds R_N of cone j of
frame q; outside the grid a lower level sees the sum of its level-N
descendants, as with an environment map.

Pinned by: the independent recursive formulation; a table built here from
an environment map (cone arc x map radiance along the cone's middle
direction) reproducing the map's fluence; the uniform table in vacuum
giving 2 pi E0 everywhere; linearity; central differences of the adjoint.
"""
import math

import numpy as np

import oracle
from oracle import recursive
from paper_2505_02041_gb300 import scenes


def levels(U):
    N = 0
    while (1 << N) < U:
        N += 1
    return N


def top_from_map(env, W, H):
    """R_N of every cone of every frame from a map env[C][M]: the cone's
    arc (Eq. 13) times the map's radiance along the middle direction v_N(j +
    1/2), mapped from frame to image coordinates (q0: +x, q1: -x, q2: +y,
    q3: -y along u; v along +y for q0 / q1, +x for q2 / q3)."""
    C, M = env.shape
    Us = (W, W, H, H)
    K = 1 << max(levels(U) for U in Us)
    top = np.zeros((4, K, C))
    for q in range(4):
        N = levels(Us[q])
        s = 1 << N
        for j in range(s):
            du, dv = s, 2 * j + 1 - s
            dx, dy = [(du, dv), (-du, dv), (dv, du), (dv, -du)][q]
            th = math.atan2(dy, dx) % (2 * math.pi)
            t = th * M / (2 * math.pi) - 0.5
            m0 = math.floor(t)
            f = t - m0
            rad = (1 - f) * env[:, m0 % M] + f * env[:, (m0 + 1) % M]
            arc = math.atan2(2 * (j + 1) - s, s) - math.atan2(2 * j - s, s)
            top[q, j] = arc * rad
    return top


def test_top_array_form_equals_recursive_form():
    for (W, H, seed) in [(12, 10, 77), (20, 6, 78), (7, 9, 79)]:
        e, s = scenes.random_scene(W, H, 2, seed)
        K = 1 << max(levels(W), levels(H))
        top = np.random.default_rng(seed).uniform(0, 2, size=(4, K, 2))
        a = oracle.fluence(e, s, top=top)
        b = recursive.fluence(e, s, top=top)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a)), (W, H)


def test_top_from_a_map_reproduces_the_map():
    for (W, H, seed) in [(16, 16, 3), (20, 6, 4)]:
        e, s = scenes.random_scene(W, H, 2, seed)
        env = np.random.default_rng(seed).uniform(0, 2, size=(2, 24))
        a = oracle.fluence(e, s, env=env)
        b = oracle.fluence(e, s, top=top_from_map(env, W, H))
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a)), (W, H)


def test_uniform_top_in_vacuum_gives_two_pi():
    W, H, E0 = 13, 11, 1.7
    top = top_from_map(np.full((1, 8), E0), W, H)
    F = oracle.fluence(np.zeros((1, H, W)), np.zeros((H, W)), top=top)
    assert np.max(np.abs(F - 2 * math.pi * E0)) <= 1e-12


def test_top_is_linear_and_zero_is_no_light():
    e, s = scenes.random_scene(12, 10, 1, 5)
    g = np.random.default_rng(6)
    t1, t2 = g.uniform(0, 1, size=(2, 4, 16, 1))
    F1 = oracle.fluence(np.zeros_like(e), s, top=t1)
    F2 = oracle.fluence(np.zeros_like(e), s, top=t2)
    F12 = oracle.fluence(np.zeros_like(e), s, top=0.5 * t1 + 2.0 * t2)
    assert np.max(np.abs(F12 - 0.5 * F1 - 2.0 * F2)) <= 1e-12 * np.max(np.abs(F12))
    assert np.max(np.abs(oracle.fluence(e, s, top=np.zeros((4, 16, 1))) - oracle.fluence(e, s))) == 0.0


def test_top_adjoint_matches_central_differences():
    e, s = scenes.random_scene(10, 8, 1, 11)
    e = e.astype(np.float64)
    s = s.astype(np.float64)
    top = np.random.default_rng(12).uniform(0, 2, size=(4, 16, 1))
    gF = np.random.default_rng(13).normal(size=e.shape)
    ge, gs = oracle.fluence_adjoint(e, s, gF, top=top)
    h = 1e-4
    for (y, x) in [(3, 4), (6, 2), (0, 9)]:
        sp, sm = s.copy(), s.copy()
        sp[y, x] += h
        sm[y, x] -= h
        fd = (np.sum(gF * oracle.fluence(e, sp, top=top)) - np.sum(gF * oracle.fluence(e, sm, top=top))) / (2 * h)
        assert abs(fd - gs[y, x]) <= 1e-6 * max(1.0, abs(fd))
