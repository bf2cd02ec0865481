"""Pins of the oracle's multi-bounce iteration (Sec. 4.2: the output
fluence fed into another iteration; Fig. 14).

Reading: a pixel with extinction sigma and single-scattering albedo rho
re-emits rho * sigma * F / (2 pi) per unit length (isotropic scattering in
2D), added to its own emission.  What pins it independently of the code:
inside a thick uniform medium the radiance transfer equation with
scattering has the closed-form solution L = c / (1 - rho) (c = e / sigma),
and K bounces give its partial sum 2 pi c (1 - rho^(K+1)) / (1 - rho); zero
bounces or zero albedo give the single-bounce fluence; the iteration is
linear in e and monotone in K; central differences check the adjoint in
e, sigma and albedo.  Planted mistakes (no sigma or no 1/(2 pi) in the
source, one bounce short, a dropped gradient term) must fail a pin.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes


def uniform_medium(rho, X=64, sg=50.0, c=1.3, C=1):
    e = np.full((C, X, X), sg * c)
    s = np.full((X, X), sg)
    a = np.full((C, X, X), rho)
    return e, s, a


def deep_interior_error(O, K, rho, **kw):
    e, s, a = uniform_medium(rho)
    F = O.fluence_bounces(e, s, a, K, **kw)
    want = 2 * math.pi * 1.3 * (1 - rho ** (K + 1)) / (1 - rho)
    return float(np.max(np.abs(F[0, 28:36, 28:36] - want)) / want)


@pytest.mark.parametrize("K,rho", [(1, 0.5), (2, 0.5), (5, 0.9), (6, 0.3)])
def test_thick_uniform_medium_partial_neumann_sum(K, rho):
    assert deep_interior_error(oracle, K, rho) <= 1e-9


def test_many_bounces_approach_the_scattering_solution():
    """40 bounces at rho = 0.5 reach 2 pi c / (1 - rho), the interior
    solution of transfer with scattering, to 1e-9."""
    e, s, a = uniform_medium(0.5)
    F = oracle.fluence_bounces(e, s, a, 40)
    assert np.max(np.abs(F[0, 28:36, 28:36] - 2 * math.pi * 1.3 / 0.5)) <= 1e-9 * 2 * math.pi * 1.3 / 0.5


def test_zero_bounces_or_zero_albedo_is_single_bounce():
    e, s = scenes.random_scene(20, 14, 2, 3)
    F1 = oracle.fluence(e, s)
    a = np.full(e.shape, 0.6)
    assert np.array_equal(oracle.fluence_bounces(e, s, a, 0), F1)
    assert np.max(np.abs(oracle.fluence_bounces(e, s, np.zeros(e.shape), 3) - F1)) <= 1e-15 * np.max(F1)


def test_linear_in_emission_and_monotone_in_bounces():
    e1, s = (x.astype(np.float64) for x in scenes.random_scene(18, 16, 1, 4))
    e2 = scenes.random_scene(18, 16, 1, 5)[0].astype(np.float64)
    a = scenes.rng(6).uniform(0, 0.9, size=e1.shape)
    F = lambda e: oracle.fluence_bounces(e, s, a, 3)
    lhs = F(2.0 * e1 - 0.5 * e2)
    rhs = 2.0 * F(e1) - 0.5 * F(e2)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    prev = oracle.fluence_bounces(e1, s, a, 0)
    for K in (1, 2, 3):
        cur = oracle.fluence_bounces(e1, s, a, K)
        assert np.all(cur >= prev - 1e-15)
        prev = cur


def adjoint_fd_error(O, blur=None):
    e, s = scenes.random_scene(12, 10, 2, 7)
    e = e.astype(np.float64)
    s = s.astype(np.float64)
    a = scenes.rng(8).uniform(0.1, 0.9, size=e.shape)
    g = scenes.rng(9).normal(size=e.shape)
    K = 2
    ge, gs, ga = O.fluence_bounces_adjoint(e, s, a, g, K, blur=blur)
    loss = lambda ee, ss, aa: float(np.sum(g * oracle.fluence_bounces(ee, ss, aa, K, blur=blur)))
    h = 1e-4
    worst = 0.0
    for (y, x) in [(2, 3), (5, 5), (7, 9), (4, 1)]:
        for which in ("e", "s", "a"):
            ep, em, sp, sm, ap, am = e.copy(), e.copy(), s.copy(), s.copy(), a.copy(), a.copy()
            if which == "e":
                ep[1, y, x] += h
                em[1, y, x] -= h
                got = ge[1, y, x]
            elif which == "s":
                sp[y, x] += h
                sm[y, x] -= h
                got = gs[y, x]
            else:
                ap[0, y, x] += h
                am[0, y, x] -= h
                got = ga[0, y, x]
            fd = (loss(ep, sp, ap) - loss(em, sm, am)) / (2 * h)
            worst = max(worst, abs(fd - got) / max(1.0, abs(fd)))
    return worst


def test_adjoint_matches_central_differences():
    assert adjoint_fd_error(oracle) <= 1e-6


def test_adjoint_with_cross_blur_matches_central_differences():
    """The blur inside every bounce (fixture pairs far from the threshold)."""
    assert adjoint_fd_error(oracle, blur=0.5) <= 1e-6


BOUNCE_MUTANTS = {
    "source without sigma": [("return e + sb * albedo * F / (2.0 * np.pi)", "return e + albedo * F / (2.0 * np.pi)")],
    "source without 1/(2 pi)": [("return e + sb * albedo * F / (2.0 * np.pi)", "return e + sb * albedo * F")],
    "one bounce short": [("    for _ in range(bounces):\n        F = _lighting(bounce_source(",
                          "    for _ in range(bounces - 1):\n        F = _lighting(bounce_source(")],
    "adjoint without the sigma term": [("        gs += np.sum(gek * albedo * Fp, axis=0) / (2.0 * np.pi)\n", "")],
}


def oracle_variant(edits):
    """A module made from a copy of the oracle package's source with `edits`
    applied (each search text found exactly once); it shares the compiled C
    oracle, so only the planted mistake in the bounce iteration differs."""
    import types
    path = oracle.__file__
    with open(path) as f:
        src = f.read()
    for old, new in edits:
        assert src.count(old) == 1, f"edit target not unique in the oracle: {old!r}"
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_variant")
    mod.__file__ = path
    exec(compile(src, path, "exec"), mod.__dict__)
    return mod


def test_bounce_mutant_edits_apply_and_the_oracle_is_plain():
    with open(oracle.__file__) as f:
        assert "mutant" not in f.read().lower()
    for edits in BOUNCE_MUTANTS.values():
        oracle_variant(edits)


@pytest.mark.parametrize("what", sorted(BOUNCE_MUTANTS))
def test_every_planted_mistake_is_caught(what):
    M = oracle_variant(BOUNCE_MUTANTS[what])
    caught = deep_interior_error(M, 2, 0.5) > 1e-9 or adjoint_fd_error(M) > 1e-6
    assert caught, what
