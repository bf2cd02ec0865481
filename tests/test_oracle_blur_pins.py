"""Pins of the oracle's cross blur (Sec. 4.2, Eq. 21, with opacity rejection).

Eq. 21 fixes the stencil: weight 4 at the pixel and 1 at each edge
neighbour, over 8.  The paper leaves "differ significantly in opacity"
open; the reading pinned here keeps a neighbour iff it is inside the grid
and its opacity 1 - exp(-sigma) is within the threshold (0.5) of the
pixel's, and renormalises the kept weights.  The pins are properties that
any implementation of that reading must have: the stencil's exact action on
quadratics (which fixes the weights and the 1/8), the removal of the
odd/even checkerboard the blur exists for, constants kept under any
rejection pattern (which fixes the renormalisation), the threshold's side
on a hand-built pair, D4 equivariance, and the adjoint's dot-product
identity and central differences of the blurred fluence.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes


def _grid(H, W):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    return x, y


@pytest.mark.parametrize("p,q", [(1.0, 3.0), (-0.5, 2.0), (0.0, 0.0)])
def test_interior_action_on_quadratics(p, q):
    """With every neighbour kept, (4 F + sum of the 4 neighbours) / 8 of
    F = a + b x + c y + p x^2 + q y^2 is F + (p + q) / 4 (second differences
    of 2p and 2q, each weighted 1/8)."""
    H, W = 9, 11
    x, y = _grid(H, W)
    F = 0.3 + 0.7 * x - 1.1 * y + p * x * x + q * y * y
    s = np.full((H, W), 0.25)
    B = oracle.cross_blur(F[None], s)[0]
    inner = (slice(1, H - 1), slice(1, W - 1))
    assert np.max(np.abs(B[inner] - (F[inner] + (p + q) / 4))) <= 1e-12


def test_removes_the_odd_even_checkerboard():
    """The checkerboard that HRC leaves (odd and even rows do not interact
    for n >= 1, Sec. 4.2) is removed exactly in the interior: a mean d plus
    c (-1)^(x+y) blurs to d."""
    H, W = 8, 10
    x, y = _grid(H, W)
    F = 2.5 + 0.75 * (-1.0) ** (x + y)
    s = np.full((H, W), 1.0)
    B = oracle.cross_blur(F[None], s)[0]
    assert np.max(np.abs(B[1:-1, 1:-1] - 2.5)) <= 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_constants_survive_any_rejection_pattern(seed):
    """A normalised average: a constant image stays constant at edges,
    corners and wherever neighbours are rejected."""
    g = np.random.default_rng(seed)
    H, W = 13, 7
    s = g.choice([0.0, 0.05, 0.7, 3.0, 50.0], size=(H, W))
    F = np.full((2, H, W), 1.75)
    B = oracle.cross_blur(F, s)
    assert np.max(np.abs(B - 1.75)) <= 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_output_is_a_convex_combination(seed):
    """Every output lies between the min and max of the pixel and its four
    neighbours (the kept weights are positive and sum to 1)."""
    g = np.random.default_rng(10 + seed)
    H, W = 12, 9
    s = g.uniform(0, 3, size=(H, W))
    F = g.normal(size=(1, H, W))
    B = oracle.cross_blur(F, s)[0]
    P = np.pad(F[0], 1, mode="edge")
    nb = np.stack([P[1:-1, 1:-1], P[:-2, 1:-1], P[2:, 1:-1], P[1:-1, :-2], P[1:-1, 2:]])
    assert np.all(B >= nb.min(0) - 1e-14) and np.all(B <= nb.max(0) + 1e-14)


def test_threshold_side_on_a_hand_built_row():
    """One row: pixel 1 is vacuum (opacity 0), its left neighbour has
    opacity 0.4 (kept at threshold 0.5), its right neighbour 0.6 (rejected).
    With F = (0, 1, 0) the centre becomes (4 * 1 + 0) / 5 = 0.8; with both
    kept it would be 4/6, with none 1.  The outcome depends on the opacity
    difference, not on the extinction difference (0.51 and 0.92)."""
    s = np.array([[-math.log(0.6), 0.0, -math.log(0.4)]])
    F = np.array([[[0.0, 1.0, 0.0]]])
    B = oracle.cross_blur(F, s, 0.5)
    assert abs(B[0, 0, 1] - 0.8) <= 1e-15
    # the same pair at a threshold of 0.7 keeps both neighbours
    assert abs(oracle.cross_blur(F, s, 0.7)[0, 0, 1] - 4.0 / 6.0) <= 1e-15
    # threshold 0 keeps only equal-opacity neighbours: none here
    assert abs(oracle.cross_blur(F, s, 0.0)[0, 0, 1] - 1.0) <= 1e-15


def test_d4_equivariance():
    g = np.random.default_rng(4)
    X = 10
    s = g.uniform(0, 2, size=(X, X))
    F = g.normal(size=(2, X, X))
    B = oracle.cross_blur(F, s)
    for k in range(4):
        Br = oracle.cross_blur(np.rot90(F, k, axes=(1, 2)).copy(), np.rot90(s, k).copy())
        assert np.max(np.abs(Br - np.rot90(B, k, axes=(1, 2)))) <= 1e-14
    Bt = oracle.cross_blur(np.transpose(F, (0, 2, 1)).copy(), s.T.copy())
    assert np.max(np.abs(Bt - np.transpose(B, (0, 2, 1)))) <= 1e-14


@pytest.mark.parametrize("W,H,C,seed", [(7, 5, 1, 0), (16, 16, 3, 1), (1, 6, 2, 2), (9, 1, 1, 3)])
def test_adjoint_dot_product_identity(W, H, C, seed):
    """<B F, G> = <F, B^T G> for fixed sigma with rejections."""
    g = np.random.default_rng(20 + seed)
    s = g.choice([0.0, 0.2, 1.0, 4.0], size=(H, W)) + g.uniform(0, 0.05, size=(H, W))
    F = g.normal(size=(C, H, W))
    G = g.normal(size=(C, H, W))
    lhs = np.sum(oracle.cross_blur(F, s) * G)
    rhs = np.sum(F * oracle.cross_blur_adjoint(G, s))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_blurred_fluence_adjoint_matches_central_differences():
    """Gradient of sum(gF * blur(F(e, s))): in e exactly linear; in sigma the
    kept set is piecewise constant, so central differences at pixels whose
    pairs sit far from the threshold match the adjoint that holds it fixed."""
    e, s = scenes.random_scene(12, 10, 2, 5)
    e = e.astype(np.float64)
    s = s.astype(np.float64)
    gF = np.random.default_rng(6).normal(size=e.shape)
    ge, gs = oracle.fluence_blurred_adjoint(e, s, gF)

    def loss(ee, ss):
        return float(np.sum(gF * oracle.fluence_blurred(ee, ss)))

    a = 1.0 - np.exp(-s)
    h = 1e-4
    checked = 0
    for (y, x) in [(2, 3), (5, 5), (7, 9), (4, 1), (8, 6), (1, 10)]:
        ep, em = e.copy(), e.copy()
        ep[1, y, x] += h
        em[1, y, x] -= h
        fd = (loss(ep, s) - loss(em, s)) / (2 * h)
        assert abs(fd - ge[1, y, x]) <= 1e-9 * max(1.0, abs(fd))
        margins = [abs(abs(a[y + dy, x + dx] - a[y, x]) - 0.5) for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0))
                   if 0 <= y + dy < s.shape[0] and 0 <= x + dx < s.shape[1]]
        if min(margins) < 1e-2:
            continue
        sp, sm = s.copy(), s.copy()
        sp[y, x] += h
        sm[y, x] -= h
        fd = (loss(e, sp) - loss(e, sm)) / (2 * h)
        assert abs(fd - gs[y, x]) <= 1e-6 * max(1.0, abs(fd))
        checked += 1
    assert checked >= 3
