"""Pins of per-channel extinction (sigma_t[C][H][W]; the paper keeps T as
C-vectors, Sec. 5).

Every step of the method acts channel by channel once the extinction does
(Merge, Eq. 7; the Eq. 20 blend; the merge down, Eqs. 14-17; the fluence
sum; the cross blur; the bounce source), so the oracle states the
per-channel method as C single-channel problems.  The pins check that
statement against the shared-extinction oracle (equal channels give its
fluence bit for bit, and its sigma gradient is the sum of the channels'),
against a closed form with a different medium per channel (the uniform
emissive medium gives 2 pi e_c / sigma_c in channel c), and the adjoint by
central differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_02041_gb300 import scenes


@pytest.mark.parametrize("W,H,C,seed", [(12, 10, 3, 5), (7, 13, 2, 6), (1, 6, 4, 7)])
def test_equal_channels_reduce_to_shared_extinction(W, H, C, seed):
    e, s = (x.astype(np.float64) for x in scenes.random_scene(W, H, C, seed))
    S = np.stack([s] * C)
    assert np.array_equal(oracle.fluence(e, S), oracle.fluence(e, s))
    g = scenes.rng(seed).normal(size=e.shape)
    ge, gs = oracle.fluence_adjoint(e, S, g)
    ge1, gs1 = oracle.fluence_adjoint(e, s, g)
    assert np.array_equal(ge, ge1)
    assert np.max(np.abs(gs.sum(0) - gs1)) <= 1e-13 * max(1.0, np.max(np.abs(gs1)))


def test_uniform_media_per_channel():
    """Three channels, three uniform emissive media (sigma 50, 20, 80 and
    e = sigma * c_c): deep inside, channel c is 2 pi c_c, as for each medium
    alone (C2: L = (e / sigma)(1 - T) per interval)."""
    X = 64
    sig = [50.0, 20.0, 80.0]
    cc = [1.3, 0.4, 2.2]
    s = np.stack([np.full((X, X), v) for v in sig])
    e = np.stack([np.full((X, X), v * c) for v, c in zip(sig, cc)])
    F = oracle.fluence(e, s)
    for c in range(3):
        assert np.max(np.abs(F[c, 28:36, 28:36] - 2 * math.pi * cc[c])) <= 1e-9 * 2 * math.pi * cc[c]


def test_channels_are_independent():
    e, s = (x.astype(np.float64) for x in scenes.random_scene(14, 11, 3, 8))
    S = np.stack([s, 1.5 * s, 0.5 * s])
    F = oracle.fluence(e, S)
    S2 = S.copy()
    S2[1] *= 3.0
    F2 = oracle.fluence(e, S2)
    assert np.array_equal(F[0], F2[0]) and np.array_equal(F[2], F2[2])
    assert not np.allclose(F[1], F2[1])


def test_per_channel_adjoint_matches_central_differences():
    e, s = (x.astype(np.float64) for x in scenes.random_scene(12, 10, 2, 9))
    S = np.stack([s, 2.0 * s + 0.1])
    g = scenes.rng(10).normal(size=e.shape)
    ge, gs = oracle.fluence_adjoint(e, S, g)
    loss = lambda ee, ss: float(np.sum(g * oracle.fluence(ee, ss)))
    h = 1e-4
    for (c, y, x) in [(0, 2, 3), (1, 5, 5), (1, 7, 9), (0, 9, 0)]:
        sp, sm = S.copy(), S.copy()
        sp[c, y, x] += h
        sm[c, y, x] -= h
        fd = (loss(e, sp) - loss(e, sm)) / (2 * h)
        assert abs(fd - gs[c, y, x]) <= 1e-6 * max(1.0, abs(fd))
        ep, em = e.copy(), e.copy()
        ep[c, y, x] += h
        em[c, y, x] -= h
        fd = (loss(ep, S) - loss(em, S)) / (2 * h)
        assert abs(fd - ge[c, y, x]) <= 1e-9 * max(1.0, abs(fd))
