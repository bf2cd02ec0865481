"""Second formulation of HRC for tiny grids (test infrastructure only).

A direct, memoised transcription of the recursive definitions, written
independently of ``hrc_oracle.c`` (no shared code):

  * Trace (Eq. 9) by an Amanatides-Woo grid walk in exact rational arithmetic
    (Sec. 5 names this DDA), instead of the C oracle's sorted clipping;
  * T_n(p, k) by Eq. 18 / Eqs. 19-20 recursively from traced T_0..T_2;
  * R_n(p, i) by Eq. 14 / Eqs. 15-17 recursively, R_N = 0 (Sec. 4.2);
  * F(x, y) = sum over the four quadrant frames of R_0([x+1, y], 1/2).

Unlike the array form it applies NO cut at the grid boundary: probes outside
the grid are evaluated by the same recursion (their rays see vacuum).  Its
agreement with the array form therefore also checks the reading that the
array form's out-of-range lookups (vacuum T, zero R) are exact.

Pure Python; meant for grids of a few dozen pixels.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np


def _frame(q, e, s):
    """Quadrant frame fields: q0 (x,y), q1 (W-1-x,y), q2 (y,x), q3 (H-1-y,x)."""
    C, H, W = e.shape
    if q == 0:
        fe, fs = e.transpose(0, 2, 1), s.T
    elif q == 1:
        fe, fs = e[:, :, ::-1].transpose(0, 2, 1), s[:, ::-1].T
    elif q == 2:
        fe, fs = e, s
    else:
        fe, fs = e[:, ::-1, :], s[::-1, :]
    return np.ascontiguousarray(fe, np.float64), np.ascontiguousarray(fs, np.float64)


def _image_of(q, W, H, u, v):
    if q == 0:
        return u, v
    if q == 1:
        return W - 1 - u, v
    if q == 2:
        return v, u
    return v, H - 1 - u


def _env_radiance(env, dx, dy):
    """Environment map env[C][M] along image direction (dx, dy): samples at
    look angles 2 pi (m + 1/2) / M from +x towards +y, linear in between."""
    M = env.shape[1]
    th = math.atan2(dy, dx) % (2 * math.pi)
    t = th / (2 * math.pi) * M - 0.5
    m0 = math.floor(t)
    f = t - m0
    return (1 - f) * env[:, m0 % M] + f * env[:, (m0 + 1) % M]


class _Frame:
    def __init__(self, fe, fs, cascades, look=None, top=None):
        self.e, self.s = fe, fs            # e[C][U][V], s[U][V]
        self.look = look                   # (du, dv) -> radiance seen that way, or None
        self.top = top                     # R_N of cone j at top[j] ([K][C]), or None
        self.C, self.U, self.V = fe.shape
        N = 0
        while (1 << N) < self.U:
            N += 1
        if cascades > 0:
            N = min(N, cascades)
        self.N = N
        self.T = lru_cache(maxsize=None)(self._T)
        self.R = lru_cache(maxsize=None)(self._R)

    def cell(self, u, v):
        if 0 <= u < self.U and 0 <= v < self.V:
            return self.s[u, v], self.e[:, u, v]
        return 0.0, np.zeros(self.C)

    def trace(self, pu, pv, du, dv):
        """Amanatides-Woo walk from (pu, pv) along (du, dv), du > 0, exact
        rational crossing parameters; returns (L tuple, T)."""
        length = math.hypot(du, dv)
        pu, pv = Fraction(pu), Fraction(pv)
        cu, cv = math.floor(pu), math.floor(pv)
        step_v = (dv > 0) - (dv < 0)
        t_u = (cu + 1 - pu) / du
        t_v = ((cv + 1 - pv) / dv if dv > 0 else (cv - pv) / dv) if dv != 0 else Fraction(10**9)
        dt_u = Fraction(1, du)
        dt_v = Fraction(1, abs(dv)) if dv != 0 else Fraction(10**9)
        t = Fraction(0)
        L = np.zeros(self.C)
        Tacc = 1.0
        while t < 1:
            t_next = min(t_u, t_v, Fraction(1))
            l = float(t_next - t) * length
            if l > 0:
                sg, em = self.cell(cu, cv)
                tau = sg * l
                w = l if tau == 0 else -math.expm1(-tau) / sg
                L = L + Tacc * em * w
                Tacc *= math.exp(-tau)
            t = t_next
            if t >= 1:
                break
            hit_u, hit_v = t_u == t, t_v == t
            if hit_u:
                cu += 1
                t_u += dt_u
            if hit_v:
                cv += step_v
                t_v += dt_v
        return tuple(L), Tacc

    @staticmethod
    def merge(a, b):
        (La, Ta), (Lb, Tb) = a, b
        return tuple(x + Ta * y for x, y in zip(La, Lb)), Ta * Tb

    def _T(self, n, pu, pv, k):
        """T_n(p, k) ~ Trace(p, p + v_n(k)), p = (pu, pv) a level-n probe."""
        s = 1 << n
        if n <= min(2, self.N):
            return self.trace(pu + Fraction(1, 2), pv + Fraction(1, 2), s, 2 * k - s)
        m, sm = n - 1, s // 2
        if k % 2 == 0:                                              # Eq. 18
            kk = k // 2
            return self.merge(self.T(m, pu, pv, kk), self.T(m, pu + sm, pv + 2 * kk - sm, kk))
        kp, km = (k + 1) // 2, (k - 1) // 2                         # Eq. 19
        Fp = self.merge(self.T(m, pu, pv, kp), self.T(m, pu + sm, pv + 2 * kp - sm, km))
        Fm = self.merge(self.T(m, pu, pv, km), self.T(m, pu + sm, pv + 2 * km - sm, kp))
        return (tuple(0.5 * (a + b) for a, b in zip(Fm[0], Fp[0])), 0.5 * (Fm[1] + Fp[1]))  # Eq. 20

    def A(self, n, jp):
        s = 1 << n
        return math.atan2(2 * (jp + 1) - s, s) - math.atan2(2 * jp - s, s)   # Eq. 13

    def _R(self, n, pu, pv, ip):
        """R_n(p, i), i = ip + 1/2 (Eqs. 14-17); R_N = 0, or with an
        environment map A_N(i) times the map along v_N(i) (footnote 1)."""
        if n >= self.N:
            if self.top is not None:
                return tuple(float(x) for x in self.top[ip])
            if self.look is None:
                return (0.0,) * self.C
            s = 1 << n
            return tuple(self.A(n, ip) * self.look(s, 2 * ip + 1 - s))
        s = 1 << n
        x = pu >> n
        out = np.zeros(self.C)
        for k_edge, j in ((ip + 1, 2 * ip + 1), (ip, 2 * ip)):     # (i+1/2, j_+), (i-1/2, j_-)
            A = self.A(n + 1, j)
            if x % 2 == 1:                                          # Eq. 14
                L, T = self.T(n, pu, pv, k_edge)
                R = self.R(n + 1, pu + s, pv + 2 * k_edge - s, j)
                out += A * np.array(L) + T * np.array(R)
            else:                                                   # Eqs. 15-17
                k2 = 2 * k_edge                                     # 2i +- 1 at level n+1
                R0 = self.R(n + 1, pu, pv, j)
                L, T = self.T(n + 1, pu, pv, k2)
                R1 = self.R(n + 1, pu + 2 * s, pv + 2 * k2 - 2 * s, j)
                out += 0.5 * (np.array(R0) + A * np.array(L) + T * np.array(R1))
        return tuple(out)


def fluence(e, s, cascades: int = 0, env=None, top=None) -> np.ndarray:
    """F[C][H][W] from the recursive formulation (float64); `env` an
    environment map [C][M], or `top` the top-level radiance [4][K][C] (cone
    j of frame q at top[q][j]): R_N only, outside the grid the recursion runs
    on through vacuum."""
    e = np.asarray(e, np.float64)
    s = np.asarray(s, np.float64)
    if e.ndim == 2:
        e = e[None]
    C, H, W = e.shape
    F = np.zeros((C, H, W))
    for q in range(4):
        fe, fs = _frame(q, e, s)
        look = None
        if env is not None:
            envq = np.asarray(env, np.float64).reshape(C, -1)

            def look(du, dv, q=q, envq=envq):
                # image direction of the frame direction (du, dv): the image
                # points of two frame points one step apart
                x0, y0 = _image_of(q, W, H, 0, 0)
                x1, y1 = _image_of(q, W, H, du, dv)
                return _env_radiance(envq, x1 - x0, y1 - y0)
        fr = _Frame(fe, fs, cascades, look, None if top is None else np.asarray(top, np.float64)[q])
        if fr.N < 1 and look is None and top is None:
            continue
        for u in range(fr.U):
            for v in range(fr.V):
                x, y = _image_of(q, W, H, u, v)
                F[:, y, x] += np.array(fr.R(0, u + 1, v, 0))
    return F


def frame_T(e, s, q: int, n: int, cascades: int = 0) -> np.ndarray:
    """T_n of frame q over Algorithm 1's ranges, shape [U_n][2^n+1][V][C+1]."""
    e = np.asarray(e, np.float64)
    s = np.asarray(s, np.float64)
    if e.ndim == 2:
        e = e[None]
    fe, fs = _frame(q, e, s)
    fr = _Frame(fe, fs, cascades)
    Un = -(-fr.U // (1 << n))
    out = np.zeros((Un, (1 << n) + 1, fr.V, fr.C + 1))
    for x in range(Un):
        for k in range((1 << n) + 1):
            for v in range(fr.V):
                L, T = fr.T(n, x << n, v, k)
                out[x, k, v, :fr.C] = L
                out[x, k, v, fr.C] = T
    return out
