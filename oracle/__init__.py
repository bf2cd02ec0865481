"""FP64 CPU oracle of Holographic Radiance Cascades (test infrastructure).

This package is TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
benchmark's CPU-baseline leg use it to check and time the CUDA path.  The
product package never imports it, and it shares no code with the product.

``hrc_oracle.c`` follows Algorithm 1 and Eqs. 7-20 step by step in double
precision (optionally with an environment map, footnote 1 of Sec. 4.2), and
the cross blur of Eq. 21 (Sec. 4.2) with its adjoint.  The
multi-bounce iteration of Sec. 4.2 (fluence fed back as a scattering
source) is composed from them here, in numpy.  ``recursive.py`` is a
second, independent formulation of Eqs. 14-20 (memoised recursion, pure
Python, tiny grids only).

Images are numpy arrays: emission ``e[C][H][W]`` and extinction ``s[H][W]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, out: str = _LIB, src: str = _SRC) -> str:
    """Compile the C oracle (or another source file `src`) with gcc (OpenMP on)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def _declare(L):
    L.orc_trace.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]
    L.orc_trace.restype = None
    L.orc_arc.argtypes = [ctypes.c_int, ctypes.c_int]
    L.orc_arc.restype = ctypes.c_double
    L.orc_levels.argtypes = [ctypes.c_int, ctypes.c_int]
    L.orc_levels.restype = ctypes.c_int
    L.orc_fluence.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
    L.orc_fluence.restype = None
    L.orc_fluence_env.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D,
                                  ctypes.c_int, _D]
    L.orc_fluence_env.restype = None
    L.orc_fluence_adjoint_env.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _D, ctypes.c_int, _D, _D]
    L.orc_fluence_adjoint_env.restype = None
    L.orc_fluence_top.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D,
                                  ctypes.c_int, _D]
    L.orc_fluence_top.restype = None
    L.orc_fluence_adjoint_top.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _D, ctypes.c_int, _D, _D]
    L.orc_fluence_adjoint_top.restype = None
    L.orc_frame_level.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
    L.orc_frame_level.restype = ctypes.c_long
    L.orc_fluence_adjoint.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _D, _D]
    L.orc_fluence_adjoint.restype = None
    L.orc_bruteforce.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
    L.orc_bruteforce.restype = None
    L.orc_cross_blur.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
    L.orc_cross_blur.restype = None
    L.orc_cross_blur_adjoint.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
    L.orc_cross_blur_adjoint.restype = None
    L.orc_num_threads.argtypes = []
    L.orc_num_threads.restype = ctypes.c_int
    L.orc_set_num_threads.argtypes = [ctypes.c_int]
    L.orc_set_num_threads.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _declare(ctypes.CDLL(_LIB))
    return _lib


class _Bound:
    """The oracle API bound to one compiled variant of hrc_oracle.c."""

    def __init__(self, handle):
        self._h = handle

    def __getattr__(self, name):
        fn = globals()[name]

        def call(*a, **k):
            global _lib
            saved = _lib
            _lib = self._h
            try:
                return fn(*a, **k)
            finally:
                _lib = saved
        return call


def load_variant(path: str, src: str):
    """Build and load a variant of the oracle compiled from the C source file
    `src` (the mutation test's edited copies); returns an object with this
    module's functions (trace, fluence, fluence_adjoint, ...)."""
    build(force=True, out=path, src=src)
    return _Bound(_declare(ctypes.CDLL(path)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _img(e, s):
    e = np.ascontiguousarray(e, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    if e.ndim == 2:
        e = e[None]
    C, H, W = e.shape
    assert s.shape == (H, W)
    return e, s, C, H, W


def trace(e, s, p, q):
    """Trace(p, q) of Eq. 9 in image coordinates: returns (L[C], T)."""
    e, s, C, H, W = _img(e, s)
    L = np.zeros(C)
    T = np.zeros(1)
    lib().orc_trace(_p(e), _p(s), C, W, H, float(p[0]), float(p[1]), float(q[0]), float(q[1]), _p(L), _p(T))
    return L, float(T[0])


def arc(n: int, ip: int) -> float:
    """A_n(i) of Eq. 13 for the cone i = ip + 1/2."""
    return lib().orc_arc(n, ip)


def levels(U: int, cascades: int = 0) -> int:
    return lib().orc_levels(U, cascades)


def _env(env, C):
    env = np.ascontiguousarray(env, dtype=np.float64)
    if env.ndim == 1:
        env = np.repeat(env[None], C, axis=0)
    assert env.ndim == 2 and env.shape[0] == C and env.shape[1] >= 1
    return env


def _top(top, C):
    top = np.ascontiguousarray(top, dtype=np.float64)
    assert top.ndim == 3 and top.shape[0] == 4 and top.shape[2] == C, "top radiance is [4][K][C]"
    return top


def _per_channel(fn, e, s, *rest):
    """Per-channel extinction s[C][H][W] (the paper stores T as C-vectors,
    Sec. 5): Merge (Eq. 7), the Eq. 20 blend, the merge down (Eqs. 14-17),
    the fluence sum, the cross blur and the bounce source all act channel
    by channel, and Trace gives channel c's radiance and transmittance from
    (e_c, sigma_c) alone, so the method is exactly C independent
    single-channel problems; fn(c, e_c, s_c, *rest_c) solves channel c.
    Returns the channel results stacked (tuples stacked element-wise)."""
    e = np.asarray(e)
    s = np.asarray(s)
    assert s.ndim == 3 and s.shape[0] == e.shape[0]
    outs = [fn(c, e[c:c + 1], s[c], *[np.asarray(r)[c:c + 1] for r in rest]) for c in range(s.shape[0])]
    if isinstance(outs[0], tuple):
        return tuple(np.concatenate([o[i] if o[i].ndim == 3 else o[i][None] for o in outs]) for i in range(len(outs[0])))
    return np.concatenate(outs)


def fluence(e, s, cascades: int = 0, env=None, top=None) -> np.ndarray:
    """Algorithm 1 (Lighting): F[C][H][W] in float64.  `env` ([C][M] or [M]):
    an environment map (footnote 1 of Sec. 4.2), radiance seen along the
    image-space look angle theta_m = 2 pi (m + 1/2) / M (theta from +x
    towards +y = down the rows), linearly interpolated.  `top` ([4][K][C]):
    the top-level radiance R_N itself, supplied by the caller (the same
    footnote: R_N computed by another method), cone j < 2^N of frame q at
    top[q][j][c]; outside the grid, as with a map, a lower level sees the
    sum of its level-N descendants."""
    if np.ndim(s) == 3:
        return _per_channel(lambda c, ec, sc: fluence(ec, sc, cascades, None if env is None else _env(env, len(e))[c:c + 1],
                                                      None if top is None else _top(top, len(e))[:, :, c:c + 1]),
                            e, s)
    e, s, C, H, W = _img(e, s)
    F = np.zeros((C, H, W))
    if top is not None:
        top = _top(top, C)
        lib().orc_fluence_top(_p(e), _p(s), C, W, H, cascades, _p(top), top.shape[1], _p(F))
    elif env is None:
        lib().orc_fluence(_p(e), _p(s), C, W, H, cascades, _p(F))
    else:
        env = _env(env, C)
        lib().orc_fluence_env(_p(e), _p(s), C, W, H, cascades, _p(env), env.shape[1], _p(F))
    return F


def frame_dims(q: int, W: int, H: int):
    return (W, H) if q < 2 else (H, W)


def frame_level(e, s, q: int, which: str, n: int, cascades: int = 0) -> np.ndarray:
    """T_n (which='T', shape [U_n][2^n+1][V][C+1]) or R_n (which='R', shape
    [U_n][2^n][V][C]) of quadrant frame q."""
    e, s, C, H, W = _img(e, s)
    U, V = frame_dims(q, W, H)
    Un = -(-U // (1 << n))
    w = 0 if which == "T" else 1
    cnt = lib().orc_frame_level(_p(e), _p(s), C, W, H, q, cascades, w, n, None)
    if cnt < 0:
        raise ValueError(f"level {which}_{n} does not exist")
    out = np.zeros(cnt)
    lib().orc_frame_level(_p(e), _p(s), C, W, H, q, cascades, w, n, _p(out))
    if w == 0:
        return out.reshape(Un, (1 << n) + 1, V, C + 1)
    return out.reshape(Un, 1 << n, V, C)


def fluence_adjoint(e, s, gF, cascades: int = 0, env=None, top=None):
    """Gradient of sum(gF * F) w.r.t. (e, s), float64 (with the environment
    map `env` or the top-level radiance `top` as in fluence, held fixed)."""
    if np.ndim(s) == 3:
        return _per_channel(lambda c, ec, sc, gc: fluence_adjoint(ec, sc, gc, cascades,
                                                                  None if env is None else _env(env, len(e))[c:c + 1],
                                                                  None if top is None else _top(top, len(e))[:, :, c:c + 1]),
                            e, s, np.asarray(gF).reshape(np.shape(e)))
    e, s, C, H, W = _img(e, s)
    gF = np.ascontiguousarray(gF, dtype=np.float64).reshape(C, H, W)
    ge = np.zeros((C, H, W))
    gs = np.zeros((H, W))
    if top is not None:
        top = _top(top, C)
        lib().orc_fluence_adjoint_top(_p(e), _p(s), _p(gF), C, W, H, cascades, _p(top), top.shape[1],
                                      _p(ge), _p(gs))
    elif env is None:
        lib().orc_fluence_adjoint(_p(e), _p(s), _p(gF), C, W, H, cascades, _p(ge), _p(gs))
    else:
        env = _env(env, C)
        lib().orc_fluence_adjoint_env(_p(e), _p(s), _p(gF), C, W, H, cascades, _p(env), env.shape[1],
                                      _p(ge), _p(gs))
    return ge, gs


def cross_blur(F, s, threshold: float = 0.5) -> np.ndarray:
    """The cross blur of Eq. 21 with opacity rejection (Sec. 4.2): each pixel
    averages itself (weight 4) with the edge neighbours (weight 1) inside the
    grid whose opacity 1 - exp(-sigma) is within `threshold` of its own, the
    kept weights renormalised.  F[C][H][W] -> float64 [C][H][W]; with
    per-channel extinction s[C][H][W], channel c tests sigma_c."""
    if np.ndim(s) == 3:
        return _per_channel(lambda c, Fc, sc: cross_blur(Fc, sc, threshold), F, s)
    F, s, C, H, W = _img(F, s)
    out = np.zeros((C, H, W))
    lib().orc_cross_blur(_p(F), _p(s), C, W, H, float(threshold), _p(out))
    return out


def cross_blur_adjoint(g, s, threshold: float = 0.5) -> np.ndarray:
    """Transpose of cross_blur for fixed sigma: dL/dF from dL/d(blurred F)."""
    if np.ndim(s) == 3:
        return _per_channel(lambda c, gc, sc: cross_blur_adjoint(gc, sc, threshold), g, s)
    g, s, C, H, W = _img(g, s)
    gF = np.zeros((C, H, W))
    lib().orc_cross_blur_adjoint(_p(g), _p(s), C, W, H, float(threshold), _p(gF))
    return gF


def fluence_blurred(e, s, threshold: float = 0.5, cascades: int = 0) -> np.ndarray:
    """Algorithm 1 (Lighting) followed by the cross blur of Eq. 21."""
    return cross_blur(fluence(e, s, cascades), s, threshold)


def fluence_blurred_adjoint(e, s, gF, threshold: float = 0.5, cascades: int = 0):
    """Gradient of sum(gF * fluence_blurred(e, s)) w.r.t. (e, s); the blur's
    kept set is held fixed (its dependence on s is piecewise constant)."""
    return fluence_adjoint(e, s, cross_blur_adjoint(gF, s, threshold), cascades)


def _lighting(e, s, cascades, blur):
    return fluence(e, s, cascades) if blur is None else fluence_blurred(e, s, blur, cascades)


def _lighting_adjoint(e, s, g, cascades, blur):
    if blur is None:
        return fluence_adjoint(e, s, g, cascades)
    return fluence_blurred_adjoint(e, s, g, blur, cascades)


def bounce_source(e, s, albedo, F):
    """Emission of the next bounce (Sec. 4.2: the output fluence fed into
    another iteration), read as isotropic single scattering in 2D: a pixel
    with extinction sigma and albedo rho scatters sigma * rho of the fluence F
    (radiance integrated over the full turn) evenly over 2 pi, so its source
    per unit length becomes e + rho * sigma * F / (2 pi)."""
    sb = s if np.ndim(s) == 3 else s[None]   # per-channel extinction: sigma_c for channel c
    return e + sb * albedo * F / (2.0 * np.pi)


def fluence_bounces(e, s, albedo, bounces: int, cascades: int = 0, blur=None):
    """Multi-bounce lighting: F_0 = Lighting(e), e_k = e + albedo * s * F_{k-1}
    / (2 pi), F_k = Lighting(e_k); returns F_bounces (float64 [C][H][W]).
    `blur` = None, or the cross-blur threshold applied by every Lighting."""
    if np.ndim(s) == 3:
        return _per_channel(lambda c, ec, sc, ac: fluence_bounces(ec, sc, ac, bounces, cascades, blur),
                            e, s, albedo)
    e, s, C, H, W = _img(e, s)
    albedo = np.ascontiguousarray(albedo, dtype=np.float64).reshape(C, H, W)
    F = _lighting(e, s, cascades, blur)
    for _ in range(bounces):
        F = _lighting(bounce_source(e, s, albedo, F), s, cascades, blur)
    return F


def fluence_bounces_adjoint(e, s, albedo, gF, bounces: int, cascades: int = 0, blur=None):
    """Gradient of sum(gF * fluence_bounces(...)) w.r.t. (e, s, albedo), by
    the reverse of the iteration: the adjoint of Lighting at each e_k, and of
    the source update through F_{k-1}, s and albedo."""
    if np.ndim(s) == 3:
        return _per_channel(lambda c, ec, sc, ac, gc: fluence_bounces_adjoint(ec, sc, ac, gc, bounces, cascades, blur),
                            e, s, albedo, np.asarray(gF).reshape(np.shape(e)))
    e, s, C, H, W = _img(e, s)
    albedo = np.ascontiguousarray(albedo, dtype=np.float64).reshape(C, H, W)
    g = np.ascontiguousarray(gF, dtype=np.float64).reshape(C, H, W)
    Fs, es = [], [e]
    F = _lighting(e, s, cascades, blur)
    for _ in range(bounces):
        Fs.append(F)
        es.append(bounce_source(e, s, albedo, F))
        F = _lighting(es[-1], s, cascades, blur)
    ge = np.zeros((C, H, W))
    gs = np.zeros((H, W))
    ga = np.zeros((C, H, W))
    for k in range(bounces, -1, -1):
        gek, gsk = _lighting_adjoint(es[k], s, g, cascades, blur)
        ge += gek
        gs += gsk
        if k == 0:
            break
        Fp = Fs[k - 1]
        gs += np.sum(gek * albedo * Fp, axis=0) / (2.0 * np.pi)
        ga += gek * s[None] * Fp / (2.0 * np.pi)
        g = gek * albedo * s[None] / (2.0 * np.pi)
    return ge, gs, ga


def bruteforce(e, s, M: int = 4096) -> np.ndarray:
    """Eq. 1 by brute force with M uniformly spaced directions per pixel."""
    e, s, C, H, W = _img(e, s)
    F = np.zeros((C, H, W))
    lib().orc_bruteforce(_p(e), _p(s), C, W, H, M, _p(F))
    return F


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(n)
