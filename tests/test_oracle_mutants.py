"""Mutation check of the oracle's pins.

Each variant is a temporary copy of hrc_oracle.c with one planted mistake
(a flipped sign, a swapped index, a dropped weight, a wrong operand, a wrong
quadrant map, a broken adjoint term), made by the (search, replace) edits
below -- each search text must occur exactly once in the oracle -- and
compiled on its own.  The oracle itself carries no trace of them.  The pins
used against the real oracle -- Fig. 2, the uniform slab, the independent
recursive formulation, the uniform emissive medium and central differences
-- must reject every variant.  The real oracle passes the same checks.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import recursive
from paper_2505_02041_gb300 import scenes
from conftest import read_golden

# name -> [(search, replace), ...] applied to a copy of oracle/hrc_oracle.c
MUTANTS = {
    "Eq. 18 far-operand offset sign": [
        ("T_get(cs, m, pu + sm, pv + 2 * kk - sm, kk), o);", "T_get(cs, m, pu + sm, pv - 2 * kk + sm, kk), o);")],
    "Eq. 19 far-operand direction": [
        ("T_get(cs, m, pu + sm, pv + 2 * kp - sm, km), Fp);", "T_get(cs, m, pu + sm, pv + 2 * kp - sm, kp), Fp);")],
    "Eq. 20 average dropped": [
        ("o[c] = 0.5 * (Fm[c] + Fp[c]);   /* Eq. 20 */", "o[c] = Fp[c];")],
    "Eq. 14 arc of the wrong half-cone": [
        ("double Am = orc_arc(n + 1, (int)jm);", "double Am = orc_arc(n + 1, (int)jm);\n                    Ap = Am;")],
    "Eq. 15 weight of R_{n+1}(p, j)": [
        ("o[c] += 0.5 * ((r0 ? r0[c] : 0.0) +", "o[c] += 0.5 * (2.0 * (r0 ? r0[c] : 0.0) +")],
    "fluence sum without the +1 offset": [
        ("R_val(&cs, 0, u + 1, v, 0);", "R_val(&cs, 0, u, v, 0);")],
    "Trace piece weight without phi": [
        ("double w = l * phi(tau);", "double w = l;")],
    "Merge with the far transmittance": [
        ("out[c] = La + Ta * Lb;", "out[c] = La + Tb * Lb;")],
    "Eq. 17 offset on the wrong level": [
        ("R_val(cs, n + 1, pu + s1, pv + 2 * kk - s1, j);", "R_val(cs, n + 1, pu + s1, pv + kk - s, j);")],
    "quadrant frame map of -y": [
        ("*y = H - 1 - u; break;", "*y = u; break;")],
    "odd / even x swapped": [
        ("if (x & 1) {\n                        /* Eq. 14", "if (!(x & 1) && x > 0) {\n                        /* Eq. 14")],
    "adjoint weight of R_{n+1}(p, j)": [
        ("gr[c] += 0.5 * g[c];", "gr[c] += 1.0 * g[c];")],
    "adjoint sign of the suffix-radiance term": [
        ("dphi(sg * l) - l * S[m * C + c]);", "dphi(sg * l) + l * S[m * C + c]);")],
    "Eq. 14 arcs of level n": [
        ("double Ap = orc_arc(n + 1, (int)jp);\n                    double Am = orc_arc(n + 1, (int)jm);",
         "double Ap = orc_arc(n, (int)ip);\n                    double Am = orc_arc(n, (int)ip);")],
    "Eq. 21 centre weight": [
        ("const double wc = 4.0;", "const double wc = 2.0;")],
    "cross blur without renormalisation of the kept weights": [
        ("            for (int c = 0; c < C; ++c) out[((size_t)c * H + y) * W + x] = acc[c] / wsum;",
         "            wsum = 8.0;\n            for (int c = 0; c < C; ++c) out[((size_t)c * H + y) * W + x] = acc[c] / wsum;")],
    "cross blur threshold on extinction instead of opacity": [
        ("    return fabs(am - ac) <= thr;", "    ac = s[y * W + x];\n    am = s[ym * W + xm];\n    return fabs(am - ac) <= thr;")],
    "cross blur adjoint scattered onto the wrong pixel": [
        ("gF[((size_t)c * H + ym) * W + xm] += gc;", "gF[((size_t)c * H + y) * W + x] += gc;")],
    "environment look direction of frame q1 mirrored": [
        ("    default: *dx = dv; *dy = -du; break;\n    }\n}", "    default: *dx = dv; *dy = -du; break;\n    }\n    if (q == 1) *dx = du;\n}")],
    "environment only at level N (out-of-grid lookups below it zero)": [
        ("v = cs->Renv[n + 1][(size_t)(2 * j) * C + c] + cs->Renv[n + 1][(size_t)(2 * j + 1) * C + c];", "v = 0.0;")],
    "environment values without the arc weight": [
        ("v = orc_arc(n, (int)j) * env_lookup(env, M, c, dx, dy);", "v = env_lookup(env, M, c, dx, dy);")],
    "top-level radiance of the next frame": [
        ("v = top[((size_t)q * K + j) * C + c];", "v = top[((size_t)((q + 1) & 3) * K + j) * C + c];")],
    "top-level radiance in reversed cone order": [
        ("v = top[((size_t)q * K + j) * C + c];", "v = top[((size_t)q * K + ((1L << N) - 1 - j)) * C + c];")],
}


def mutant_source(edits):
    """The oracle's C source with `edits` applied (each search text found
    exactly once)."""
    with open(os.path.join(os.path.dirname(oracle.__file__), "hrc_oracle.c")) as f:
        src = f.read()
    for old, new in edits:
        assert src.count(old) == 1, f"edit target not unique in the oracle: {old!r}"
        src = src.replace(old, new)
    return src


def failed_pins(O):
    """Names of the pins that variant O fails."""
    bad = []
    g = {r[0]: float(r[1]) for r in read_golden("fig2_worked_example.txt")}
    s = np.zeros((1, 3))
    e = np.zeros((1, 1, 3))
    s[0, :2] = math.log(2.0)
    e[0, 0, :2] = 4.0 * math.log(2.0)
    L, T = O.trace(e, s, (0.0, 0.5), (2.0, 0.5))
    if abs(L[0] - g["L_a_d"]) > 1e-12 or abs(T - g["T_a_d"]) > 1e-12:
        bad.append("fig2")
    sg, em = 0.7, 1.3
    ss = np.full((16, 16), sg)
    ee = np.full((1, 16, 16), em)
    L, T = O.trace(ee, ss, (3.2, 4.1), (9.7, 11.3))
    d = math.hypot(6.5, 7.2)
    if abs(L[0] - em / sg * -math.expm1(-sg * d)) > 1e-12:
        bad.append("slab")
    e1, s1 = scenes.random_scene(12, 10, 1, 77)
    if np.max(np.abs(O.fluence(e1, s1) - recursive.fluence(e1, s1))) > 1e-10:
        bad.append("recursive")
    for n in (3, 4):
        if np.max(np.abs(O.frame_level(e1, s1, 0, "T", n) - recursive.frame_T(e1, s1, 0, n))) > 1e-10:
            bad.append(f"T{n}")
    X = 64
    c = 1.7
    Fu = O.fluence(np.full((1, X, X), c), np.ones((X, X)))
    if np.max(np.abs(Fu[0, 28:36, 28:36] - 2 * math.pi * c)) > 1e-9:
        bad.append("uniform")
    e2, s2 = scenes.random_scene(10, 8, 1, 78)
    e2 = e2.astype(np.float64)
    s2 = s2.astype(np.float64)
    gF = np.random.default_rng(5).normal(size=e2.shape)
    ge, gs = O.fluence_adjoint(e2, s2, gF)
    h = 1e-4
    for (y, x) in [(3, 4), (6, 2)]:
        sp, sm = s2.copy(), s2.copy()
        sp[y, x] += h
        sm[y, x] -= h
        fd = (np.sum(gF * O.fluence(e2, sp)) - np.sum(gF * O.fluence(e2, sm))) / (2 * h)
        if abs(fd - gs[y, x]) > 1e-6 * max(1.0, abs(fd)):
            bad.append("fd")
            break
    bad += failed_blur_pins(O)
    bad += failed_env_pins(O)
    bad += failed_top_pins(O)
    return bad


def failed_top_pins(O):
    """The caller-supplied top-level radiance: a table built from a map
    reproduces the map's fluence, and the uniform table in vacuum gives
    2 pi E0."""
    from test_oracle_top_pins import top_from_map
    bad = []
    e, s = scenes.random_scene(20, 6, 2, 4)
    env = np.random.default_rng(4).uniform(0, 2, size=(2, 24))
    a = O.fluence(e, s, env=env)
    if np.max(np.abs(a - O.fluence(e, s, top=top_from_map(env, 20, 6)))) > 1e-12 * np.max(np.abs(a)):
        bad.append("top-map")
    F = O.fluence(np.zeros((1, 11, 13)), np.zeros((11, 13)), top=top_from_map(np.full((1, 8), 1.7), 13, 11))
    if np.max(np.abs(F - 2 * math.pi * 1.7)) > 1e-12:
        bad.append("top-uniform")
    return bad


def failed_env_pins(O):
    """The environment-map pins (footnote 1 of Sec. 4.2): uniform map in
    vacuum, array form = recursive form, light from -x behind an opaque
    right half."""
    bad = []
    F = O.fluence(np.zeros((1, 9, 11)), np.zeros((9, 11)), env=np.full((1, 8), 1.7))
    if np.max(np.abs(F - 2 * math.pi * 1.7)) > 1e-13:
        bad.append("env-uniform")
    e, s = scenes.random_scene(12, 10, 1, 77)
    env = np.random.default_rng(4).uniform(0, 2, size=(1, 24))
    if np.max(np.abs(O.fluence(e, s, env=env) - recursive.fluence(e, s, env=env))) > 1e-11:
        bad.append("env-recursive")
    X = 32
    sw = np.zeros((X, X))
    sw[:, X // 2:] = 1e3
    th = 2 * math.pi * (np.arange(256) + 0.5) / 256
    lobe = np.where(np.cos(th - math.pi) > 0, np.cos(th - math.pi), 0.0) ** 8
    Fw = O.fluence(np.zeros((1, X, X)), sw, env=lobe[None])[0]
    if np.max(np.abs(Fw[:, :X // 2 - 8] - 35 * math.pi / 128)) > 0.02 * 35 * math.pi / 128:
        bad.append("env-direction")
    return bad


def failed_blur_pins(O):
    """The cross-blur pins (Eq. 21): action on a quadratic, constants under
    rejections, the threshold side of a hand-built row, the adjoint's
    dot-product identity."""
    bad = []
    y, x = np.mgrid[0:7, 0:9].astype(np.float64)
    B = O.cross_blur((x * x + 3 * y * y)[None], np.full((7, 9), 0.3))[0]
    if np.max(np.abs(B[1:-1, 1:-1] - (x * x + 3 * y * y + 1.0)[1:-1, 1:-1])) > 1e-12:
        bad.append("blur-quadratic")
    g = np.random.default_rng(3)
    s = g.choice([0.0, 0.7, 3.0, 50.0], size=(8, 6))
    if np.max(np.abs(O.cross_blur(np.full((1, 8, 6), 2.0), s) - 2.0)) > 1e-14:
        bad.append("blur-constant")
    row = np.array([[-math.log(0.6), 0.0, -math.log(0.4)]])
    if abs(O.cross_blur(np.array([[[0.0, 1.0, 0.0]]]), row)[0, 0, 1] - 0.8) > 1e-15:
        bad.append("blur-threshold")
    F = g.normal(size=(2, 8, 6))
    G = g.normal(size=(2, 8, 6))
    if abs(np.sum(O.cross_blur(F, s) * G) - np.sum(F * O.cross_blur_adjoint(G, s))) > 1e-12:
        bad.append("blur-adjoint")
    return bad


def test_real_oracle_passes_every_pin():
    assert failed_pins(oracle) == []


def test_mutant_edits_apply_and_the_oracle_is_plain():
    """Every edit finds its target exactly once, and the oracle's source
    holds no switch for a planted mistake."""
    with open(os.path.join(os.path.dirname(oracle.__file__), "hrc_oracle.c")) as f:
        src = f.read()
    assert "MUTANT" not in src
    for edits in MUTANTS.values():
        assert mutant_source(edits) != src


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_planted_mistake_is_caught(name):
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    src = os.path.join(d, "hrc_oracle_mutant.c")
    lib = os.path.join(d, "liboracle_mutant.so")
    try:
        with open(src, "w") as f:
            f.write(mutant_source(MUTANTS[name]))
        O = oracle.load_variant(lib, src)
        assert failed_pins(O), f"planted mistake '{name}' passed every pin"
    finally:
        for p in (src, lib):
            if os.path.exists(p):
                os.remove(p)
        os.rmdir(d)
