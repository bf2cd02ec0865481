"""Seeded synthetic 2D scenes shaped like the paper's test scenes.

The paper uses self-made scenes (Section 5: emitters, a penumbra-casting
occluder, a fractal volumetric medium) and states that no standard 2D test
scenes exist. These generators stand in for them. They hold none of the
method's arithmetic: they only rasterise shapes into an emission map
``e[C][H][W]`` (per-unit-length source term of Eq. 4) and an extinction map
``sigma_t[H][W]`` (Eq. 2), both float32, row-major, pixel (x, y) being the unit
square [x, x+1] x [y, y+1].

Paint order for every scene: background extinction, then emitters (set e,
keep the extinction beneath), then occluders (set extinction, zero e). A
pixel belongs to a shape when its centre lies inside it.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` so the
oracle and the CUDA path see bit-identical inputs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "empty",
    "paint_disk",
    "paint_rect",
    "paint_capsule",
    "value_noise_fbm",
    "scene_disks_boxes",
    "scene_disks_rects_fog",
    "scene_volumetric_walls",
    "scene_by_name",
    "batched_sizes",
    "random_scene",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def empty(W: int, H: int, C: int):
    return np.zeros((C, H, W), np.float32), np.zeros((H, W), np.float32)


def _window(W, H, x0, x1, y0, y1):
    """Pixel-centre grids of the pixels whose centres may lie in the box
    [x0, x1] x [y0, y1] (clipped to the image), and their slices."""
    xa, xb = max(int(np.floor(x0)) - 1, 0), min(int(np.ceil(x1)) + 1, W)
    ya, yb = max(int(np.floor(y0)) - 1, 0), min(int(np.ceil(y1)) + 1, H)
    xa, ya = min(xa, W), min(ya, H)
    y, x = np.mgrid[ya:max(yb, ya), xa:max(xb, xa)]
    return x + 0.5, y + 0.5, (slice(ya, max(yb, ya)), slice(xa, max(xb, xa)))


def paint_disk(e, s, cx, cy, r, rgb):
    """Emitter disk: sets e inside, keeps the extinction beneath."""
    C, H, W = e.shape
    X, Y, win = _window(W, H, cx - r, cx + r, cy - r, cy + r)
    m = (X - cx) ** 2 + (Y - cy) ** 2 <= r * r
    for c in range(C):
        e[c][win][m] = rgb[c]
    return m


def paint_rect(e, s, cx, cy, w, h, angle, sigma):
    """Occluder rectangle (rotated by ``angle`` about its centre)."""
    C, H, W = e.shape
    rad = 0.5 * np.hypot(w, h)
    X, Y, win = _window(W, H, cx - rad, cx + rad, cy - rad, cy + rad)
    ca, sa = np.cos(angle), np.sin(angle)
    dx, dy = X - cx, Y - cy
    a = ca * dx + sa * dy
    b = -sa * dx + ca * dy
    m = (np.abs(a) <= 0.5 * w) & (np.abs(b) <= 0.5 * h)
    s[win][m] = sigma
    for c in range(C):
        e[c][win][m] = 0.0
    return m


def paint_capsule(e, s, x0, y0, x1, y1, width, sigma):
    """Occluder wall: all pixel centres within width/2 of the segment."""
    C, H, W = e.shape
    hw = 0.5 * width
    X, Y, win = _window(W, H, min(x0, x1) - hw, max(x0, x1) + hw, min(y0, y1) - hw, max(y0, y1) + hw)
    dx, dy = x1 - x0, y1 - y0
    L2 = dx * dx + dy * dy
    t = np.clip(((X - x0) * dx + (Y - y0) * dy) / max(L2, 1e-12), 0.0, 1.0)
    px, py = x0 + t * dx, y0 + t * dy
    m = (X - px) ** 2 + (Y - py) ** 2 <= hw * hw
    s[win][m] = sigma
    for c in range(C):
        e[c][win][m] = 0.0
    return m


def value_noise_fbm(W: int, H: int, g: np.random.Generator, octaves: int = 4):
    """Fractal value noise in [0, 1]: the first lattice cell is max(W,H)/8 px,
    each further octave halves cell size and amplitude; lattice values are
    U(0,1), interpolated with smoothstep; the sum is normalised to [0, 1]."""
    X = max(W, H)
    cell = X / 8.0
    amp = 1.0
    acc = np.zeros((H, W), np.float64)
    xs, ys = np.arange(W) + 0.5, np.arange(H) + 0.5
    for _ in range(octaves):
        nx, ny = int(np.ceil(W / cell)) + 2, int(np.ceil(H / cell)) + 2
        lat = g.random((ny, nx))
        fx, fy = xs / cell, ys / cell
        ix, iy = np.floor(fx).astype(int), np.floor(fy).astype(int)
        tx, ty = fx - ix, fy - iy
        sx, sy = tx * tx * (3 - 2 * tx), ty * ty * (3 - 2 * ty)
        a = lat[np.ix_(iy, ix)]
        b = lat[np.ix_(iy, ix + 1)]
        c = lat[np.ix_(iy + 1, ix)]
        d = lat[np.ix_(iy + 1, ix + 1)]
        top = a + (b - a) * sx[None, :]
        bot = c + (d - c) * sx[None, :]
        acc += amp * (top + (bot - top) * sy[:, None])
        cell *= 0.5
        amp *= 0.5
    lo, hi = acc.min(), acc.max()
    return ((acc - lo) / max(hi - lo, 1e-30)).astype(np.float32)


def scene_disks_boxes(W=64, H=64, C=1, seed=0, n_disks=3, n_boxes=2):
    """Small vacuum scene: emitter disks of radius 3 (value U(1,5)) and
    axis-aligned opaque boxes (extinction 1e3, integer sides 4..12)."""
    g = rng(seed)
    e, s = empty(W, H, C)
    for _ in range(n_disks):
        cx, cy = g.uniform(3, W - 3), g.uniform(3, H - 3)
        val = g.uniform(1, 5, size=C)
        paint_disk(e, s, cx, cy, 3.0, val)
    for _ in range(n_boxes):
        w, h = int(g.integers(4, 13)), int(g.integers(4, 13))
        x0 = int(g.integers(0, max(W - w, 0) + 1))
        y0 = int(g.integers(0, max(H - h, 0) + 1))
        s[y0:y0 + h, x0:x0 + w] = 1e3
        e[:, y0:y0 + h, x0:x0 + w] = 0.0
    return e, s


def scene_disks_rects_fog(W=512, H=512, C=3, seed=1, n_disks=20, n_rects=40,
                          fog=0.02, rect_sigma=50.0):
    """Emitter disks (radius U(2,20), per-channel value U(0,4)) and rotated
    non-emissive rectangles (sides U(4,64), extinction 50) in thin fog."""
    g = rng(seed)
    e, s = empty(W, H, C)
    s[:] = fog
    scale = max(W, H) / 512.0
    for _ in range(n_disks):
        cx, cy = g.uniform(0, W), g.uniform(0, H)
        r = g.uniform(2, 20) * max(scale, 0.25)
        paint_disk(e, s, cx, cy, r, g.uniform(0, 4, size=C))
    for _ in range(n_rects):
        cx, cy = g.uniform(0, W), g.uniform(0, H)
        w, h = g.uniform(4, 64) * max(scale, 0.25), g.uniform(4, 64) * max(scale, 0.25)
        paint_rect(e, s, cx, cy, w, h, g.uniform(0, np.pi), rect_sigma)
    return e, s


def scene_volumetric_walls(W=1024, H=1024, C=3, seed=2, n_disks=30, n_walls=100):
    """Fractal volumetric medium (extinction 5*fBm in [0,5]) with emitter
    disks as in ``scene_disks_rects_fog`` and thin walls (capsules of width
    1..3 px, length U(X/32, X/4), extinction 200)."""
    g = rng(seed)
    e, s = empty(W, H, C)
    s[:] = 5.0 * value_noise_fbm(W, H, g)
    X = max(W, H)
    scale = X / 512.0
    for _ in range(n_disks):
        cx, cy = g.uniform(0, W), g.uniform(0, H)
        r = g.uniform(2, 20) * scale
        paint_disk(e, s, cx, cy, r, g.uniform(0, 4, size=C))
    for _ in range(n_walls):
        x0, y0 = g.uniform(0, W), g.uniform(0, H)
        L = g.uniform(X / 32, X / 4)
        a = g.uniform(0, 2 * np.pi)
        wdt = int(g.integers(1, 4))
        paint_capsule(e, s, x0, y0, x0 + L * np.cos(a), y0 + L * np.sin(a), wdt, 200.0)
    return e, s


def random_scene(W, H, C, seed, fog=0.05):
    """Small heterogeneous scene for parity tests: random emission and
    extinction everywhere (no structure), so every pixel matters."""
    g = rng(seed)
    e = g.uniform(0.0, 2.0, size=(C, H, W)).astype(np.float32)
    s = (fog + g.exponential(0.5, size=(H, W))).astype(np.float32)
    return e, s


def batched_sizes(n=64, seed=4, choices=(128, 256, 512, 1024, 2048)):
    g = rng(seed)
    return [int(c) for c in g.choice(np.array(choices), size=n)]


def scene_by_name(name: str):
    """The named workloads: returns (e, sigma_t)."""
    if name == "disks64":          # 64^2, C=1, vacuum, 3 disks, 2 boxes
        return scene_disks_boxes(64, 64, 1, 0)
    if name == "fog512":           # 512^2, C=3, fog, 20 disks, 40 rects
        return scene_disks_rects_fog(512, 512, 3, 1)
    if name == "volumetric1024":   # 1024^2, C=3, fBm medium, 30 disks, 100 walls
        return scene_volumetric_walls(1024, 1024, 3, 2)
    if name == "fog2048":          # single 2048^2, C=3 scene
        return scene_disks_rects_fog(2048, 2048, 3, 5)
    raise KeyError(name)
