"""Seeded synthetic inputs: multiscale Gaussian-sum densities and dyadic leaf lists.

Shared by the tests, the benchmark and the oracle comparisons.  It contains
none of the box code's arithmetic: only random draws, the analytic density
f(x) = sum_k a_k exp(-|x - c_k|^2 / (2 w_k^2)) (the paper's test densities
are randomly placed Gaussians, Sec. 4.1 and Sec. 4.3; width = standard
deviation), and integer dyadic leaf lists.

Draw order per configuration (numpy PCG64 ``default_rng(seed)``): centres
(cx, cy), then widths, then amplitudes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class GaussianSum:
    cx: np.ndarray
    cy: np.ndarray
    w: np.ndarray
    a: np.ndarray

    def __call__(self, xy: np.ndarray) -> np.ndarray:
        """Density at points xy[..., 2] (FP64)."""
        xy = np.asarray(xy, dtype=np.float64)
        out = np.zeros(xy.shape[:-1])
        x, y = xy[..., 0], xy[..., 1]
        for cx, cy, w, a in zip(self.cx, self.cy, self.w, self.a):
            out += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * w * w))
        return out

    @property
    def n(self) -> int:
        return int(self.cx.shape[0])


def gaussians(n: int, seed: int, wlog10=None, wuni=None, centre_box=0.5, amp="normal") -> GaussianSum:
    """n Gaussians: centres U[-centre_box, centre_box]^2, widths log-uniform in
    10**wlog10 (or uniform in wuni), amplitudes N(0,1) or ones."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-centre_box, centre_box, size=(n, 2))
    if wuni is not None:
        w = rng.uniform(wuni[0], wuni[1], size=n)
    else:
        w = 10.0 ** rng.uniform(wlog10[0], wlog10[1], size=n)
    a = np.ones(n) if amp == "ones" else rng.standard_normal(n)
    return GaussianSum(c[:, 0].copy(), c[:, 1].copy(), w, a)


# The workloads: density generators and tree recipes.
def config_density(cfg: int) -> GaussianSum:
    """Density of workload ``cfg`` (1: 3 broad Gaussians; 2: 20 Gaussians, widths
    1e-3..1e-1; 3: 200 Gaussians, widths 1e-4..1e-1)."""
    if cfg == 1:
        return gaussians(3, 0, wuni=(0.1, 0.3), amp="ones")
    if cfg == 2:
        return gaussians(20, 1, wlog10=(-3.0, -1.0))
    if cfg == 3:
        return gaussians(200, 2, wlog10=(-4.0, -1.0))
    raise ValueError(cfg)


def batch_density(k: int) -> tuple[GaussianSum, int, float]:
    """Density k of the 64-tree batch, its order p (8, 12, 16 round-robin) and
    the refinement tolerance eps = max(1e-11, 10^-p) (the paper pairs the
    order with the tolerance, p ~ log10(1/eps), Sec. 4.2).

    A per-tree knob t ~ U[0,1] (drawn first from the tree's seed) sets the
    number of Gaussians (3..20) and the smallest width; with the per-order
    width offset the trees span roughly 2e2..2e4 leaves, log-uniformly."""
    rng = np.random.default_rng(1000 + k)
    t = rng.uniform(0.0, 1.0)
    n = int(round(3 + 17 * t))
    p = (8, 12, 16)[k % 3]
    wmin = -1.0 - {8: 0.0, 12: 0.35, 16: 0.75}[p] - 1.6 * t
    return gaussians(n, 1000 + k, wlog10=(wmin, -0.9)), p, max(1e-11, 10.0 ** (-p))


def fictitious_curve_sources(n_panels: int = 256, q: int = 16, r0: float = 0.8, amp: float = 0.1, k: int = 5,
                             strip: float = 0.08):
    """Quadrature nodes of the fictitious curve of ``star_domain`` (the smooth
    curve r(t) = r0 + amp cos(k t) - strip, counterclockwise): n_panels equal
    panels in t, q Gauss-Legendre nodes each (the paper discretises its
    curves by Gauss-Legendre panels, Sec. 3.1).  Returns (xy[n, 2], w[n]
    arc-length weights, normal[n, 2] outward unit normals, t[n])."""
    g, gw = np.polynomial.legendre.leggauss(q)
    h = 2.0 * math.pi / n_panels
    t = ((np.arange(n_panels)[:, None] + 0.5) * h + 0.5 * h * g[None, :]).reshape(-1)
    wt = np.tile(0.5 * h * gw, n_panels)
    r = r0 + amp * np.cos(k * t) - strip
    dr = -amp * k * np.sin(k * t)
    xy = np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    d = np.stack([dr * np.cos(t) - r * np.sin(t), dr * np.sin(t) + r * np.cos(t)], axis=1)
    speed = np.linalg.norm(d, axis=1)
    normal = np.stack([d[:, 1], -d[:, 0]], axis=1) / speed[:, None]
    return xy, wt * speed, normal, t


def glue_densities(t: np.ndarray):
    """Smooth synthetic jump densities on the curve parameter t: sigma (the
    normal-derivative jump) and tau (the value jump) of Sec. 3.4."""
    return np.cos(3 * t) + 0.5 * np.sin(5 * t), np.sin(2 * t) + 0.3 * np.cos(7 * t)


def random_targets(n: int, seed: int = 101) -> np.ndarray:
    """n points uniform in [-1,1]^2."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, 2))


def uniform_leaves(level: int):
    """All 4^level leaves of a uniform tree, in row-major (iy slow) order."""
    n = 2 ** level
    iy, ix = np.divmod(np.arange(n * n), n)
    return (np.full(n * n, level, dtype=np.int32), ix.astype(np.int32), iy.astype(np.int32))


def geometric_leaves(g: GaussianSum, kappa: float = 1.0, max_level: int = 14):
    """Adaptive dyadic leaves of [-1,1]^2 from a purely geometric rule, then 2:1
    balanced (edge and corner neighbours).

    A box of half-side r is split while some Gaussian of width w < kappa*r has
    its centre within 12 w + 2 r of the box centre.  This gives trees with the
    same multiscale character as resolution-driven refinement without any
    polynomial arithmetic; it is used to make trees independently of the
    library's own refinement."""
    leaves = set()
    stack = [(0, 0, 0)]
    while stack:
        lv, i, j = stack.pop()
        r = 1.0 / 2 ** lv
        cx, cy = -1.0 + (2 * i + 1) * r, -1.0 + (2 * j + 1) * r
        d = np.hypot(g.cx - cx, g.cy - cy)
        split = lv < max_level and bool(np.any((g.w < kappa * r) & (d < 12 * g.w + 2 * r)))
        if split:
            for di in (0, 1):
                for dj in (0, 1):
                    stack.append((lv + 1, 2 * i + di, 2 * j + dj))
        else:
            leaves.add((lv, i, j))
    leaves = balance_leaves(leaves)
    arr = np.array(sorted(leaves), dtype=np.int64)
    return arr[:, 0].astype(np.int32), arr[:, 1].astype(np.int32), arr[:, 2].astype(np.int32)


def balance_leaves(leaves: set) -> set:
    """Split leaves until every pair of touching leaves differs by at most one level."""
    leaves = set(leaves)

    def covering(lv, i, j):
        # the leaf containing box (lv, i, j) at level <= lv, or None if it is subdivided
        for l2 in range(lv, -1, -1):
            s = lv - l2
            key = (l2, i >> s, j >> s)
            if key in leaves:
                return key
        return None

    changed = True
    while changed:
        changed = False
        for (lv, i, j) in sorted(leaves, key=lambda t: -t[0]):
            if (lv, i, j) not in leaves:
                continue
            n = 2 ** lv
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    if di == 0 and dj == 0:
                        continue
                    a, b = i + di, j + dj
                    if not (0 <= a < n and 0 <= b < n):
                        continue
                    c = covering(lv, a, b)
                    if c is not None and c[0] < lv - 1:
                        leaves.discard(c)
                        cl, ci, cj = c
                        for x in (0, 1):
                            for y in (0, 1):
                                leaves.add((cl + 1, 2 * ci + x, 2 * cj + y))
                        changed = True
    return leaves


def leaf_geometry(level, ix, iy, x0=-1.0, y0=-1.0, L=2.0) -> np.ndarray:
    """(cx, cy, r) per leaf for the root [x0, x0+L] x [y0, y0+L]."""
    level = np.asarray(level, dtype=np.int64)
    r = L * 0.5 / np.power(2.0, level)
    cx = x0 + (2.0 * np.asarray(ix, dtype=np.float64) + 1.0) * r
    cy = y0 + (2.0 * np.asarray(iy, dtype=np.float64) + 1.0) * r
    return np.stack([cx, cy, r], axis=1)


def sample_leaves(nleaf: int, k: int, seed: int = 7) -> np.ndarray:
    """k distinct leaf indices for sampled parity checks."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nleaf, size=min(k, nleaf), replace=False))


def sample_leaves_per_level(levels: np.ndarray, k: int, seed: int = 7) -> np.ndarray:
    """Up to k leaves from every level present (per-level error reports)."""
    rng = np.random.default_rng(seed)
    out = []
    for lv in np.unique(levels):
        idx = np.nonzero(levels == lv)[0]
        out.extend(rng.choice(idx, size=min(k, idx.size), replace=False).tolist())
    return np.array(sorted(out), dtype=np.int64)


def mass_hint(g: GaussianSum) -> float:
    """Untruncated total mass sum_k 2 pi a_k w_k^2 (for sanity checks only)."""
    return float(np.sum(2.0 * math.pi * g.a * g.w ** 2))


def star_domain(n: int = 600, r0: float = 0.8, amp: float = 0.1, k: int = 5, strip: float = 0.08):
    """A smooth star-shaped domain and its bulk region, as closed polygons of n
    vertices each (counterclockwise): the domain boundary r(t) = r0 + amp cos(k t)
    and the fictitious curve r(t) - strip, a radial inward offset (the paper's
    geometries are not available; Sec. 3.1 builds its curve by an inward offset
    of the boundary).  Returns (gamma, gamma_b), each [n, 2]."""
    t = 2.0 * math.pi * np.arange(n) / n
    r = r0 + amp * np.cos(k * t)
    gamma = np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    rb = r - strip
    gamma_b = np.stack([rb * np.cos(t), rb * np.sin(t)], axis=1)
    return gamma, gamma_b
