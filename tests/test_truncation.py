"""The truncated quadtree of Alg. 2 (both criteria, Sec. 3.2.1), on the host.

A star-shaped domain Omega (boundary gamma) with a bulk region Omega_B
(fictitious curve gamma_b, an inward offset); f is a Gaussian sum known on
Omega and extended by zero outside it.  The library's tree is checked with a
geometry written here independently (vertex-in-box, corner and edge-crossing
tests instead of the library's clipping): every leaf class, the separation
criterion (no leaf meets both Omega_B and the outside of Omega; a leaf that
meets the strip has a diagonal of at most half the local strip width), the
resolution criterion on leaves inside Omega, the zero extension's node mask,
and the lists (discarded leaves are no source and no target)."""
import numpy as np
import pytest

import paper_2501_17967_gb300 as bc
from paper_2501_17967_gb300 import synth

P = 8
EPS = 1e-8
MAXLV = 9


def inside(poly, x, y):
    """Winding number (nonzero rule) of the closed polygon around points (x, y)."""
    x = np.asarray(x, dtype=float)[..., None]
    y = np.asarray(y, dtype=float)[..., None]
    x0, y0 = poly[:, 0], poly[:, 1]
    x1, y1 = np.roll(x0, -1), np.roll(y0, -1)
    cross = (x1 - x0) * (y - y0) - (x - x0) * (y1 - y0)
    up = (y0 <= y) & (y1 > y) & (cross > 0)
    down = (y0 > y) & (y1 <= y) & (cross < 0)
    return (up.sum(-1) - down.sum(-1)) != 0


def seg_cross(ax, ay, bx, by, cx, cy, dx, dy):
    """Do segments ab and cd (arrays) properly cross or touch?"""
    def orient(px, py, qx, qy, rx, ry):
        return np.sign((qx - px) * (ry - py) - (qy - py) * (rx - px))
    o1, o2 = orient(ax, ay, bx, by, cx, cy), orient(ax, ay, bx, by, dx, dy)
    o3, o4 = orient(cx, cy, dx, dy, ax, ay), orient(cx, cy, dx, dy, bx, by)
    return (o1 * o2 <= 0) & (o3 * o4 <= 0)


def side(poly, x0, x1, y0, y1):
    """'cut' if the curve meets the box, else 'in' / 'out' of the region."""
    vx, vy = poly[:, 0], poly[:, 1]
    if np.any((vx >= x0) & (vx <= x1) & (vy >= y0) & (vy <= y1)):
        return "cut"
    cx = np.array([x0, x1, x1, x0]); cy = np.array([y0, y0, y1, y1])
    ins = inside(poly, cx, cy)
    if ins.any() and not ins.all():
        return "cut"
    wx, wy = np.roll(vx, -1), np.roll(vy, -1)
    for k in range(4):
        if np.any(seg_cross(vx, vy, wx, wy, cx[k], cy[k], cx[(k + 1) % 4], cy[(k + 1) % 4])):
            return "cut"
    return "in" if ins.all() else "out"


@pytest.fixture(scope="module")
def truncated():
    ctx = bc.Context(p=P, device=-1, cache_dir=None)
    gamma, gamma_b = synth.star_domain()
    g = synth.gaussians(6, 8, wlog10=(-1.6, -1.0))
    tree = bc.Tree.refine_truncated(ctx, g, gamma, gamma_b, eps=EPS, max_level=MAXLV)
    return ctx, tree, g, gamma, gamma_b


def test_leaf_classes_and_separation(truncated):
    ctx, tree, g, gamma, gamma_b = truncated
    lv, ix, iy = tree.leaves()
    cls = tree.leaf_class()
    assert set(np.unique(cls)) == {0, 1, 2}
    for k in range(tree.nleaf):
        r = 1.0 / 2 ** lv[k]
        x0, y0 = -1.0 + 2 * ix[k] * r, -1.0 + 2 * iy[k] * r
        s_o = side(gamma, x0, x0 + 2 * r, y0, y0 + 2 * r)
        s_b = side(gamma_b, x0, x0 + 2 * r, y0, y0 + 2 * r)
        assert cls[k] == {"out": 0, "cut": 1, "in": 2}[s_o], (k, cls[k], s_o)
        if lv[k] < MAXLV:
            # separation: not both Omega_B and the outside of Omega
            assert not (s_b != "out" and s_o != "in"), (k, s_o, s_b)
            if s_o != "out" and s_b != "in":   # meets the strip
                c = np.array([x0 + r, y0 + r])
                a = gamma[np.argmin(((gamma - c) ** 2).sum(1))]
                b = gamma_b[np.argmin(((gamma_b - c) ** 2).sum(1))]
                assert 2 * np.sqrt(2) * r <= 0.5 * np.hypot(*(a - b)) * (1 + 1e-12), k


def test_resolution_and_zero_extension(truncated):
    ctx, tree, g, gamma, gamma_b = truncated
    lv, ix, iy = tree.leaves()
    cls = tree.leaf_class()
    nodes = tree.nodes()
    mask = tree.node_mask()
    assert np.array_equal(mask.astype(bool), inside(gamma, nodes[..., 0], nodes[..., 1]))
    assert not mask[cls == 0].any() and mask[cls == 2].all()
    # coefficients of the zero-extended f on every leaf inside Omega resolved to eps
    from numpy.polynomial import chebyshev as C
    x = -np.cos((2 * np.arange(P) + 1) * np.pi / (2 * P))
    V = C.chebvander(x, P - 1)
    root = synth.leaf_geometry([0], [0], [0])
    xr = root[0, 0] + root[0, 2] * np.tile(x, P); yr = root[0, 1] + root[0, 2] * np.repeat(x, P)
    vscale = np.abs(g(np.stack([xr, yr], 1)) * inside(gamma, xr, yr)).max()
    for k in np.nonzero(cls == 2)[0]:
        f = g(nodes[k]).reshape(P, P)   # [jy][jx]
        c = np.linalg.solve(V, np.linalg.solve(V, f).T).T   # c[b][a]: T_a(x) T_b(y)
        tail = max(np.abs(c[P - 2:, :]).max(), np.abs(c[:, P - 2:]).max())
        if lv[k] < MAXLV:
            assert tail <= EPS * vscale * (1 + 1e-6), (k, tail, EPS * vscale)


def test_lists_skip_discarded_leaves(truncated):
    ctx, tree, g, gamma, gamma_b = truncated
    cls = tree.leaf_class()
    ptr, idx, _ = tree.lists(0)   # near: per target leaf, source leaves
    for o in range(tree.nleaf):
        srcs = idx[ptr[o]:ptr[o + 1]]
        if cls[o] == 0:
            assert srcs.size == 0
        assert np.all(cls[srcs] != 0)
    ptr, idx, _ = tree.lists(2)   # W: per target leaf
    assert all(ptr[o + 1] == ptr[o] for o in range(tree.nleaf) if cls[o] == 0)
    ptr, idx, _ = tree.lists(3)   # X: per box, source leaves
    assert np.all(cls[idx] != 0)


def test_truncation_argument_checks():
    ctx = bc.Context(p=P, device=-1, cache_dir=None)
    gamma, gamma_b = synth.star_domain()
    g = synth.gaussians(3, 1, wlog10=(-1.2, -1.0))
    with pytest.raises(bc.BoxCodeError):   # bulk curve outside the domain
        bc.Tree.refine_truncated(ctx, g, gamma_b, gamma, eps=EPS, max_level=6)
    with pytest.raises(bc.BoxCodeError):   # domain outside the root box
        bc.Tree.refine_truncated(ctx, g, 2.0 * gamma, gamma_b, eps=EPS, max_level=6)
