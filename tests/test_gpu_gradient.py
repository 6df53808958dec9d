"""Value and gradient of v_bulk off the grid (the glue data of Sec. 3.4: the
jumps tau and sigma need v_bulk and its normal derivative on the fictitious
curve).

Three checks:
  - against an independent host derivative of the same leaf interpolant
    (numpy Chebyshev fit of the node values and its derivative) at random
    points, at nodes and within 1e-13 of nodes (the cancellation-prone case
    of barycentric differentiation), bar 1e-12 of the leaf's scale;
  - against the oracle's value and gradient (direct quadrature of eq. (vbulk)
    and its derivative) at the vertices of the fictitious curve of a
    truncated star-shaped domain, with the normal derivative formed there;
  - points outside the root box: NaN on the device path, BC_ERR_ARG on the
    host path.

Bar against the oracle, derived from the apply's own bar: the node values
are within E = 1e-10 max|u| of the true potential; the interpolant of a node
error vector is bounded by Lambda_p E (Lebesgue constant of the p first-kind
Chebyshev points, < 2/pi log(p) + 1 < 2.8 at p = 16) and, being a polynomial
of degree p - 1 on [-1, 1], its derivative by Markov's inequality is at most
(p - 1)^2 times that, i.e. Lambda_p (p - 1)^2 E / r in physical units on a
leaf of half-width r.  The interpolation error of the smooth potential itself
adds at most the same bar again (the value test shows it below 1e-11).  The
split modes' node errors are 40-bit rounding noise, uncorrelated from node to
node, so their gradients carry that noise times the derivative factor
(1.4e-8 of max|grad u| measured on the star domain, inside the bound); the FP64 mode's node errors are the smooth truncation
error of the expansions and its gradient also meets a flat 1e-9 of
max|grad u| (1.4e-11 measured)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

P = 16


def _host_interp_grad(ub, xi, eta):
    """Value and reference-coordinate derivatives of the tensor interpolant of
    ub[p, p] (row jy, column jx) at (xi, eta) via Chebyshev coefficients."""
    C = np.polynomial.chebyshev
    xn = oracle.cheb_nodes(P)
    V = C.chebvander(xn, P - 1)
    coef = np.linalg.solve(V, np.linalg.solve(V, ub).T).T   # coef[ky, kx]
    vx, vy = C.chebvander(np.array([xi]), P - 1)[0], C.chebvander(np.array([eta]), P - 1)[0]
    dvx = np.array([C.chebval(xi, C.chebder(np.eye(P)[k])) for k in range(P)])
    dvy = np.array([C.chebval(eta, C.chebder(np.eye(P)[k])) for k in range(P)])
    return vy @ coef @ vx, vy @ coef @ dvx, dvy @ coef @ vx


def _containing_leaf(geom, x, y):
    for b in range(geom.shape[0]):
        cx, cy, r = geom[b]
        if cx - r <= x < cx + r and cy - r <= y < cy + r:
            return b
    return None


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return bc.Context(p=P, nterms=24, device=0)


def test_gradient_matches_host_interpolant(ctx):
    g = synth.config_density(2)
    tree = bc.Tree.refine(ctx, g, eps=1e-10, max_level=14)
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    geom = synth.leaf_geometry(lv, ix, iy)
    u = bc.apply(tree, torch.from_numpy(g(tree.nodes())).cuda())
    un = u.cpu().numpy().reshape(-1, P, P)
    rng = np.random.default_rng(5)
    pts = rng.uniform(-0.95, 0.95, (60, 2))
    nodes = oracle.leaf_nodes(geom, P)
    b_pick = rng.choice(len(lv), 6, replace=False)
    exact = nodes[b_pick, rng.integers(0, P * P, 6)]
    near = exact + np.array([1e-13, -2e-14])
    pts = np.vstack([pts, exact, near])
    val, grad = bc.eval_points_grad(tree, u, torch.from_numpy(pts).cuda())
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    val0 = bc.eval_points(tree, u, torch.from_numpy(pts).cuda()).cpu().numpy()
    assert np.all(np.isfinite(grad))
    assert np.abs(val - val0).max() <= 1e-14 * np.abs(un).max()
    worst = 0.0
    for k, (x, y) in enumerate(pts):
        b = _containing_leaf(geom, x, y)
        cx, cy, r = geom[b]
        v, dx, dy = _host_interp_grad(un[b], (x - cx) / r, (y - cy) / r)
        scale = np.abs(un[b]).max()
        assert abs(v - val[k]) <= 1e-13 * scale
        e = max(abs(dx / r - grad[k, 0]), abs(dy / r - grad[k, 1])) / (scale / r)
        worst = max(worst, e)
    print(f"gradient vs host interpolant derivative: {worst:.2e} of max|u_B|/r")
    assert worst < 1e-12, worst


def test_normal_derivative_on_fictitious_curve(ctx):
    gamma, gamma_b = synth.star_domain()
    g = synth.config_density(2)
    tree = bc.Tree.refine_truncated(ctx, g, gamma, gamma_b, eps=1e-11, max_level=18)
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    geom = synth.leaf_geometry(lv, ix, iy)
    mask = tree.node_mask().astype(bool)
    fz = np.where(mask, g(tree.nodes()), 0.0)
    pts = gamma_b[::4]
    # outward normal of the counterclockwise polygon at each vertex
    nxt, prv = np.roll(gamma_b, -1, 0)[::4], np.roll(gamma_b, 1, 0)[::4]
    t = nxt - prv
    nrm = np.stack([t[:, 1], -t[:, 0]], 1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    inside = ((np.abs(pts[:, None, 0] - geom[None, :, 0]) <= geom[None, :, 2])
              & (np.abs(pts[:, None, 1] - geom[None, :, 1]) <= geom[None, :, 2]))
    r_pt = np.where(inside, geom[None, :, 2], np.inf).min(1)
    assert np.all(np.isfinite(r_pt))
    for mode in (bc.FP64, bc.SPLIT_BF16):
        u = bc.apply(tree, torch.from_numpy(fz).cuda(), precision=mode)
        val, grad = bc.eval_points_grad(tree, u, torch.from_numpy(pts).cuda())
        val, grad = val.cpu().numpy(), grad.cpu().numpy()
        if mode == bc.FP64:
            ref_v = oracle.potential(P, geom, fz, pts)
            ref_g = oracle.gradient(P, geom, fz, pts)
        ev = np.abs(val - ref_v).max() / np.abs(ref_v).max()
        eg = np.abs(grad - ref_g).max() / np.abs(ref_g).max()
        dn, dn_ref = (grad * nrm).sum(1), (ref_g * nrm).sum(1)
        en = np.abs(dn - dn_ref).max() / np.abs(ref_g).max()
        print(f"fictitious curve, {len(pts)} points, mode {mode}: value {ev:.2e}, gradient {eg:.2e}, "
              f"normal derivative {en:.2e}")
        assert ev < 1e-10, ev
        E = 1e-10 * np.abs(u.cpu().numpy()).max()
        bound = 2 * 2.8 * (P - 1) ** 2 * E / r_pt + 1e-10 * np.abs(ref_g).max()
        assert np.all(np.abs(grad - ref_g).max(1) <= bound)
        assert np.all(np.abs(dn - dn_ref) <= bound)
        if mode == bc.FP64:
            assert eg < 1e-9 and en < 1e-9, (eg, en)


def test_points_outside_root(ctx):
    g = synth.config_density(1)
    tree = bc.Tree.refine(ctx, g, eps=1e-8, max_level=8)
    u = bc.apply(tree, torch.from_numpy(g(tree.nodes())).cuda())
    pts = np.array([[0.1, 0.2], [1.5, 0.0], [0.0, -1.0000001]])
    val, grad = bc.eval_points_grad(tree, u, torch.from_numpy(pts).cuda())
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    assert np.isfinite(val[0]) and np.all(np.isfinite(grad[0]))
    assert np.all(np.isnan(val[1:])) and np.all(np.isnan(grad[1:]))
    # host path validates and refuses
    import ctypes
    v = np.empty(3)
    gr = np.empty(6)
    un = np.ascontiguousarray(u.cpu().numpy())
    rc = bc._load().bc_eval_points_grad(ctx.handle, tree.handle, un.ctypes.data_as(ctypes.c_void_p),
                                        np.ascontiguousarray(pts).ctypes.data_as(ctypes.c_void_p), 3,
                                        v.ctypes.data_as(ctypes.c_void_p), gr.ctypes.data_as(ctypes.c_void_p),
                                        None)
    assert rc == -1
