"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

The oracle evaluates u(x) = (1/2pi) sum_B int_B log|x-y| f_B(y) dy, which is
v_bulk = -int Phi f of the paper (Sec. 3.2, eq. (vbulk); Phi from Sec. 2), so
that Laplace(u) = f.  Each test below checks it against something other than
itself:
  * closed forms: constant density on a rectangle, centre of a square,
    radially symmetric Gaussian (exponential integral);
  * an independent library quadrature (scipy dblquad) on one leaf;
  * the PDE itself: Laplace(u) = f by spectral differentiation;
  * exact invariants: scaling law, dihedral symmetry, linearity, additivity.
A dropped term, a wrong sign or a transposed index in the oracle fails at
least one of them.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

pytestmark = []


def _F(a, b):
    """int_0^a int_0^b (1/2) log(x^2 + y^2) dy dx, signed a, b (closed form)."""
    if a == 0.0 or b == 0.0:
        return 0.0
    s = math.copysign(1.0, a) * math.copysign(1.0, b)
    a, b = abs(a), abs(b)
    return s * 0.5 * (a * b * (math.log(a * a + b * b) - 3.0)
                      + a * a * math.atan(b / a) + b * b * math.atan(a / b))


def rect_potential(x, y, x0, x1, y0, y1):
    """(1/2pi) int_R log|x-y| dy for the constant density 1 on R (closed form)."""
    return (_F(x1 - x, y1 - y) - _F(x0 - x, y1 - y) - _F(x1 - x, y0 - y)
            + _F(x0 - x, y0 - y)) / (2.0 * math.pi)


def uniform_leaves(level):
    n = 2 ** level
    ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    return [level] * (n * n), ix.ravel().tolist(), iy.ravel().tolist()


def refine_leaves(pred, max_level):
    """Dyadic leaves of [-1,1]^2 obtained by splitting every box where pred(cx,cy,r) holds."""
    out = ([], [], [])
    stack = [(0, 0, 0)]
    while stack:
        lv, i, j = stack.pop()
        r = 1.0 / 2 ** lv
        cx, cy = -1.0 + (2 * i + 1) * r, -1.0 + (2 * j + 1) * r
        if lv < max_level and pred(cx, cy, r):
            for di in (0, 1):
                for dj in (0, 1):
                    stack.append((lv + 1, 2 * i + di, 2 * j + dj))
        else:
            out[0].append(lv)
            out[1].append(i)
            out[2].append(j)
    return out


def test_s_rule_moments(oracle_mod):
    """The Duffy-ray product rule integrates s^(k+1) log s exactly: -1/(k+2)^2."""
    for ns in (16, 24, 32):
        s, wr, wl = oracle_mod.s_rule(ns)
        for k in range(ns):
            assert abs(np.dot(wl, s ** k) + 1.0 / (k + 2) ** 2) < 1e-15
            assert abs(np.dot(wr, s ** k) - 1.0 / (k + 2)) < 1e-15


def test_nodes_are_first_kind_chebyshev(oracle_mod):
    for p in (8, 12, 16):
        x = oracle_mod.cheb_nodes(p)
        assert np.all(np.diff(x) > 0)
        # first-kind points are the roots of T_p
        Tp = C.chebval(x, [0] * p + [1])
        assert np.abs(Tp).max() < 1e-13


def test_interpolant_reproduces_polynomials(oracle_mod):
    """f_B is the tensor interpolant: exact for degree <= p-1 in each variable."""
    rng = np.random.default_rng(5)
    for p in (8, 16):
        c = rng.standard_normal((p, p)) / (1 + np.add.outer(np.arange(p), np.arange(p))) ** 1.5
        x = oracle_mod.cheb_nodes(p)
        X, Y = np.meshgrid(x, x, indexing="xy")   # [jy][jx]
        fv = C.chebval2d(X, Y, c.T)               # c[a][b]: a in x, b in y
        pts = rng.uniform(-1, 1, (50, 2))
        got = oracle_mod.interp(p, fv, pts)
        want = C.chebval2d(pts[:, 0], pts[:, 1], c.T)
        assert np.abs(got - want).max() < 1e-13


def test_centre_of_square(oracle_mod):
    """int_{[-1,1]^2} log|y| dy = 2 ln 2 + pi - 6."""
    for p in (8, 16):
        geom = oracle_mod.leaf_geometry([0], [0], [0])
        u = oracle_mod.potential(p, geom, np.ones((1, p, p)), np.array([[0.0, 0.0]]))
        assert abs(u[0] * 2 * math.pi - (2 * math.log(2) + math.pi - 6)) < 2e-15


def test_constant_density_closed_form(oracle_mod):
    """f = 1 on an adaptive cover of [-1,1]^2: u equals the rectangle formula at
    every node and at off-grid points near edges, corners and outside."""
    p = 12
    lv, ix, iy = refine_leaves(lambda cx, cy, r: abs(cx - 0.3) + abs(cy + 0.2) < 3 * r, 4)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    f = np.ones((len(lv), p, p))
    nodes = oracle_mod.leaf_nodes(geom, p).reshape(-1, 2)
    rng = np.random.default_rng(0)
    pick = nodes[rng.choice(nodes.shape[0], 400, replace=False)]
    extra = np.array([[1.0 + 1e-3, 0.3], [-1.2, -1.0000001], [3.0, 4.0], [0.9999, 0.5],
                      [0.5, 0.5], [0.0, 0.0], [-1.0, -1.0], [0.25, -0.5]])
    pts = np.vstack([pick, extra])
    u = oracle_mod.potential(p, geom, f, pts)
    ex = np.array([rect_potential(x, y, -1, 1, -1, 1) for x, y in pts])
    assert np.abs(u - ex).max() < 1e-14 * np.abs(ex).max()


def _dblquad_leaf(fun, xi, eta):
    """int_{[-1,1]^2} log|x - y| fun(y) dy by scipy dblquad, split at x so that
    the log singularity sits on rectangle corners."""
    import warnings

    from scipy import integrate
    xs = sorted(set([-1.0, 1.0] + ([xi] if -1 < xi < 1 else [])))
    ys = sorted(set([-1.0, 1.0] + ([eta] if -1 < eta < 1 else [])))
    tot = 0.0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for a0, a1 in zip(xs[:-1], xs[1:]):
            for b0, b1 in zip(ys[:-1], ys[1:]):
                v, _ = integrate.dblquad(
                    lambda y, x: 0.5 * np.log((x - xi) ** 2 + (y - eta) ** 2) * fun(x, y),
                    a0, a1, b0, b1, epsabs=1e-15, epsrel=1e-13)
                tot += v
    return tot


def test_one_leaf_against_scipy(oracle_mod):
    """Independent library quadrature on a single leaf with a random polynomial
    density: targets inside (node, near an edge, near a corner), just outside,
    and far away."""
    pytest.importorskip("scipy")
    p = 8
    rng = np.random.default_rng(11)
    c = rng.standard_normal((p, p)) / (1 + np.add.outer(np.arange(p), np.arange(p)))
    x = oracle_mod.cheb_nodes(p)
    X, Y = np.meshgrid(x, x, indexing="xy")
    fv = C.chebval2d(X, Y, c.T)[None]
    geom = oracle_mod.leaf_geometry([0], [0], [0])
    fun = lambda a, b: C.chebval2d(a, b, c.T)
    pts = np.array([[x[2], x[5]], [-0.998, 0.997], [1.003, -0.4], [2.5, -3.0]])
    u = oracle_mod.potential(p, geom, fv, pts)
    ref = np.array([_dblquad_leaf(fun, a, b) for a, b in pts]) / (2 * math.pi)
    assert np.abs(u - ref).max() < 5e-14 * max(1.0, np.abs(ref).max())


def test_gaussian_closed_form(oracle_mod):
    """Radial Gaussian a exp(-r^2/(2 s^2)) far from the root edges (tail < 1e-17):
    u(r) = a s^2 [ln r + E1(r^2/(2 s^2))/2], u(0) = a s^2 [ln(s sqrt 2) - gamma/2]."""
    special = pytest.importorskip("scipy.special")
    p = 16
    a, s, c0 = 1.7, 0.04, np.array([0.1, -0.2])
    lv, ix, iy = refine_leaves(
        lambda cx, cy, r: (math.hypot(cx - c0[0], cy - c0[1]) < 10 * s + 1.5 * r) and r > 0.6 * s, 9)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    nodes = oracle_mod.leaf_nodes(geom, p)
    fvals = a * np.exp(-((nodes[..., 0] - c0[0]) ** 2 + (nodes[..., 1] - c0[1]) ** 2) / (2 * s * s))
    # the interpolant must itself resolve f (checked on random points of each leaf)
    rng = np.random.default_rng(1)
    worst = 0.0
    for b in rng.choice(len(lv), 12, replace=False):
        q = rng.uniform(-1, 1, (20, 2))
        fi = oracle_mod.interp(p, fvals[b], q)
        phys = geom[b, :2] + geom[b, 2] * q
        fe = a * np.exp(-((phys[:, 0] - c0[0]) ** 2 + (phys[:, 1] - c0[1]) ** 2) / (2 * s * s))
        worst = max(worst, np.abs(fi - fe).max())
    assert worst < 1e-12 * a
    pts = np.array([c0, c0 + [0.013, 0.0], c0 + [0.05, -0.07], c0 + [0.3, 0.41], [0.9, 0.9]])
    u = oracle_mod.potential(p, geom, fvals.reshape(len(lv), p, p), pts)
    r = np.hypot(pts[:, 0] - c0[0], pts[:, 1] - c0[1])
    ref = np.empty_like(r)
    ref[0] = a * s * s * (math.log(s * math.sqrt(2.0)) - 0.5772156649015329 / 2)
    ref[1:] = a * s * s * (np.log(r[1:]) + 0.5 * special.exp1(r[1:] ** 2 / (2 * s * s)))
    assert np.abs(u - ref).max() < 5e-13 * np.abs(ref).max()


def test_laplacian_of_potential_is_density(oracle_mod):
    """Laplace(u) = +f on a leaf (sign convention of the paper): spectral second
    derivatives of u at the leaf nodes reproduce f."""
    p = 16
    lv, ix, iy = uniform_leaves(2)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    nodes = oracle_mod.leaf_nodes(geom, p)
    fv = np.exp(-2.0 * ((nodes[..., 0] - 0.2) ** 2 + (nodes[..., 1] + 0.1) ** 2)) * (1 + nodes[..., 0])
    leaf = 5
    u = oracle_mod.potential(p, geom, fv, nodes[leaf]).reshape(p, p)  # [jy][jx]
    x = oracle_mod.cheb_nodes(p)
    V = C.chebvander2d(np.tile(x, p), np.repeat(x, p), [p - 1, p - 1])   # columns (i,j): T_i(x)T_j(y)
    coef = np.linalg.solve(V, u.ravel()).reshape(p, p)               # coef[i][j]
    r = geom[leaf, 2]
    uxx = C.chebder(coef, 2, axis=0) / r ** 2
    uyy = C.chebder(coef, 2, axis=1) / r ** 2
    lap = (C.chebval2d(np.tile(x, p), np.repeat(x, p), np.pad(uxx, ((0, 2), (0, 0))))
           + C.chebval2d(np.tile(x, p), np.repeat(x, p), np.pad(uyy, ((0, 0), (0, 2)))))
    err = np.abs(lap - fv[leaf].ravel()).max() / np.abs(fv).max()
    assert err < 1e-8, err


def test_scaling_law(oracle_mod):
    """Scaling the tree and the density support by s: u_s(s x) = s^2 u(x) + s^2 ln(s) M/(2pi)."""
    p = 8
    lv, ix, iy = refine_leaves(lambda cx, cy, r: cx + cy > -0.5 and r > 0.3, 3)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((len(lv), p, p))
    g1 = oracle_mod.leaf_geometry(lv, ix, iy)
    sc = 0.37
    g2 = oracle_mod.leaf_geometry(lv, ix, iy, x0=-sc, y0=-sc, L=2 * sc)
    pts = rng.uniform(-1.2, 1.2, (30, 2))
    u1 = oracle_mod.potential(p, g1, f, pts)
    u2 = oracle_mod.potential(p, g2, f, sc * pts)
    # M = int f over the unscaled domain, by the leaf quadrature of the oracle's own interpolant
    w1 = oracle_mod.potential(p, g1, f, np.array([[1e6, 0.0]]))
    M = w1[0] * 2 * math.pi / math.log(1e6)   # far field: u -> M log|x| / 2pi (+ O(1/|x|))
    M_exact = sum(np.sum(f[b] * _fejer_tensor(p)) * g1[b, 2] ** 2 for b in range(len(lv)))
    assert abs(M - M_exact) < 1e-5 * abs(M_exact) + 1e-5
    want = sc * sc * u1 + sc * sc * math.log(sc) * M_exact / (2 * math.pi)
    assert np.abs(u2 - want).max() < 1e-14 * np.abs(want).max()


def _fejer_tensor(p):
    """Fejer first-rule weights (exact for degree <= p-1 on first-kind nodes)."""
    th = (2 * np.arange(p) + 1) * math.pi / (2 * p)
    w = np.array([2.0 / p * (1 - 2 * sum(math.cos(2 * k * t) / (4 * k * k - 1) for k in range(1, p // 2 + 1)))
                  for t in th])[::-1]
    return np.outer(w, w)


def test_dihedral_symmetry(oracle_mod):
    """Rotating the tree and the density by 90 degrees rotates the potential."""
    p = 8
    lv, ix, iy = refine_leaves(lambda cx, cy, r: cx > 0.1 and cy < 0.3 and r > 0.2, 3)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((len(lv), p, p))
    g = oracle_mod.leaf_geometry(lv, ix, iy)
    # rotation (x, y) -> (-y, x): leaf (l, i, j) -> (l, 2^l - 1 - j, i); node (jx, jy) -> (p-1-jy, jx)
    lv2 = lv
    ix2 = [2 ** l - 1 - j for l, j in zip(lv, iy)]
    iy2 = list(ix)
    f2 = np.empty_like(f)
    for jy in range(p):
        for jx in range(p):
            f2[:, jx, p - 1 - jy] = f[:, jy, jx]
    g2 = oracle_mod.leaf_geometry(lv2, ix2, iy2)
    pts = rng.uniform(-1.1, 1.1, (25, 2))
    u1 = oracle_mod.potential(p, g, f, pts)
    u2 = oracle_mod.potential(p, g2, f2, np.stack([-pts[:, 1], pts[:, 0]], axis=1))
    assert np.abs(u1 - u2).max() < 1e-14 * np.abs(u1).max()


def test_linearity_and_source_split(oracle_mod):
    """u is linear in f, and restricting sources to complementary sets adds up."""
    p = 8
    lv, ix, iy = uniform_leaves(2)
    g = oracle_mod.leaf_geometry(lv, ix, iy)
    rng = np.random.default_rng(9)
    f1 = rng.standard_normal((16, p, p))
    f2 = rng.standard_normal((16, p, p))
    pts = rng.uniform(-1, 1, (20, 2))
    u1 = oracle_mod.potential(p, g, f1, pts)
    u2 = oracle_mod.potential(p, g, f2, pts)
    u12 = oracle_mod.potential(p, g, 2.0 * f1 - 0.5 * f2, pts)
    assert np.abs(u12 - (2 * u1 - 0.5 * u2)).max() < 1e-14 * np.abs(u12).max()
    A = np.arange(0, 16, 2)
    B = np.arange(1, 16, 2)
    n = pts.shape[0]
    uA = oracle_mod.potential(p, g, f1, pts, sources=(np.arange(n + 1) * len(A), np.tile(A, n)))
    uB = oracle_mod.potential(p, g, f1, pts, sources=(np.arange(n + 1) * len(B), np.tile(B, n)))
    assert np.abs(uA + uB - u1).max() < 1e-14 * np.abs(u1).max()


def _lagrange_1d(p, m, t):
    """l_m(t) on the first-kind Chebyshev nodes, by the product formula
    (independent of the oracle's barycentric interpolation)."""
    k = np.arange(p)
    x = -np.cos((2 * k + 1) * np.pi / (2 * p))
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    for q in range(p):
        if q != m:
            out = out * (t - x[q]) / (x[m] - x[q])
    return out


def test_adjoint_columns_are_the_transpose(oracle_mod):
    """Each adjoint column contracted with the density equals the bilinear form
    <A f, g> taken from the forward oracle: sum_{j in B1, B2} f_j (A^T g)_j =
    <A f_r, g>, f_r = f on leaves B1, B2 and 0 elsewhere (every column of two
    leaves of a 2:1-refined tree, one of them finer).  The restricted form
    (target_leaves) gives the same columns when g vanishes outside those
    leaves.  A layout slip (the (jx, jy) order of a column, the wrong target
    set or a transposed index) fails it."""
    p = 6
    lv, ix, iy = refine_leaves(lambda cx, cy, r: r > 0.9 or (cx < 0 and cy < 0 and r > 0.3), 3)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    n = len(lv)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n, p * p))
    g = rng.standard_normal((n, p * p))
    pick = [int(np.argmax(np.array(lv))), int(np.argmin(np.array(lv)))]   # a fine and a coarse leaf
    assert n == 7 and lv[pick[0]] == 2 and lv[pick[1]] == 1
    fr = np.zeros_like(f)
    fr[pick] = f[pick]
    nodes = oracle_mod.leaf_nodes(geom, p).reshape(-1, 2)
    lhs = float(np.dot(oracle_mod.potential(p, geom, fr, nodes), g.ravel()))
    cols = [(b, j) for b in pick for j in range(p * p)]
    at = oracle_mod.adjoint_columns(p, geom, g, cols)
    rhs = float(np.dot(at, np.concatenate([f[b] for b in pick])))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0), (lhs, rhs)
    # restricted contraction: g supported on a few leaves
    tl = [0, 3, n - 1]
    gs = np.zeros_like(g)
    gs[tl] = g[tl]
    full = oracle_mod.adjoint_columns(p, geom, gs, cols[:12])
    part = oracle_mod.adjoint_columns(p, geom, gs, cols[:12], target_leaves=tl)
    assert np.abs(full - part).max() <= 1e-15 * np.abs(full).max()


def test_adjoint_column_against_scipy(oracle_mod):
    """One column of A^T on a single leaf against scipy dblquad of the Lagrange
    basis function: (A^T e_i)_j = (1/2pi) int log|x_i - y| l_j(y) dy for a
    target node i inside the leaf, with j = (jx, jy) off the diagonal so that a
    swapped x/y order of the column would show."""
    pytest.importorskip("scipy")
    p = 4
    geom = oracle_mod.leaf_geometry([0], [0], [0])
    x = oracle_mod.cheb_nodes(p)
    jx, jy, i = 1, 3, 6              # column node (x index 1, y index 3); target node 6 = (2, 1)
    j = jy * p + jx
    g = np.zeros((1, p * p))
    g[0, i] = 1.0
    got = oracle_mod.adjoint_columns(p, geom, g, [(0, j)])[0]
    xi, eta = x[i % p], x[i // p]
    ref = _dblquad_leaf(lambda a, b: _lagrange_1d(p, jx, a) * _lagrange_1d(p, jy, b), xi, eta) / (2 * math.pi)
    assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref)), (got, ref)


def _Fa(a, b):
    """d/da of _F: int_0^b (1/2) log(a^2 + t^2) dt (closed form, signed b)."""
    if b == 0.0:
        return 0.0
    if a == 0.0:
        return 0.5 * (b * math.log(b * b) - 2.0 * b)
    return 0.5 * (b * math.log(a * a + b * b) - 2.0 * b + 2.0 * a * math.atan(b / a))


def rect_gradient(x, y, x0, x1, y0, y1):
    """Gradient of rect_potential (closed form): d/dx and d/dy of
    (1/2pi) [F(x1-x, y1-y) - F(x0-x, y1-y) - F(x1-x, y0-y) + F(x0-x, y0-y)]."""
    gx = (-_Fa(x1 - x, y1 - y) + _Fa(x0 - x, y1 - y) + _Fa(x1 - x, y0 - y) - _Fa(x0 - x, y0 - y))
    gy = (-_Fa(y1 - y, x1 - x) + _Fa(y1 - y, x0 - x) + _Fa(y0 - y, x1 - x) - _Fa(y0 - y, x0 - x))
    return np.array([gx, gy]) / (2.0 * math.pi)


def test_gradient_constant_density_closed_form(oracle_mod):
    """The oracle's gradient of the potential of f = 1 on a 2:1-refined tree
    against the closed form, at targets inside leaves (at a node, near an edge,
    near a corner), on a shared edge, and outside the root."""
    p = 8
    lv, ix, iy = refine_leaves(lambda cx, cy, r: r > 0.9 or (cx > 0 and cy > 0 and r > 0.3), 3)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    f = np.ones((len(lv), p, p))
    x = oracle_mod.cheb_nodes(p)
    pts = np.array([[-0.5 + 0.5 * x[3], -0.5 + 0.5 * x[5]], [0.2, 0.999], [0.999, -0.998], [0.0, 0.37],
                    [0.75, 0.26], [1.6, -0.3], [-2.5, 1.8]])
    g = oracle_mod.gradient(p, geom, f, pts)
    ref = np.array([rect_gradient(a, b, -1.0, 1.0, -1.0, 1.0) for a, b in pts])
    assert np.abs(g - ref).max() < 1e-13 * np.abs(ref).max(), np.abs(g - ref).max()


def test_gradient_gaussian_closed_form(oracle_mod):
    """Radial Gaussian a exp(-r^2/(2 s^2)): grad u = u'(r) (x - c)/r with
    u'(r) = a s^2 (1 - exp(-r^2/(2 s^2)))/r (derivative of the E1 form)."""
    p = 16
    a, s, c0 = 1.7, 0.04, np.array([0.1, -0.2])
    lv, ix, iy = refine_leaves(
        lambda cx, cy, r: (math.hypot(cx - c0[0], cy - c0[1]) < 10 * s + 1.5 * r) and r > 0.6 * s, 9)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    nodes = oracle_mod.leaf_nodes(geom, p)
    fvals = a * np.exp(-((nodes[..., 0] - c0[0]) ** 2 + (nodes[..., 1] - c0[1]) ** 2) / (2 * s * s))
    pts = np.array([c0 + [0.013, 0.0], c0 + [0.05, -0.07], c0 + [-0.021, 0.033], c0 + [0.3, 0.41], [0.9, 0.9]])
    g = oracle_mod.gradient(p, geom, fvals.reshape(len(lv), p, p), pts)
    d = pts - c0
    r = np.hypot(d[:, 0], d[:, 1])
    up = a * s * s * (1.0 - np.exp(-r ** 2 / (2 * s * s))) / r
    ref = up[:, None] * d / r[:, None]
    assert np.abs(g - ref).max() < 1e-12 * np.abs(ref).max(), np.abs(g - ref).max()


def test_gradient_matches_differences_of_the_potential(oracle_mod):
    """Central differences of the pinned potential (step 1e-4, O(h^2)) agree
    with the gradient for a random polynomial density on a 2:1 tree, at targets
    inside leaves and away from them.  (The density jumps across leaf edges, so
    u is only C^1 there and differences across an edge are O(h); targets on
    edges are pinned by the closed form above.)"""
    p = 8
    lv, ix, iy = refine_leaves(lambda cx, cy, r: r > 0.9 or (cx < 0 and cy > 0 and r > 0.3), 3)
    geom = oracle_mod.leaf_geometry(lv, ix, iy)
    rng = np.random.default_rng(4)
    f = rng.standard_normal((len(lv), p, p))
    pts = np.array([[-0.3, 0.41], [0.52, -0.77], [0.07, 0.123], [-0.63, 0.62], [1.4, 0.2]])
    h = 1e-4
    fd = np.zeros_like(pts)
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd[:, k] = (oracle_mod.potential(p, geom, f, pts + e) - oracle_mod.potential(p, geom, f, pts - e)) / (2 * h)
    g = oracle_mod.gradient(p, geom, f, pts)
    assert np.abs(g - fd).max() < 1e-6 * np.abs(g).max(), np.abs(g - fd).max()


# ---------------------------------------------------------------------------
# Glue layer potential (Sec. 3.4): closed forms on a circle and Gauss's
# identity on the star-shaped fictitious curve.
# ---------------------------------------------------------------------------
def _circle(n, R, c):
    th = 2 * np.pi * np.arange(n) / n
    nrm = np.stack([np.cos(th), np.sin(th)], 1)
    return np.asarray(c) + R * nrm, np.full(n, 2 * np.pi * R / n), nrm


def test_layer_single_layer_circle_closed_form(oracle_mod):
    """S[1] on a circle of radius R: -R log R inside, -R log|x - c| outside
    (trapezoid rule, geometrically convergent away from the curve)."""
    R, c = 0.7, np.array([0.1, -0.05])
    src, w, nrm = _circle(400, R, c)
    rng = np.random.default_rng(1)
    ang = rng.uniform(0, 2 * np.pi, 20)
    rad_in, rad_out = rng.uniform(0, 0.5 * R, 20), rng.uniform(1.6 * R, 4 * R, 20)
    pin = c + rad_in[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    pout = c + rad_out[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    zero = np.zeros_like(src)
    uin = oracle_mod.layer(src, w, zero, pin)
    uout = oracle_mod.layer(src, w, zero, pout)
    assert np.allclose(uin, -R * np.log(R), rtol=0, atol=1e-13)
    assert np.allclose(uout, -R * np.log(rad_out), rtol=0, atol=1e-13)


def test_layer_double_layer_gauss_identity(oracle_mod):
    """-D[1] = 1 inside a closed curve and 0 outside (Gauss), on a circle and
    on the Gauss-Legendre panels of the star-shaped fictitious curve; with
    a sign flip of the normals the interior value flips too."""
    R, c = 0.6, np.array([-0.2, 0.15])
    src, w, nrm = _circle(300, R, c)
    m = w[:, None] * nrm
    pts = np.array([c, c + [0.2, 0.1], c + [1.5, 0.0], c + [-0.9, 0.7]])
    u = oracle_mod.layer(src, np.zeros(len(w)), m, pts)
    assert np.allclose(u, [1, 1, 0, 0], rtol=0, atol=1e-13)
    assert np.allclose(oracle_mod.layer(src, np.zeros(len(w)), -m, pts[:2]), [-1, -1], atol=1e-13)
    # Gauss-Legendre panels on r(t) = 0.72 + 0.1 cos 5t (counterclockwise)
    g, gw = np.polynomial.legendre.leggauss(16)
    h = 2 * np.pi / 128
    t = ((np.arange(128)[:, None] + 0.5) * h + 0.5 * h * g[None, :]).ravel()
    r, dr = 0.72 + 0.1 * np.cos(5 * t), -0.5 * np.sin(5 * t)
    xy = np.stack([r * np.cos(t), r * np.sin(t)], 1)
    d = np.stack([dr * np.cos(t) - r * np.sin(t), dr * np.sin(t) + r * np.cos(t)], 1)
    sp = np.linalg.norm(d, axis=1)
    ws, ns = np.tile(0.5 * h * gw, 128) * sp, np.stack([d[:, 1], -d[:, 0]], 1) / sp[:, None]
    pts = np.array([[0.0, 0.0], [0.3, -0.2], [1.2, 0.4], [-0.95, -0.9]])
    u = oracle_mod.layer(xy, np.zeros(len(ws)), ws[:, None] * ns, pts)
    assert np.allclose(u, [1, 1, 0, 0], rtol=0, atol=1e-12)


def test_layer_linearity_and_coincident_source(oracle_mod):
    """Charges and dipoles add; a target on a source node skips that pair
    only (the rest of the sum is unchanged)."""
    rng = np.random.default_rng(4)
    src = rng.uniform(-1, 1, (30, 2))
    q, m = rng.standard_normal(30), rng.standard_normal((30, 2))
    t = np.vstack([rng.uniform(-1, 1, (5, 2)), src[7:8]])
    both = oracle_mod.layer(src, q, m, t)
    sep = oracle_mod.layer(src, q, 0 * m, t) + oracle_mod.layer(src, 0 * q, m, t)
    assert np.allclose(both, sep, rtol=1e-14, atol=1e-14)
    keep = np.arange(30) != 7
    assert np.isclose(both[-1], oracle_mod.layer(src[keep], q[keep], m[keep], t[-1:])[0], rtol=1e-14)


# ---------------------------------------------------------------------------
# Strip solve (Sec. 3.3): block-tridiagonal system with periodic corners.
# ---------------------------------------------------------------------------
def test_strip_block_circulant_by_dft(oracle_mod):
    """Identical blocks (A, B, C) on every element: the system is block
    circulant, so the block DFT diagonalises it: x_hat_j = (A + B w^j +
    C w^-j)^-1 b_hat_j with w = exp(2 pi i / N).  Fails on a swapped B/C or a
    corner placed on the wrong side."""
    rng = np.random.default_rng(21)
    for N, m in ((7, 3), (2, 4), (1, 2), (16, 5)):
        A0 = rng.standard_normal((m, m)) + 4 * m * np.eye(m)
        B0, C0 = rng.standard_normal((m, m)), 0.5 * rng.standard_normal((m, m))
        b = rng.standard_normal((N, m, 2))
        x = oracle_mod.strip_solve(np.tile(A0, (N, 1, 1)), np.tile(B0, (N, 1, 1)), np.tile(C0, (N, 1, 1)), b)
        bh = np.fft.fft(b, axis=0)
        w = np.exp(2j * np.pi * np.arange(N) / N)
        xh = np.stack([np.linalg.solve(A0 + B0 * w[j] + C0 / w[j], bh[j]) for j in range(N)])
        assert np.allclose(x, np.fft.ifft(xh, axis=0).real, rtol=0, atol=1e-12), (N, m)


def test_strip_periodic_second_difference(oracle_mod):
    """m = 1, A = 2 + h^2, B = C = -1: the periodic discretisation of
    -u'' + u = f on N points; for f = cos(2 pi s / N) the exact discrete
    solution is f / (2 - 2 cos(2 pi / N) + h^2)."""
    N, h = 40, 0.1
    s = np.arange(N)
    f = np.cos(2 * np.pi * s / N)[:, None, None]
    one = np.ones((N, 1, 1))
    x = oracle_mod.strip_solve((2 + h * h) * one, -one, -one, f)
    exact = f / (2 - 2 * np.cos(2 * np.pi / N) + h * h)
    assert np.abs(x - exact).max() <= 1e-13 * np.abs(exact).max()
