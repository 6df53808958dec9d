"""GPU parity of the transposed operator and of per-level results against the oracle.

* The adjoint apply h = A^T g, in every precision mode, against the oracle's
  transposed operator (columns (A^T g)_j = sum_i g_i A_ij with
  A_ij = (1/2pi) int_B(j) log|x_i - y| l_j(y) dy, the discrete form of
  eq. (vbulk), Sec. 3.2).  g is random on a set S of leaves and zero
  elsewhere, so the oracle needs the targets of S only; S holds the sampled
  column leaves and every leaf touching them (near-field adjoint) plus random
  leaves (far-field adjoint), and further column leaves are drawn on every
  level regardless of S.
* A tree from the library's own Alg. 2 refinement (20 Gaussians, eps 1e-11):
  forward and adjoint, every mode, error per level.
* A tree of 114,688 leaves (p = 16) with a Gaussian-sum density whose
  centres, widths and amplitudes are torch parameters: gradients of
  0.5 ||u - u_t||^2 through the autograd Function against central finite
  differences (h = 1e-6) on 8 random parameters, the transposed operator on
  sampled oracle columns, and the dot-product identity.
Error metric: max |x - x*| / max |x*| over the evaluated entries; bar 1e-10
(the accuracy the paper reports for its solver, Sec. 4).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10
P = 16
MODES = pytest.mark.parametrize("mode", [bc.FP64, bc.SPLIT_BF16, bc.SPLIT_BF16_ALL], ids=["fp64", "split", "split_all"])


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return bc.Context(p=P, nterms=24, device=0)


def touching(lv, ix, iy, t):
    """Leaves that touch leaf t across an edge or a corner, t included
    (computed from the dyadic indices, independently of the library's lists)."""
    lv, ix, iy = (np.asarray(a, dtype=np.int64) for a in (lv, ix, iy))
    L = int(lv.max())
    s = L - lv
    x0, x1 = ix << s, (ix + 1) << s
    y0, y1 = iy << s, (iy + 1) << s
    ok = (x0 <= x1[t]) & (x0[t] <= x1) & (y0 <= y1[t]) & (y0[t] <= y1)
    return np.nonzero(ok)[0]


def adjoint_sample(lv, ix, iy, seed, per_level=1, k_cols=3, n_rand=24):
    """(S, columns): S = sampled column leaves, their touching leaves and random
    leaves; columns = k_cols random nodes of per_level leaves of every level in
    S's sample and of as many more drawn independently (mostly far from S)."""
    rng = np.random.default_rng(seed)
    levels = np.asarray(lv)
    near_cols = synth.sample_leaves_per_level(levels, per_level, seed=seed)
    far_cols = synth.sample_leaves_per_level(levels, per_level, seed=seed + 1)
    S = set()
    for b in near_cols:
        S.update(touching(lv, ix, iy, int(b)).tolist())
    S.update(rng.choice(len(lv), size=min(n_rand, len(lv)), replace=False).tolist())
    cols = []
    for b in np.concatenate([near_cols, far_cols]):
        for j in rng.choice(P * P, size=k_cols, replace=False):
            cols.append((int(b), int(j)))
    return np.array(sorted(S), dtype=np.int64), cols


def per_level(levels, err_rows, scale):
    """{level: max error of the rows at that level / scale}."""
    out = {}
    for lvl, e in zip(levels, err_rows):
        out[int(lvl)] = max(out.get(int(lvl), 0.0), float(e) / scale)
    return out


def check_adjoint(tree, lv, ix, iy, modes, seed):
    geom = synth.leaf_geometry(lv, ix, iy)
    S, cols = adjoint_sample(lv, ix, iy, seed)
    rng = np.random.default_rng(seed + 7)
    g = np.zeros((len(lv), P * P))
    g[S] = rng.standard_normal((len(S), P * P))
    ref = oracle.adjoint_columns(P, geom, g, cols, target_leaves=S)
    gd = torch.from_numpy(g).cuda()
    res = {}
    for mode in modes:
        h = bc.apply_adjoint(tree, gd, precision=mode).cpu().numpy().reshape(-1, P * P)
        got = np.array([h[b, j] for b, j in cols])
        scale = np.abs(ref).max()
        levels = [lv[b] for b, _ in cols]
        res[mode] = (float(np.abs(got - ref).max() / scale), per_level(levels, np.abs(got - ref), scale))
    bc._check(bc._load().bc_sync(tree.ctx.handle, None))
    return res


@pytest.fixture(scope="module")
def adaptive(ctx):
    g = synth.gaussians(8, 21, wlog10=(-2.3, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=9)
    return bc.Tree(ctx, lv, ix, iy), lv, ix, iy


@MODES
def test_adjoint_against_oracle_columns(ctx, adaptive, mode):
    """A^T g on the adaptive test tree (2194 leaves, 10 levels, W and X lists)
    against oracle columns, near and far, on every level."""
    tree, lv, ix, iy = adaptive
    st = tree.stats()
    assert st["n_w"] > 0 and st["n_x"] > 0
    err, lvl = check_adjoint(tree, lv, ix, iy, [mode], seed=31)[mode]
    print(f"adjoint mode {mode}: {err:.2e}; per level " + " ".join(f"{k}:{v:.1e}" for k, v in sorted(lvl.items())))
    assert err < TOL, (err, lvl)


@pytest.fixture(scope="module")
def alg2(ctx):
    """The 20-Gaussian density refined by the library (Alg. 2, eps 1e-11)."""
    g = synth.config_density(2)
    tree = bc.Tree.refine(ctx, g, eps=1e-11, max_level=18)
    lv, ix, iy = tree.leaves()
    return tree, g, np.asarray(lv), np.asarray(ix), np.asarray(iy)


@MODES
def test_alg2_tree_forward_and_adjoint_per_level(ctx, alg2, mode):
    """Forward at every node of 2 leaves per level, and adjoint columns, on the
    library-refined tree (1330 leaves, 11 levels), against the oracle."""
    tree, g, lv, ix, iy = alg2
    geom = synth.leaf_geometry(lv, ix, iy)
    fvals = g(oracle.leaf_nodes(geom, P))
    pick = synth.sample_leaves_per_level(lv, 2, seed=41)
    ref = oracle.potential_at_nodes(P, geom, fvals, leaf_ids=pick)
    u = bc.apply(tree, torch.from_numpy(fvals).cuda(), precision=mode).cpu().numpy().reshape(-1, P * P)
    scale = np.abs(ref).max()
    fwd = float(np.abs(u[pick] - ref).max() / scale)
    fwd_lvl = per_level(lv[pick], np.abs(u[pick] - ref).max(axis=1), scale)
    adj, adj_lvl = check_adjoint(tree, lv, ix, iy, [mode], seed=43)[mode]
    print(f"alg2 tree mode {mode}: forward {fwd:.2e} adjoint {adj:.2e}")
    print("  forward per level " + " ".join(f"{k}:{v:.1e}" for k, v in sorted(fwd_lvl.items())))
    print("  adjoint per level " + " ".join(f"{k}:{v:.1e}" for k, v in sorted(adj_lvl.items())))
    assert fwd < TOL and adj < TOL, (fwd, adj)


def big_leaves():
    """114,688 leaves: the uniform level-8 tree with its lower-left quadrant at
    level 9 (2:1 balanced: adjacent leaves differ by at most one level)."""
    lv8, ix8, iy8 = synth.uniform_leaves(8)
    keep = ~((ix8 < 128) & (iy8 < 128))
    lv9, ix9, iy9 = synth.uniform_leaves(9)
    sel = (ix9 < 256) & (iy9 < 256)
    lv = np.concatenate([lv8[keep], lv9[sel]])
    ix = np.concatenate([ix8[keep], ix9[sel]])
    iy = np.concatenate([iy8[keep], iy9[sel]])
    return lv, ix, iy


def test_gradients_on_a_large_tree(ctx):
    """Config-5 scale: dL/dtheta through BoxCodeApply (split and FP64) against
    central differences on 8 random parameters; the split adjoint against 24
    oracle columns; <A f, g> = <f, A^T g>."""
    lv, ix, iy = big_leaves()
    assert len(lv) == 114688
    tree = bc.Tree(ctx, lv, ix, iy)
    geom = synth.leaf_geometry(lv, ix, iy)
    nodes = torch.from_numpy(oracle.leaf_nodes(geom, P)).cuda()
    g0 = synth.gaussians(6, 3, wlog10=(-1.6, -1.0))
    theta0 = torch.tensor(np.c_[g0.cx, g0.cy, np.log(g0.w), g0.a], device="cuda")

    def density(th):
        x, y = nodes[..., 0], nodes[..., 1]
        f = torch.zeros_like(x)
        for k in range(th.shape[0]):
            w = torch.exp(th[k, 2])
            f = f + th[k, 3] * torch.exp(-((x - th[k, 0]) ** 2 + (y - th[k, 1]) ** 2) / (2 * w * w))
        return f.contiguous()

    gen = torch.Generator(device="cuda").manual_seed(3)
    with torch.no_grad():
        ut = bc.apply(tree, density(theta0 + 1e-2 * torch.randn(theta0.shape, generator=gen, device="cuda",
                                                                 dtype=torch.float64)))
    rng = np.random.default_rng(5)
    params = [(int(i), int(j)) for i, j in zip(rng.integers(0, 6, 8), rng.integers(0, 4, 8))]
    for mode, tol in ((bc.SPLIT_BF16, 1e-5), (bc.FP64, 1e-6)):
        def loss(th):
            u = bc.BoxCodeApply.apply(density(th), tree, mode)
            return 0.5 * ((u - ut) ** 2).sum()

        th = theta0.clone().requires_grad_(True)
        loss(th).backward()
        grad = th.grad.detach()
        h = 1e-6
        fd, an = [], []
        for (i, j) in params:
            e = torch.zeros_like(theta0)
            e[i, j] = h
            with torch.no_grad():
                fd.append(((loss(theta0 + e) - loss(theta0 - e)) / (2 * h)).item())
            an.append(grad[i, j].item())
        fd, an = np.array(fd), np.array(an)
        rel = float(np.abs(fd - an).max() / np.abs(an).max())
        print(f"large tree mode {mode}: FD vs adjoint gradient {rel:.2e}")
        assert rel < tol, (mode, rel, fd, an)
    # the split adjoint against oracle columns (g random on a few leaves)
    S = np.sort(rng.choice(len(lv), size=48, replace=False))
    cols = [(int(b), int(j)) for b, j in zip(rng.choice(S, 12), rng.integers(0, P * P, 12))]
    cols += [(int(b), int(j)) for b, j in zip(rng.integers(0, len(lv), 12), rng.integers(0, P * P, 12))]
    gv = np.zeros((len(lv), P * P))
    gv[S] = rng.standard_normal((len(S), P * P))
    ref = oracle.adjoint_columns(P, geom, gv, cols, target_leaves=S)
    hs = bc.apply_adjoint(tree, torch.from_numpy(gv).cuda(), precision=bc.SPLIT_BF16).cpu().numpy()
    got = np.array([hs.reshape(-1, P * P)[b, j] for b, j in cols])
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"large tree split adjoint vs oracle columns {err:.2e}")
    assert err < TOL, err
    # dot-product identity (FP64 operator)
    fr = torch.randn((len(lv), P * P), generator=gen, device="cuda", dtype=torch.float64)
    gr = torch.randn((len(lv), P * P), generator=gen, device="cuda", dtype=torch.float64)
    lhs = torch.dot(bc.apply(tree, fr).ravel(), gr.ravel()).item()
    rhs = torch.dot(fr.ravel(), bc.apply_adjoint(tree, gr).ravel()).item()
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs)), (lhs, rhs)
    bc._check(bc._load().bc_sync(ctx.handle, None))
