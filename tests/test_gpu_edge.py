"""Edge cases of the volume apply (eq. (vbulk), Sec. 3.2) against the oracle,
FP64 and split, forward and adjoint:

  - degenerate trees: the root as the only leaf, the uniform levels 1 and 2
    (everything near; the first level with V lists but no climb);
  - a deep tree, leaves down to level 18 around a narrow Gaussian (per-level
    r^2 down to 1.5e-11 and log r down to -12.5; the oracle integrates the
    same leaf interpolants, so the Gaussian need not be resolved);
  - a root box other than [-1,1]^2 (x0 = 3.5, y0 = -7.25, L = 5): the
    potential carries the scaling law's log L term;
  - zero input gives exactly zero output; the adjoint satisfies the
    dot-product identity on each tree.

Bar: 1e-10 relative max-norm against the oracle (Sec. 4's tolerance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

P = 16
TOL = 1e-10
MODES = [bc.FP64, bc.SPLIT_BF16]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return bc.Context(p=P, nterms=24, device=0)


def _check(tree, lv, ix, iy, g, x0=-1.0, y0=-1.0, L=2.0, pick=None):
    geom = synth.leaf_geometry(lv, ix, iy, x0, y0, L)
    nodes = oracle.leaf_nodes(geom, P)
    fv = g(nodes.reshape(-1, 2)).reshape(-1, P * P)
    f = torch.from_numpy(fv.reshape(-1)).cuda()
    if pick is None:
        pick = np.arange(len(lv))
    ref = oracle.potential_at_nodes(P, geom, fv, leaf_ids=pick)
    rng = np.random.default_rng(len(lv))
    gr = torch.from_numpy(rng.standard_normal(fv.size)).cuda()
    worst = 0.0
    for mode in MODES:
        u = bc.apply(tree, f, precision=mode)
        un = u.cpu().numpy().reshape(-1, P * P)
        err = float(np.abs(un[pick] - ref).max() / np.abs(ref).max())
        worst = max(worst, err)
        assert err < TOL, (mode, err)
        # the adjoint: <A f, g> = <f, A^T g>
        h = bc.apply_adjoint(tree, gr, precision=mode)
        lhs, rhs = torch.dot(u, gr).item(), torch.dot(f, h).item()
        scale = (u.abs() * gr.abs()).sum().item()
        assert abs(lhs - rhs) <= 1e-10 * scale, (mode, lhs, rhs)
        z = bc.apply(tree, torch.zeros_like(f), precision=mode)
        assert torch.count_nonzero(z).item() == 0
    return worst


@pytest.mark.parametrize("level", [0, 1, 2])
def test_uniform_degenerate_levels(ctx, level):
    lv, ix, iy = synth.uniform_leaves(level)
    tree = bc.Tree(ctx, lv, ix, iy)
    err = _check(tree, lv, ix, iy, synth.config_density(1))
    print(f"uniform level {level} ({len(lv)} leaves): {err:.2e}")


def test_deep_tree(ctx):
    g = synth.GaussianSum(np.array([0.1234]), np.array([-0.3717]), np.array([5e-6]), np.array([1.0]))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=18)
    assert int(np.max(lv)) == 18
    tree = bc.Tree(ctx, lv, ix, iy)
    deep = np.nonzero(lv >= 15)[0]
    pick = np.unique(np.concatenate([deep[:6], synth.sample_leaves_per_level(lv, 1, seed=2)]))
    err = _check(tree, lv, ix, iy, g, pick=pick)
    print(f"deep tree ({len(lv)} leaves, levels {lv.min()}..{lv.max()}): {err:.2e}")


def test_shifted_scaled_root(ctx):
    x0, y0, L = 3.5, -7.25, 5.0
    lv, ix, iy = synth.uniform_leaves(3)
    g0 = synth.config_density(1)
    # the same Gaussians mapped into the new root box

    def g(xy):
        ref = (np.asarray(xy) - np.array([x0, y0])) * (2.0 / L) - 1.0
        return g0(ref)
    tree = bc.Tree(ctx, lv, ix, iy, x0=x0, y0=y0, L=L)
    err = _check(tree, lv, ix, iy, g, x0, y0, L)
    print(f"root [{x0},{x0 + L}] x [{y0},{y0 + L}]: {err:.2e}")


@pytest.mark.parametrize("p", [8, 12])
def test_split_orders_8_12(p):
    """Split precision at p = 8 (64 nodes: the tensor kernel's K = 64 tiles)
    and p = 12 (144 nodes, zero-padded to K = 256; near-field operators of 144
    rows in two jobs) on an adaptive tree, forward and adjoint, against the
    oracle at every node of sampled leaves (levels 2 and up) and by the
    dot-product identity; the same bar as p = 16."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = bc.Context(p=p, nterms=24, device=0)
    g = synth.config_density(1)
    tree = bc.Tree.refine(c, g, eps=1e-10, max_level=10)
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    geom = synth.leaf_geometry(lv, ix, iy)
    nodes = oracle.leaf_nodes(geom, p)
    fv = g(nodes.reshape(-1, 2)).reshape(-1, p * p)
    f = torch.from_numpy(fv.reshape(-1)).cuda()
    pick = synth.sample_leaves_per_level(lv, 1, seed=p)
    ref = oracle.potential_at_nodes(p, geom, fv, leaf_ids=pick)
    u = bc.apply(tree, f, precision=bc.SPLIT_BF16)
    err = float(np.abs(u.cpu().numpy().reshape(-1, p * p)[pick] - ref).max() / np.abs(ref).max())
    u64 = bc.apply(tree, f)
    d64 = float(((u - u64).abs().max() / u64.abs().max()).item())
    gr = torch.from_numpy(np.random.default_rng(p).standard_normal(fv.size)).cuda()
    h = bc.apply_adjoint(tree, gr, precision=bc.SPLIT_BF16)
    h64 = bc.apply_adjoint(tree, gr)
    da = float(((h - h64).abs().max() / h64.abs().max()).item())
    lhs, rhs = torch.dot(u, gr).item(), torch.dot(f, h).item()
    scale = (u.abs() * gr.abs()).sum().item()
    print(f"split p={p} ({tree.nleaf} leaves): oracle {err:.2e}, vs FP64 forward {d64:.2e} adjoint {da:.2e}")
    assert err < TOL, err
    assert d64 < 1e-10 and da < 1e-10, (d64, da)
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)
