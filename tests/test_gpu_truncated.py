"""The truncated box code on the GPU against the oracle (Alg. 2 with both
criteria, keep-cut boxes: Sec. 3.2.1 and its remark on cut boxes).

On a star-shaped domain with a fictitious curve inside it, f is the
20-Gaussian density extended by zero outside the domain.  The applies (FP64
and split) are compared with the oracle's potential of the same zero-extended
node values at every node of sampled active leaves (cut leaves included), and
the adjoint with oracle columns of active leaves.  Discarded leaves (outside
the domain) give exactly zero and their input values are ignored, in both
directions.  Bar: 1e-10 relative max-norm (Sec. 4)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10
P = 16


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=P, nterms=24, device=0)
    gamma, gamma_b = synth.star_domain()
    g = synth.config_density(2)
    tree = bc.Tree.refine_truncated(ctx, g, gamma, gamma_b, eps=1e-11, max_level=18)
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    cls = tree.leaf_class()
    mask = tree.node_mask().astype(bool)
    fz = np.where(mask, g(tree.nodes()), 0.0)
    return ctx, tree, lv, ix, iy, cls, fz


@pytest.mark.parametrize("mode", [bc.FP64, bc.SPLIT_BF16], ids=["fp64", "split"])
def test_truncated_forward_against_oracle(setup, mode):
    ctx, tree, lv, ix, iy, cls, fz = setup
    assert (cls == 0).any() and (cls == 1).any()
    f = torch.from_numpy(fz).cuda()
    u = bc.apply(tree, f, precision=mode).cpu().numpy()
    assert np.all(u[cls == 0] == 0.0)
    # input at discarded leaves is ignored
    fg = fz.copy()
    fg[cls == 0] = 1e3
    ug = bc.apply(tree, torch.from_numpy(fg).cuda(), precision=mode).cpu().numpy()
    assert np.array_equal(u, ug)
    act = np.nonzero(cls != 0)[0]
    pick = np.unique(np.concatenate([act[synth.sample_leaves_per_level(lv[act], 2, seed=3)],
                                     np.nonzero(cls == 1)[0][:4]]))
    geom = synth.leaf_geometry(lv, ix, iy)
    ref = oracle.potential_at_nodes(P, geom, fz, leaf_ids=pick)
    err = float(np.abs(u[pick] - ref).max() / np.abs(ref).max())
    print(f"truncated tree ({tree.nleaf} leaves, {int((cls == 0).sum())} discarded, {int((cls == 1).sum())} cut) "
          f"mode {mode}: forward {err:.2e}")
    assert err < TOL, err
    bc._check(bc._load().bc_sync(ctx.handle, None))


@pytest.mark.parametrize("mode", [bc.FP64, bc.SPLIT_BF16], ids=["fp64", "split"])
def test_truncated_adjoint_against_oracle(setup, mode):
    ctx, tree, lv, ix, iy, cls, fz = setup
    rng = np.random.default_rng(9)
    act = np.nonzero(cls != 0)[0]
    S = np.sort(rng.choice(act, size=40, replace=False))
    gv = np.zeros((tree.nleaf, P * P))
    gv[S] = rng.standard_normal((len(S), P * P))
    h = bc.apply_adjoint(tree, torch.from_numpy(gv).cuda(), precision=mode).cpu().numpy().reshape(-1, P * P)
    assert np.all(h[cls == 0] == 0.0)
    gg = gv.copy()
    gg[cls == 0] = 1e3   # ignored
    hg = bc.apply_adjoint(tree, torch.from_numpy(gg).cuda(), precision=mode).cpu().numpy().reshape(-1, P * P)
    assert np.array_equal(h, hg)
    cols = [(int(b), int(j)) for b, j in zip(np.r_[S[:8], rng.choice(act, 8)], rng.integers(0, P * P, 16))]
    geom = synth.leaf_geometry(lv, ix, iy)
    ref = oracle.adjoint_columns(P, geom, gv, cols, target_leaves=S)
    got = np.array([h[b, j] for b, j in cols])
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"truncated tree mode {mode}: adjoint {err:.2e}")
    assert err < TOL, err
    bc._check(bc._load().bc_sync(ctx.handle, None))
