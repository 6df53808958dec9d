"""Batched applies: many trees of uneven size in one launch per pass (union of
trees, CUDA graph, autotuned launch shapes) must reproduce the single-tree
applies, forward and adjoint, FP64 and split precision; and a sampled leaf of
each order is checked against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch_setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctxs = {p: bc.Context(p=p, device=0) for p in (8, 12, 16)}
    per_p = {8: [], 12: [], 16: []}
    for k in range(12):
        g, p, eps = synth.batch_density(k)
        tree = bc.Tree.refine(ctxs[p], g, eps=eps, max_level=16)
        f = torch.from_numpy(g(tree.nodes())).cuda()
        per_p[p].append((tree, g, f))
    return ctxs, per_p


@pytest.mark.parametrize("p", [8, 12, 16])
def test_batch_matches_single_tree_applies(batch_setup, p):
    ctxs, per_p = batch_setup
    items = per_p[p]
    batch = bc.Batch(ctxs[p], [t for t, _, _ in items])
    assert batch.nleaf == sum(t.nleaf for t, _, _ in items)
    precs = [bc.FP64] + ([bc.SPLIT_BF16] if p in bc.SPLIT_ORDERS else [])
    for prec in precs:
        for adjoint in (False, True):
            outs = [torch.full_like(f, float("nan")) for _, _, f in items]
            batch.run([f for _, _, f in items], outs, precision=prec, adjoint=adjoint)
            outs2 = [torch.empty_like(f) for _, _, f in items]
            batch.run([f for _, _, f in items], outs2, precision=prec, adjoint=adjoint)   # graph replay
            for (t, _, f), o, o2 in zip(items, outs, outs2):
                ref = bc.apply_adjoint(t, f, precision=prec) if adjoint else bc.apply(t, f, precision=prec)
                err = ((o - ref).abs().max() / ref.abs().max()).item()
                assert err <= 1e-13, (p, prec, adjoint, err)
                assert torch.equal(o, o2)


def test_batch_autotune_and_oracle(batch_setup):
    ctxs, per_p = batch_setup
    items = per_p[16]
    batch = bc.Batch(ctxs[16], [t for t, _, _ in items])
    shapes = batch.autotune(bc.SPLIT_BF16)
    assert all(s[0] > 0 and s[1] > 0 for s in shapes.values())
    outs = [torch.empty_like(f) for _, _, f in items]
    batch.run([f for _, _, f in items], outs, precision=bc.SPLIT_BF16)
    for (t, g, f), o in list(zip(items, outs))[:2]:
        lv, ix, iy = t.leaves()
        geom = synth.leaf_geometry(lv, ix, iy)
        pick = synth.sample_leaves(t.nleaf, 3, seed=1)
        ref = oracle.potential_at_nodes(16, geom, f.cpu().numpy().reshape(-1, 16, 16), leaf_ids=pick)
        got = o.cpu().numpy().reshape(-1, 256)[pick]
        assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-10


@pytest.mark.parametrize("p", [8, 12, 16])
def test_batch_oracle_sample_per_order(batch_setup, p):
    """Batched forward and adjoint of one tree of each order against the
    oracle: every node of 8 random leaves (forward), and 8 adjoint columns
    with g random on 6 leaves and zero elsewhere; FP64, and split where the
    order provides it.  Bar 1e-10 relative max-norm (Sec. 4)."""
    ctxs, per_p = batch_setup
    items = per_p[p]
    batch = bc.Batch(ctxs[p], [t for t, _, _ in items])
    k = int(np.argmax([t.nleaf for t, _, _ in items]))   # the largest tree of this order
    t, g, f = items[k]
    lv, ix, iy = t.leaves()
    geom = synth.leaf_geometry(lv, ix, iy)
    pick = synth.sample_leaves(t.nleaf, 8, seed=p)
    ref = oracle.potential_at_nodes(p, geom, f.cpu().numpy().reshape(-1, p, p), leaf_ids=pick)
    rng = np.random.default_rng(p)
    S = np.sort(rng.choice(t.nleaf, 6, replace=False))
    gl = [torch.zeros_like(ff) for _, _, ff in items]
    gv = np.zeros((t.nleaf, p * p))
    gv[S] = rng.standard_normal((6, p * p))
    gl[k] = torch.from_numpy(gv.reshape(-1)).cuda().reshape(gl[k].shape)
    cols = [(int(b), int(j)) for b, j in zip(np.r_[S[:4], rng.choice(t.nleaf, 4)], rng.integers(0, p * p, 8))]
    href = oracle.adjoint_columns(p, geom, gv, cols, target_leaves=S)
    precs = [bc.FP64] + ([bc.SPLIT_BF16] if p in bc.SPLIT_ORDERS else [])
    for prec in precs:
        outs = [torch.empty_like(ff) for _, _, ff in items]
        batch.run([ff for _, _, ff in items], outs, precision=prec)
        got = outs[k].cpu().numpy().reshape(-1, p * p)[pick]
        ef = np.abs(got - ref).max() / np.abs(ref).max()
        adj = [torch.empty_like(ff) for _, _, ff in items]
        batch.run(gl, adj, precision=prec, adjoint=True)
        h = adj[k].cpu().numpy().reshape(-1, p * p)
        ea = np.abs(np.array([h[b, j] for b, j in cols]) - href).max() / np.abs(href).max()
        print(f"batch p={p} precision {prec} ({t.nleaf} leaves): forward {ef:.2e}, adjoint {ea:.2e}")
        assert ef < 1e-10 and ea < 1e-10, (ef, ea)


def test_batch_rejects_mixed_contexts(batch_setup):
    ctxs, per_p = batch_setup
    with pytest.raises(bc.BoxCodeError):
        bc.Batch(ctxs[8], [per_p[8][0][0], per_p[12][0][0]])
