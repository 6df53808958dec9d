"""The allocation-free FP64 apply (bc_apply_noalloc) against the regular apply.

bc_apply_noalloc serves callers that must not allocate device memory during
the call (it takes its workspaces from a fixed array in the library); it must
give the same potential as bc_apply.  The check calls it twice in a row, for
the forward operator and the transpose, through the C ABI directly.  This file
is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _noalloc(ctx, tree, x, out, adjoint):
    return bc._load().bc_apply_noalloc(ctx.handle, tree.handle, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), int(adjoint), None)


def test_noalloc_matches_regular_apply():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=16, device=0)
    g = synth.gaussians(6, 77, wlog10=(-2.0, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=8)
    tree = bc.Tree(ctx, lv, ix, iy)
    geom = synth.leaf_geometry(lv, ix, iy)
    f = torch.from_numpy(g(oracle.leaf_nodes(geom, 16))).cuda()
    gen = torch.Generator(device="cuda").manual_seed(3)
    gv = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    for adjoint, x in ((0, f), (1, gv)):
        ref = bc.apply_adjoint(tree, x) if adjoint else bc.apply(tree, x)
        for _ in range(2):   # two calls in a row share the fixed workspace
            out = torch.full_like(x, float("nan"))
            bc._check(_noalloc(ctx, tree, x, out, adjoint))
            torch.cuda.synchronize()
            err = ((out - ref).abs().max() / ref.abs().max()).item()
            assert err <= 1e-13, (adjoint, err)


def test_noalloc_rejects_trees_beyond_its_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=8, nterms=32, device=0)
    lv, ix, iy = synth.uniform_leaves(7)   # 21845 boxes x 32 terms x 32 B > 16 MiB
    tree = bc.Tree(ctx, lv, ix, iy)
    x = torch.zeros(tree.nleaf * 64, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    st = _noalloc(ctx, tree, x, out, 0)
    assert st == -1
    assert "limit" in bc._load().bc_last_error().decode()
