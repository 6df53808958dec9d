"""The glue layer potential S[sigma] - D[tau] (Sec. 3.4) by the FMM at every
leaf node, against the oracle's direct sum and against closed forms.

Cases: the star-shaped domain's truncated tree with Gauss-Legendre sources on
its fictitious curve and smooth jump densities (W and X lists present,
sources in leaves of several levels); a circle of sources in an adaptive tree
(single layer -R log R inside, -R log|x - c| outside; double layer 1 inside
and 0 outside, at nodes away from the circle); host arrays against device
arrays; no sources; a source on a node and on leaf edges.

Bar: the near field is summed exactly and the far field carries the
truncation error of the expansions.  Point sources anywhere in a box,
corners included, converge like (sqrt 2 / (4 - sqrt 2))^P ~ 0.55^P across
the V list (smooth volume densities converge much faster): nterms 24 gave
6e-11..1.5e-10 here, so the layer runs with nterms 30 (the library
default), a further 0.55^6 ~ 0.03.  The bar is 1e-10 of max |u| over the
sample (Sec. 4's tolerance); the closed forms hold to the trapezoid rule's
error (below 1e-14 at the selected nodes) plus the truncation, so the bar
there is 1e-11 absolute."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

P = 16
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return bc.Context(p=P, nterms=30, device=0)


@pytest.fixture(scope="module")
def star(ctx):
    gamma, gamma_b = synth.star_domain()
    tree = bc.Tree.refine_truncated(ctx, synth.config_density(2), gamma, gamma_b, eps=1e-11, max_level=18)
    xy, w, nrm, t = synth.fictitious_curve_sources(256, 16)
    sig, tau = synth.glue_densities(t)
    q, m = w * sig, (w * tau)[:, None] * nrm
    return tree, xy, q, m


def _nodes(tree):
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    geom = synth.leaf_geometry(lv, ix, iy)
    return lv, geom, oracle.leaf_nodes(geom, P)


def _leaves_holding(geom, pts):
    inside = ((np.abs(pts[:, None, 0] - geom[None, :, 0]) <= geom[None, :, 2])
              & (np.abs(pts[:, None, 1] - geom[None, :, 1]) <= geom[None, :, 2]))
    return np.unique(np.nonzero(inside)[1])


@pytest.mark.parametrize("prec", [bc.FP64, bc.SPLIT_BF16])
def test_layer_against_oracle(ctx, star, prec):
    """FP64, and split precision (the L2P at every leaf on the tensor cores:
    its digit products are exact and the rounding of the 40-bit operands and
    locals adds about 1e-12 of max |u|, well inside the bar)."""
    tree, xy, q, m = star
    layer = bc.Layer(tree, xy)
    info = layer.info()
    assert info["sources"] == len(q) and info["n_w"] > 0 and info["n_v"] > 0
    u = layer.apply(torch.from_numpy(q).cuda(), torch.from_numpy(m).cuda(),
                    precision=prec).cpu().numpy().reshape(-1, P * P)
    lv, geom, nodes = _nodes(tree)
    hold = _leaves_holding(geom, xy)
    rng = np.random.default_rng(2)
    pick = np.unique(np.concatenate([rng.choice(hold, 12, replace=False),
                                     synth.sample_leaves_per_level(lv, 2, seed=5)]))
    ref = oracle.layer(xy, q, m, nodes[pick].reshape(-1, 2)).reshape(len(pick), P * P)
    err = np.abs(u[pick] - ref).max() / np.abs(ref).max()
    print(f"layer ({prec}): {len(q)} sources, {tree.nleaf} leaves, {info}; sample {len(pick)} leaves: {err:.2e}")
    assert err < TOL, err
    # host arrays give the device result bit for bit
    uh = layer.apply(torch.from_numpy(q), torch.from_numpy(m), precision=prec).numpy().reshape(-1, P * P)
    assert np.array_equal(uh, u)
    if prec == bc.SPLIT_BF16:
        # the split L2P against the FP64 one over every node of the tree
        u64 = layer.apply(torch.from_numpy(q).cuda(), torch.from_numpy(m).cuda()).cpu().numpy().reshape(-1, P * P)
        d = np.abs(u - u64).max() / np.abs(u64).max()
        print(f"split vs FP64 L2P, all {tree.nleaf} leaves: {d:.2e}")
        assert d < 1e-11, d
        with pytest.raises(bc.BoxCodeError):
            layer.apply(torch.from_numpy(q).cuda(), torch.from_numpy(m).cuda(), precision=bc.SPLIT_BF16_ALL)


def test_layer_scattered_sources_against_oracle(ctx):
    """Charges and dipoles scattered over the whole root box of an adaptive
    tree, so that every list kind carries sources (X entries included)."""
    tree = bc.Tree.refine(ctx, synth.config_density(2), eps=1e-11, max_level=18)
    rng = np.random.default_rng(12)
    src = rng.uniform(-1, 1, (3000, 2))
    q, m = rng.standard_normal(3000), rng.standard_normal((3000, 2))
    layer = bc.Layer(tree, src)
    info = layer.info()
    assert info["n_x"] > 0 and info["n_w"] > 0
    u = layer.apply(torch.from_numpy(q).cuda(), torch.from_numpy(m).cuda()).cpu().numpy().reshape(-1, P * P)
    lv, geom, nodes = _nodes(tree)
    pick = synth.sample_leaves_per_level(lv, 2, seed=9)
    ref = oracle.layer(src, q, m, nodes[pick].reshape(-1, 2)).reshape(len(pick), P * P)
    err = np.abs(u[pick] - ref).max() / np.abs(ref).max()
    print(f"scattered: {info}; {len(pick)} leaves: {err:.2e}")
    assert err < TOL, err


def test_layer_circle_closed_forms(ctx):
    # an adaptive tree refined toward a circle, sources on the circle
    R, c = 0.55, np.array([0.07, -0.11])
    g = synth.gaussians(3, 7, wlog10=(-1.6, -1.2))
    tree = bc.Tree.refine(ctx, g, eps=1e-9, max_level=10)
    n = 1024
    th = 2 * np.pi * np.arange(n) / n
    nrm = np.stack([np.cos(th), np.sin(th)], 1)
    src, w = c + R * nrm, np.full(n, 2 * np.pi * R / n)
    layer = bc.Layer(tree, src)
    lv, geom, nodes = _nodes(tree)
    x = nodes.reshape(-1, 2)
    d = np.linalg.norm(x - c, axis=1)
    inner, outer = d < 0.8 * R, d > 1.25 * R
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    us = layer.apply(torch.from_numpy(w).cuda(), torch.zeros((n, 2), dtype=torch.float64, device="cuda"))
    ud = layer.apply(zero, torch.from_numpy(w[:, None] * nrm).cuda())
    us, ud = us.cpu().numpy(), ud.cpu().numpy()
    es = max(np.abs(us[inner] + R * np.log(R)).max(), np.abs(us[outer] + R * np.log(d[outer])).max())
    ed = max(np.abs(ud[inner] - 1.0).max(), np.abs(ud[outer]).max())
    print(f"circle: single layer {es:.2e}, double layer {ed:.2e}")
    assert es < 1e-11 and ed < 1e-11, (es, ed)


def test_layer_edge_cases(ctx):
    tree = bc.Tree(ctx, *synth.uniform_leaves(3))
    lv, geom, nodes = _nodes(tree)
    # no sources
    empty = bc.Layer(tree, np.zeros((0, 2)))
    z = empty.apply(torch.zeros(0, dtype=torch.float64, device="cuda"),
                    torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(z).item() == 0
    # a source on a node, sources on leaf edges and corners, one on the root's edge
    src = np.array([nodes[5, 17], [0.0, 0.0], [0.25, 0.1], [-0.5, -0.75], [1.0, 0.3], [0.3, -1.0]])
    rng = np.random.default_rng(8)
    q, m = rng.standard_normal(len(src)), rng.standard_normal((len(src), 2))
    u = bc.Layer(tree, src).apply(torch.from_numpy(q).cuda(), torch.from_numpy(m).cuda()).cpu().numpy()
    ref = oracle.layer(src, q, m, nodes.reshape(-1, 2))
    err = np.abs(u - ref).max() / np.abs(ref).max()
    print(f"edge cases: {err:.2e}")
    assert err < TOL and np.all(np.isfinite(u))
    with pytest.raises(bc.BoxCodeError):
        bc.Layer(tree, np.array([[1.5, 0.0]]))


def test_near_sum_log_against_cuda():
    """The near sums' table-driven logarithm (after Tang, 1990) and reciprocal
    against the CUDA math library's log and IEEE division, on random squared
    distances over 19 decades, on x = 1 +- small, and on both sides of every
    table interval boundary over 41 binades.  Bars: |error| <= 2^-51
    max(1, |log x|) for the logarithm (absolute near x = 1, where the near
    sums need only absolute accuracy) and 2^-51 relative for 1/x."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(3)
    parts = [10.0 ** rng.uniform(-16, 3, 1 << 20)]
    k = np.arange(1, 16)
    parts += [1.0 + 10.0 ** -k, 1.0 - 10.0 ** -k, 1.0 + np.arange(1, 64) * 2.0 ** -52, 1.0 - np.arange(1, 64) * 2.0 ** -53]
    e, j = np.meshgrid(np.arange(-20, 21), np.arange(128), indexing="ij")
    b = np.ldexp(1.0 + j / 128.0, e).ravel()
    parts += [b, np.nextafter(b, 0.0), np.nextafter(b, np.inf)]
    x = torch.from_numpy(np.concatenate(parts)).cuda()
    lg, inv = torch.empty_like(x), torch.empty_like(x)
    bc._check(bc._load().bc_debug_log_inv(0, ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(lg.data_ptr()),
                                         ctypes.c_void_p(inv.data_ptr()), None))
    torch.cuda.synchronize()
    ref_l, ref_i = torch.log(x), 1.0 / x
    el = ((lg - ref_l).abs() / ref_l.abs().clamp(min=1.0)).max().item()
    ei = ((inv - ref_i).abs() / ref_i.abs()).max().item()
    print(f"table log: max error {el / 2.0 ** -53:.2f} units of 2^-53 (scaled); reciprocal {ei / 2.0 ** -53:.2f}")
    assert el <= 2.0 ** -51 and ei <= 2.0 ** -51, (el, ei)
