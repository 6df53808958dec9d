"""GPU parity: the CUDA box code against the CPU oracle, element by element.

Every case builds a seeded synthetic density (Gaussian sums, the paper's test
densities of Sec. 4), applies the operator on the GPU through the C ABI and
compares with the oracle's direct quadrature of eq. (vbulk) on the same
leaves, at all nodes of sampled leaves.  Error metric: max |u - u*| / max |u*|
over the evaluated targets.  Bar: 1e-10 (the accuracy the paper reports for
its solver, Sec. 4); the FP64 path is expected near 1e-12.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2501_17967_gb300 as bc  # noqa: E402
from paper_2501_17967_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def ctx16():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return bc.Context(p=16, device=0)


def relerr(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def make(ctx, lv, ix, iy, density, x0=-1.0, y0=-1.0, L=2.0):
    tree = bc.Tree(ctx, lv, ix, iy, x0, y0, L)
    geom = synth.leaf_geometry(lv, ix, iy, x0, y0, L)
    fvals = density(oracle.leaf_nodes(geom, ctx.p)).reshape(len(lv), ctx.p, ctx.p)
    f = torch.from_numpy(fvals).cuda()
    return tree, geom, fvals, f


def touching_sets(lv, ix, iy, targets):
    """Per target leaf: leaves that touch it or are it (independent of the library's lists)."""
    lv, ix, iy = (np.asarray(a, dtype=np.int64) for a in (lv, ix, iy))
    L = lv.max()
    s = L - lv
    x0, x1 = ix << s, (ix + 1) << s
    y0, y1 = iy << s, (iy + 1) << s
    out = []
    for t in targets:
        ok = (x0 <= x1[t]) & (x0[t] <= x1) & (y0 <= y1[t]) & (y0[t] <= y1)
        out.append(np.nonzero(ok)[0])
    return out


def csr_for_nodes(sets, p):
    idx = []
    ptr = [0]
    for s in sets:
        for _ in range(p * p):
            idx.extend(s.tolist())
            ptr.append(len(idx))
    return np.array(ptr, dtype=np.int64), np.array(idx, dtype=np.int64)


def test_uniform_near_field_only(ctx16):
    """Near-field pass alone (self + 8 colleague tables) vs the oracle restricted
    to touching source leaves."""
    p = 16
    g = synth.config_density(1)
    lv, ix, iy = synth.uniform_leaves(3)
    tree, geom, fvals, f = make(ctx16, lv, ix, iy, g)
    ctx16.debug(pass_mask=1)
    try:
        u = bc.apply(tree, f).cpu().numpy().reshape(-1, p * p)
    finally:
        ctx16.debug(pass_mask=3)
    pick = np.array([0, 9, 27, 36, 63])
    src = csr_for_nodes(touching_sets(lv, ix, iy, pick), p)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick, sources=src)
    err = relerr(u[pick], ref)
    assert err < 1e-13, err


def test_uniform_config1_full(ctx16):
    """Workload 1: uniform level-3 tree (64 leaves, N = 16384), 3 broad Gaussians."""
    p = 16
    g = synth.config_density(1)
    lv, ix, iy = synth.uniform_leaves(3)
    tree, geom, fvals, f = make(ctx16, lv, ix, iy, g)
    u = bc.apply(tree, f).cpu().numpy().reshape(-1, p * p)
    pick = np.arange(0, 64, 3)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick)
    err = relerr(u[pick], ref)
    print(f"config1 FP64 rel err {err:.3e}")
    assert err < TOL, err


@pytest.fixture(scope="module")
def adaptive(ctx16):
    g = synth.gaussians(8, 21, wlog10=(-2.3, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=9)
    return (lv, ix, iy, g) + make(ctx16, lv, ix, iy, g)


def test_adaptive_full(ctx16, adaptive):
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    p = 16
    s = tree.stats()
    assert s["n_w"] > 0 and s["n_x"] > 0 and s["nlevels"] >= 7
    u = bc.apply(tree, f).cpu().numpy().reshape(-1, p * p)
    pick = synth.sample_leaves_per_level(np.asarray(lv), 3, seed=3)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick)
    err = relerr(u[pick], ref)
    print(f"adaptive ({len(lv)} leaves, {s['nlevels']} levels) FP64 rel err {err:.3e}")
    assert err < TOL, err


@pytest.mark.parametrize("p", [6, 9])
def test_fp64_node_counts_not_multiple_of_eight(p):
    """Orders whose node count does not split evenly over the four warps of the
    leaf-to-expansion and X-list products (p = 6: 36 nodes, 9 per warp; p = 9:
    81 nodes): FP64 apply on an adaptive tree with W and X lists against the
    oracle, and the adjoint identity <A f, g> = <f, A^T g>."""
    ctx = bc.Context(p=p, device=0)
    g = synth.gaussians(8, 21, wlog10=(-2.3, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=7)
    tree, geom, fvals, f = make(ctx, lv, ix, iy, g)
    s = tree.stats()
    assert s["n_w"] > 0 and s["n_x"] > 0
    u = bc.apply(tree, f)
    un = u.cpu().numpy().reshape(-1, p * p)
    pick = synth.sample_leaves_per_level(np.asarray(lv), 2, seed=4)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick)
    err = relerr(un[pick], ref)
    print(f"p = {p}: FP64 rel err {err:.3e}")
    assert err < TOL, err
    gen = torch.Generator(device="cuda").manual_seed(7)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    lhs = torch.dot(u.ravel(), gg.ravel()).item()
    rhs = torch.dot(f.ravel(), bc.apply_adjoint(tree, gg).ravel()).item()
    scale = (u.abs() * gg.abs()).sum().item()
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs, scale)


def test_adaptive_near_and_far_split(ctx16, adaptive):
    """near-only + far-only applies add up to the full apply (linearity of the passes)."""
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    full = bc.apply(tree, f)
    ctx16.debug(pass_mask=1)
    un = bc.apply(tree, f)
    ctx16.debug(pass_mask=2)
    uf = bc.apply(tree, f)
    ctx16.debug(pass_mask=3)
    d = (un + uf - full).abs().max().item()
    assert d <= 1e-13 * full.abs().max().item()
    # near-only against the oracle restricted to touching leaves
    p = 16
    pick = synth.sample_leaves(len(lv), 6, seed=5)
    src = csr_for_nodes(touching_sets(lv, ix, iy, pick), p)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick, sources=src)
    err = relerr(un.cpu().numpy().reshape(-1, p * p)[pick], ref)
    assert err < 1e-13, err


def test_adjoint_dot_product(ctx16, adaptive):
    """<A f, g> = <f, A^T g> for random f, g (exact transpose of the discrete operator)."""
    lv, ix, iy, gd, tree, geom, fvals, f = adaptive
    gen = torch.Generator(device="cuda").manual_seed(0)
    fr = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    gr = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    lhs = torch.dot(bc.apply(tree, fr).ravel(), gr.ravel()).item()
    rhs = torch.dot(fr.ravel(), bc.apply_adjoint(tree, gr).ravel()).item()
    scale = (bc.apply(tree, fr).abs() * gr.abs()).sum().item()
    assert abs(lhs - rhs) <= 1e-14 * scale, (lhs, rhs, scale)


def test_m2l_triangular_and_orders(ctx16, adaptive):
    """The triangular M2L truncation (k + l <= P) keeps the exact-transpose
    property and stays close to the full series; a context with a short
    expansion (nterms 12, the 16-wide M2L kernel) agrees with nterms 30 to
    its truncation level."""
    lv, ix, iy, gd, tree, geom, fvals, f = adaptive
    gen = torch.Generator(device="cuda").manual_seed(3)
    fr = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    gr = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    full = bc.apply(tree, f)
    ctx16.set_option("m2l_triangular", 1)
    try:
        tri = bc.apply(tree, f)
        lhs = torch.dot(bc.apply(tree, fr).ravel(), gr.ravel()).item()
        rhs = torch.dot(fr.ravel(), bc.apply_adjoint(tree, gr).ravel()).item()
        scale = (bc.apply(tree, fr).abs() * gr.abs()).sum().item()
    finally:
        ctx16.set_option("m2l_triangular", 0)
    assert abs(lhs - rhs) <= 1e-14 * scale, (lhs, rhs, scale)
    d = ((tri - full).abs().max() / full.abs().max()).item()
    assert 0.0 < d < 1e-6, d
    ctx12 = bc.Context(p=16, nterms=12, device=0)
    t12 = bc.Tree(ctx12, lv, ix, iy)
    d12 = ((bc.apply(t12, f) - full).abs().max() / full.abs().max()).item()
    assert 0.0 < d12 < 1e-5, d12
    lhs = torch.dot(bc.apply(t12, fr).ravel(), gr.ravel()).item()
    rhs = torch.dot(fr.ravel(), bc.apply_adjoint(t12, gr).ravel()).item()
    assert abs(lhs - rhs) <= 1e-14 * scale, (lhs, rhs)


def test_adjoint_against_oracle_columns(ctx16):
    """Sampled entries of A^T g against the oracle's transposed operator."""
    p = 16
    g = synth.gaussians(3, 4, wlog10=(-1.4, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, max_level=4)
    tree, geom, fvals, f = make(ctx16, lv, ix, iy, g)
    gen = np.random.default_rng(2)
    gv = gen.standard_normal((len(lv), p * p))
    h = bc.apply_adjoint(tree, torch.from_numpy(gv).cuda()).cpu().numpy().reshape(-1, p * p)
    cols = [(int(b), int(j)) for b, j in zip(gen.integers(0, len(lv), 6), gen.integers(0, p * p, 6))]
    ref = oracle.adjoint_columns(p, geom, gv, cols)
    got = np.array([h[b, j] for b, j in cols])
    err = float(np.abs(got - ref).max() / np.abs(h).max())
    assert err < TOL, err


@pytest.mark.parametrize("p", [8, 12])
def test_other_orders(p):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=p, device=0)
    g = synth.gaussians(4, 30 + p, wlog10=(-1.8, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=2.0, max_level=7)
    tree, geom, fvals, f = make(ctx, lv, ix, iy, g)
    u = bc.apply(tree, f).cpu().numpy().reshape(-1, p * p)
    pick = synth.sample_leaves(len(lv), 12, seed=p)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick)
    assert relerr(u[pick], ref) < TOL


def test_host_pointer_path_matches_device(ctx16, adaptive):
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    ud = bc.apply(tree, f).cpu()
    fh = f.cpu()
    uh = bc.apply(tree, fh)
    assert torch.equal(ud, uh)
    pinned = fh.pin_memory()
    up = bc.apply(tree, pinned, out=torch.empty_like(pinned).pin_memory())
    assert torch.equal(ud, up)


def test_split_pinned_host_arrays_in_place(ctx16, adaptive):
    """Split precision with host arrays: pinned ones are read and written in
    place by the kernels, pageable ones are staged, and a pinned input with a
    pageable output is staged; each gives the device result bit for bit, in
    both directions."""
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    gen = torch.Generator(device="cuda").manual_seed(19)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    S = bc.SPLIT_BF16
    ud = bc.apply(tree, f, precision=S).cpu()
    hd = bc.apply_adjoint(tree, gg, precision=S).cpu()
    fp, gp = f.cpu().pin_memory(), gg.cpu().pin_memory()
    up = bc.apply(tree, fp, out=torch.empty_like(fp).pin_memory(), precision=S)
    hp = bc.apply_adjoint(tree, gp, out=torch.empty_like(gp).pin_memory(), precision=S)
    assert torch.equal(up, ud) and torch.equal(hp, hd)
    assert torch.equal(bc.apply(tree, f.cpu(), precision=S), ud)
    assert torch.equal(bc.apply_adjoint(tree, gg.cpu(), precision=S), hd)
    assert torch.equal(bc.apply(tree, fp, out=torch.zeros(fp.shape, dtype=fp.dtype), precision=S), ud)


def test_eval_points(ctx16, adaptive):
    """Off-grid targets: interpolation of the leaf-node potential vs the oracle's
    potential at the points (bounded by the interpolation error), and vs an
    independent host barycentric evaluation of the same node values."""
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    p = 16
    u = bc.apply(tree, f)
    pts = synth.random_targets(400, seed=101)
    pts = np.vstack([pts, [[-1.0, -1.0], [1.0, 1.0], [0.0, 0.0], [1.0, -1.0]]])
    val = bc.eval_points(tree, u, torch.from_numpy(pts).cuda()).cpu().numpy()
    ref = oracle.potential(p, geom, fvals, pts)
    assert relerr(val, ref) < TOL
    # host barycentric on the containing leaf
    un = u.cpu().numpy().reshape(-1, p * p)
    xn = oracle.cheb_nodes(p)
    lam = np.where(np.arange(p) % 2, -1.0, 1.0) * np.sin((2 * np.arange(p) + 1) * math.pi / (2 * p))
    for k in range(0, len(pts), 37):
        x, y = pts[k]
        inside = [b for b in range(len(lv)) if
                  geom[b, 0] - geom[b, 2] <= x < geom[b, 0] + geom[b, 2] + (1e-300 if x < 1 else 1)
                  and geom[b, 1] - geom[b, 2] <= y < geom[b, 1] + geom[b, 2] + (1e-300 if y < 1 else 1)]
        b = inside[0]
        xi, eta = (x - geom[b, 0]) / geom[b, 2], (y - geom[b, 1]) / geom[b, 2]
        lx = lam / (xi - xn); lx /= lx.sum()
        ly = lam / (eta - xn); ly /= ly.sum()
        assert abs(ly @ un[b].reshape(p, p) @ lx - val[k]) < 1e-13 * np.abs(un).max()


def test_errors_reported(ctx16, adaptive):
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    with pytest.raises(bc.BoxCodeError):
        bc.apply(tree, f, out=f)                                   # aliasing
    with pytest.raises(ValueError):
        bc.apply(tree, f[:3])                                      # wrong size
    other = bc.Context(p=16, device=0)
    t2 = bc.Tree(other, lv, ix, iy)
    with pytest.raises(bc.BoxCodeError):
        bc._check(bc._load().bc_apply(ctx16.handle, t2.handle, f.data_ptr(), torch.empty_like(f).data_ptr(),
                                      0, None))
    with pytest.raises(bc.BoxCodeError):
        bc.apply(tree, f, precision=7)


def test_autograd_matches_finite_differences(ctx16):
    """Gradient of L = 0.5 ||u(f(theta)) - u_t||^2 w.r.t. Gaussian parameters
    theta through BoxCodeApply (adjoint kernels) vs central differences."""
    p = 16
    g = synth.gaussians(3, 3, wlog10=(-1.3, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, max_level=5)
    tree = bc.Tree(ctx16, lv, ix, iy)
    geom = synth.leaf_geometry(lv, ix, iy)
    nodes = torch.from_numpy(oracle.leaf_nodes(geom, p)).cuda()
    theta0 = torch.tensor(np.c_[g.cx, g.cy, np.log(g.w), g.a], device="cuda")

    def density(th):
        x, y = nodes[..., 0:1], nodes[..., 1:2]
        cx, cy, lw, a = th[:, 0], th[:, 1], th[:, 2], th[:, 3]
        w = torch.exp(lw)
        return (a * torch.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w))).sum(-1)

    with torch.no_grad():
        ut = bc.apply(tree, density(theta0 + 0.01 * torch.randn_like(theta0)).contiguous())

    def loss(th):
        u = bc.BoxCodeApply.apply(density(th).contiguous(), tree)
        return 0.5 * ((u - ut) ** 2).sum()

    th = theta0.clone().requires_grad_(True)
    loss(th).backward()
    grad = th.grad.clone()
    h = 1e-6
    fd = torch.zeros_like(theta0)
    for i in range(theta0.shape[0]):
        for j in range(theta0.shape[1]):
            e = torch.zeros_like(theta0)
            e[i, j] = h
            with torch.no_grad():
                fd[i, j] = (loss(theta0 + e) - loss(theta0 - e)) / (2 * h)
    rel = ((grad - fd).abs().max() / grad.abs().max()).item()
    assert rel < 1e-6, rel


# ---------------------------------------------------------------------------
# Split precision, p = 16: the near-field tables, leaf-to-expansion, X list,
# expansion-to-leaf and W list on BF16 tensor cores (tcgen05) as exact
# products of 40-bit fixed-point digits; M2L, shifts, log terms and sums FP64.
# Each product's rounding is about 2^-40 of its largest term times a small
# multiple (balanced power-of-two column scales), ~1e-11 of max|u| after the
# expansion-to-leaf step; the bound checked is the 1e-10 target (TOL).  The
# near field alone stays at the 1e-12 level (SPLIT_NEAR_TOL).
# ---------------------------------------------------------------------------
SPLIT_NEAR_TOL = 1e-11
SPLIT_MODES = pytest.mark.parametrize("mode", [1, 2], ids=["split", "split_all"])


@SPLIT_MODES
def test_split_config1_vs_oracle(ctx16, mode):
    p = 16
    g = synth.config_density(1)
    lv, ix, iy = synth.uniform_leaves(3)
    tree, geom, fvals, f = make(ctx16, lv, ix, iy, g)
    us = bc.apply(tree, f, precision=mode)
    bc._check(bc._load().bc_sync(ctx16.handle, None))
    u = us.cpu().numpy().reshape(-1, p * p)
    pick = np.arange(0, 64, 3)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick)
    err = relerr(u[pick], ref)
    print(f"config1 split mode {mode} rel err {err:.3e}")
    assert err < TOL, err


@SPLIT_MODES
def test_split_adaptive_vs_fp64_and_oracle(ctx16, adaptive, mode):
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    p = 16
    u64 = bc.apply(tree, f)
    us = bc.apply(tree, f, precision=mode)
    bc._check(bc._load().bc_sync(ctx16.handle, None))
    d = ((us - u64).abs().max() / u64.abs().max()).item()
    assert d < TOL, d
    pick = synth.sample_leaves_per_level(np.asarray(lv), 2, seed=9)
    ref = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=pick)
    err = relerr(us.cpu().numpy().reshape(-1, p * p)[pick], ref)
    print(f"adaptive split mode {mode} rel err {err:.3e} (vs fp64 {d:.3e})")
    assert err < TOL, err


def test_split_near_only_and_adjoint(ctx16, adaptive):
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    ctx16.debug(pass_mask=1)
    try:
        n64 = bc.apply(tree, f)
        ns = bc.apply(tree, f, precision=bc.SPLIT_BF16)
    finally:
        ctx16.debug(pass_mask=3)
    assert ((ns - n64).abs().max() / n64.abs().max()).item() < SPLIT_NEAR_TOL
    gen = torch.Generator(device="cuda").manual_seed(5)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    h64 = bc.apply_adjoint(tree, gg)
    hs = bc.apply_adjoint(tree, gg, precision=bc.SPLIT_BF16)
    bc._check(bc._load().bc_sync(ctx16.handle, None))
    assert ((hs - h64).abs().max() / h64.abs().max()).item() < TOL
    # host-pointer path gives the same split result as the device path
    uh = bc.apply(tree, f.cpu(), precision=bc.SPLIT_BF16)
    assert torch.equal(uh, bc.apply(tree, f, precision=bc.SPLIT_BF16).cpu())


def test_split_unsupported_order_reports():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=10, device=0)   # split tables exist for p = 8, 12 and 16 only
    lv, ix, iy = synth.uniform_leaves(2)
    tree = bc.Tree(ctx, lv, ix, iy)
    f = torch.zeros(16 * 100, dtype=torch.float64, device="cuda")
    with pytest.raises(bc.BoxCodeError) as e:
        bc.apply(tree, f, precision=bc.SPLIT_BF16)
    assert e.value.status == -6


def test_split_wait_timeout_is_reported_and_context_survives(ctx16, adaptive):
    """A bounded device-side wait that runs out (the table copy is withheld)
    gives BC_ERR_TIMEOUT at bc_sync; the context keeps working afterwards."""
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    ctx16.set_option("wait_limit", 2000)
    ctx16.set_option("debug_withhold_copy", 1)
    try:
        bc.apply(tree, f, precision=bc.SPLIT_BF16)
        st = bc._load().bc_sync(ctx16.handle, None)
    finally:
        ctx16.set_option("debug_withhold_copy", 0)
        ctx16.set_option("wait_limit", 2 ** 26)
    assert st == -5
    assert "wait" in bc._load().bc_last_error().decode()
    bc._check(bc._load().bc_sync(ctx16.handle, None))     # flag cleared
    u64 = bc.apply(tree, f)
    us = bc.apply(tree, f, precision=bc.SPLIT_BF16)
    bc._check(bc._load().bc_sync(ctx16.handle, None))
    assert ((us - u64).abs().max() / u64.abs().max()).item() < TOL


def test_split_parts_each_within_tolerance(ctx16, adaptive):
    """Each tensor-core product alone (the others FP64) stays within the split
    tolerance in both directions; with none of them the split apply equals
    the FP64 apply bit for bit."""
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    gen = torch.Generator(device="cuda").manual_seed(11)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    u64, h64 = bc.apply(tree, f), bc.apply_adjoint(tree, gg)
    try:
        for parts in (0, 1, 2, 4, 8, 16, 32, 64):
            ctx16.set_option("debug_split_parts", parts)
            us = bc.apply(tree, f, precision=bc.SPLIT_BF16)
            hs = bc.apply_adjoint(tree, gg, precision=bc.SPLIT_BF16)
            bc._check(bc._load().bc_sync(ctx16.handle, None))
            if parts == 0:
                assert torch.equal(us, u64) and torch.equal(hs, h64)
                continue
            du = ((us - u64).abs().max() / u64.abs().max()).item()
            dh = ((hs - h64).abs().max() / h64.abs().max()).item()
            print(f"split part {parts}: fwd {du:.2e} adj {dh:.2e}")
            assert 0.0 < du < TOL and 0.0 < dh < TOL, (parts, du, dh)
    finally:
        ctx16.set_option("debug_split_parts", -1)


def test_split_overlap_gives_identical_results(ctx16, adaptive):
    """The X-list and near-field tensor launches on the internal stream (the
    default, split_overlap = 1), on any number of CTAs, compute exactly what
    the in-line launch computes, in both directions."""
    lv, ix, iy, g, tree, geom, fvals, f = adaptive
    gen = torch.Generator(device="cuda").manual_seed(13)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    u1 = bc.apply(tree, f, precision=bc.SPLIT_BF16)
    h1 = bc.apply_adjoint(tree, gg, precision=bc.SPLIT_BF16)
    try:
        ctx16.set_option("split_overlap", 0)
        u0 = bc.apply(tree, f, precision=bc.SPLIT_BF16)
        h0 = bc.apply_adjoint(tree, gg, precision=bc.SPLIT_BF16)
        ctx16.set_option("split_overlap", 1)
        outs = []
        for ctas in (7, 40, 152):
            ctx16.set_option("split_overlap_ctas", ctas)
            outs.append((bc.apply(tree, f, precision=bc.SPLIT_BF16),
                         bc.apply_adjoint(tree, gg, precision=bc.SPLIT_BF16)))
        bc._check(bc._load().bc_sync(ctx16.handle, None))
    finally:
        ctx16.set_option("split_overlap", 1)
        ctx16.set_option("split_overlap_ctas", 0)
    assert torch.equal(u0, u1) and torch.equal(h0, h1)
    for uc, hc in outs:
        assert torch.equal(uc, u1) and torch.equal(hc, h1)


@pytest.mark.parametrize("nterms", [8, 12, 31])
def test_split_double_float_shifts_other_orders(nterms):
    """At other expansion orders, in both directions: the double-float level
    shifts alone (part 64, every product in FP64) agree with the FP64 shifts
    to double-float rounding; the upward one runs on its triangular term
    schedule (at 8, 12 and 31 terms: 2, 3 and 17 terms per lane, up to 5
    partial sums per coefficient).  The full split apply stays within the
    split tolerance of the FP64 apply.  (Two split applies that differ only
    in the shifts differ by up to one step of the 40-bit digit grid, about
    1e-12: the expansions feed the digits of later products.)"""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=16, nterms=nterms, device=0)
    g = synth.gaussians(8, 21, wlog10=(-2.3, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=9)
    tree, geom, fvals, f = make(ctx, lv, ix, iy, g)
    gen = torch.Generator(device="cuda").manual_seed(17)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    u64, h64 = bc.apply(tree, f), bc.apply_adjoint(tree, gg)
    try:
        out = {}
        for parts in (0, 64, 127):
            ctx.set_option("debug_split_parts", parts)
            out[parts] = (bc.apply(tree, f, precision=bc.SPLIT_BF16),
                          bc.apply_adjoint(tree, gg, precision=bc.SPLIT_BF16))
        bc._check(bc._load().bc_sync(ctx.handle, None))
    finally:
        ctx.set_option("debug_split_parts", -1)
    for k, ref in enumerate((u64, h64)):
        tag = "adj" if k else "fwd"
        d_df = ((out[64][k] - out[0][k]).abs().max() / out[0][k].abs().max()).item()
        d_all = ((out[127][k] - ref).abs().max() / ref.abs().max()).item()
        print(f"nterms {nterms} {tag}: double-float vs FP64 shifts {d_df:.2e}, split vs FP64 {d_all:.2e}")
        assert 0.0 < d_df < 1e-13, (nterms, tag, d_df)
        assert d_all < TOL, (nterms, tag, d_all)


@pytest.mark.parametrize("nterms", [8, 13, 24, 31])
def test_m2l_tensor_core_kernel_matches_fma_kernel(nterms):
    """The FP64 M2L by FMAs (the default) and on the FP64 tensor cores (MMA
    tiles of the binomial matrix) give the same local expansions up to rounding,
    forward and adjoint, at expansion orders that fill the 8 x 4 MMA tiles
    partially and exactly; both match the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = bc.Context(p=16, nterms=nterms, device=0)
    g = synth.gaussians(8, 21, wlog10=(-2.3, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=8)
    tree, geom, fvals, f = make(ctx, lv, ix, iy, g)
    gen = torch.Generator(device="cuda").manual_seed(23)
    gg = torch.randn(f.shape, generator=gen, device="cuda", dtype=torch.float64)
    out = {}
    try:
        for kind in (0, 1):
            ctx.set_option("m2l_kernel", kind)
            out[kind] = (bc.apply(tree, f), bc.apply_adjoint(tree, gg))
    finally:
        ctx.set_option("m2l_kernel", 0)
    for k in range(2):
        d = ((out[0][k] - out[1][k]).abs().max() / out[1][k].abs().max()).item()
        assert d < 1e-13, (nterms, k, d)
    if nterms == 24:
        pick = synth.sample_leaves_per_level(np.asarray(lv), 1, seed=5)
        ref = oracle.potential_at_nodes(16, geom, fvals, leaf_ids=pick)
        err = relerr(out[1][0].cpu().numpy().reshape(-1, 256)[pick], ref)
        assert err < TOL, err
