"""Host-side tests of the C ABI library (no GPU needed).

* the shared library loads and exports every function declared in
  include/boxcode.h;
* tree validation rejects overlapping, gapped and unbalanced leaf sets;
* the interaction lists cover every (target leaf, source leaf) pair exactly
  once (brute force over small adaptive trees);
* the adaptive refinement (paper Alg. 2, resolution criterion) resolves the
  density and returns a 2:1-balanced tree;
* tables: near-table row sums equal the closed-form potential of a constant
  density (every one of the 33 tables), the self table reproduces the centre
  value 2 ln 2 + pi - 6, and tables related by a reflection agree after the
  matching node permutation.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2501_17967_gb300 as bc
from paper_2501_17967_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "boxcode.h")


def _F(a, b):
    if a == 0.0 or b == 0.0:
        return 0.0
    s = math.copysign(1.0, a) * math.copysign(1.0, b)
    a, b = abs(a), abs(b)
    return s * 0.5 * (a * b * (math.log(a * a + b * b) - 3.0) + a * a * math.atan(b / a) + b * b * math.atan(a / b))


def square_potential(x, y):
    """(1/2pi) int_{[-1,1]^2} log|x-y| dy (closed form)."""
    return (_F(1 - x, 1 - y) - _F(-1 - x, 1 - y) - _F(1 - x, -1 - y) + _F(-1 - x, -1 - y)) / (2 * math.pi)


@pytest.fixture(scope="module")
def lib():
    return bc._load()


def test_library_exports_every_declared_symbol(lib):
    text = open(HEADER).read()
    names = set(re.findall(r"^\s*(?:bc_status|void|int64_t|const char \*)\s*\*?\s*(bc_\w+)\s*\(", text, re.M))
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    declared_in_binding = {s[0] for s in bc.SIGNATURES}
    assert names == declared_in_binding


@pytest.fixture(scope="module")
def hctx():
    return bc.Context(p=8, device=-1, cache_dir=None)


def test_set_option_validation(hctx):
    """Options are checked on the host: unknown names and out-of-range values
    give BC_ERR_ARG; valid values are accepted."""
    for name, bad in (("debug_split_parts", 128), ("debug_split_parts", -2), ("debug_split_parts", 2.5),
                      ("wait_limit", 0), ("split_overlap_ctas", -1), ("split_overlap_ctas", 2.5),
                      ("split_overlap", 4), ("split_overlap", 0.5), ("no_such_option", 1)):
        with pytest.raises(bc.BoxCodeError) as e:
            hctx.set_option(name, bad)
        assert e.value.status == -1, (name, bad)
    for name, good in (("debug_split_parts", 0), ("debug_split_parts", 127), ("debug_split_parts", -1),
                       ("wait_limit", 2 ** 26),
                       ("m2l_triangular", 0), ("split_overlap_ctas", 76), ("split_overlap_ctas", 0),
                       ("split_overlap", 2), ("split_overlap", 1)):
        hctx.set_option(name, good)


def test_context_argument_checks():
    """bc_create rejects orders and expansion lengths outside the provided range."""
    for kw in ({"p": 3}, {"p": 17}, {"nterms": 3}, {"nterms": 33}):
        with pytest.raises(bc.BoxCodeError) as e:
            bc.Context(device=-1, cache_dir=None, **kw)
        assert e.value.status == -1, kw


def test_tree_validation_errors(hctx):
    lv, ix, iy = synth.uniform_leaves(2)
    with pytest.raises(bc.BoxCodeError) as e:   # gap
        bc.Tree(hctx, lv[1:], ix[1:], iy[1:])
    assert e.value.status == -2
    with pytest.raises(bc.BoxCodeError):         # overlap: a leaf and its parent
        bc.Tree(hctx, np.r_[lv, 1], np.r_[ix, 0], np.r_[iy, 0])
    with pytest.raises(bc.BoxCodeError):         # duplicate
        bc.Tree(hctx, np.r_[lv, 2], np.r_[ix, 0], np.r_[iy, 0])
    with pytest.raises(bc.BoxCodeError):         # index out of range
        bc.Tree(hctx, [0], [1], [0])
    # unbalanced: level-3 leaf (3,3,0) touches the level-1 leaf (1,1,0)
    leaves = {(1, 1, 0), (1, 0, 1), (1, 1, 1), (2, 0, 0), (2, 0, 1), (2, 1, 1),
              (3, 2, 0), (3, 3, 0), (3, 2, 1), (3, 3, 1)}
    arr = np.array(sorted(leaves))
    with pytest.raises(bc.BoxCodeError) as e:
        bc.Tree(hctx, arr[:, 0], arr[:, 1], arr[:, 2])
    assert "balanced" in str(e.value)
    # the balanced version is accepted
    arr = np.array(sorted(synth.balance_leaves(leaves)))
    t = bc.Tree(hctx, arr[:, 0], arr[:, 1], arr[:, 2])
    assert t.nleaf == len(arr)


def _touch(a, b):
    (la, ia, ja), (lb, ib, jb) = a, b
    lf = max(la, lb)
    a0, a1 = ia << (lf - la), (ia + 1) << (lf - la)
    c0, c1 = ja << (lf - la), (ja + 1) << (lf - la)
    b0, b1 = ib << (lf - lb), (ib + 1) << (lf - lb)
    d0, d1 = jb << (lf - lb), (jb + 1) << (lf - lb)
    return a0 <= b1 and b0 <= a1 and c0 <= d1 and d0 <= c1 and not (a0 < b1 and b0 < a1 and c0 < d1 and d0 < c1)


def _check_lists(tree):
    blv, bix, biy, bpar, bleaf = tree.boxes()
    nb = blv.shape[0]
    lv, ix, iy = tree.leaves()
    nleaf = lv.shape[0]
    leaf_box = np.full(nleaf, -1)
    for b in range(nb):
        if bleaf[b] >= 0:
            leaf_box[bleaf[b]] = b
    # descendants-or-self leaves of each box
    desc = [set() for _ in range(nb)]
    for k in range(nleaf):
        b = leaf_box[k]
        while b >= 0:
            desc[b].add(k)
            b = bpar[b]
    near, vl, wl, xl = (tree.lists(k) for k in range(4))
    cover = np.zeros((nleaf, nleaf), dtype=np.int64)
    for t in range(nleaf):
        # (a) near list, validated geometrically
        for e in range(near[0][t], near[0][t + 1]):
            s = near[1][e]
            assert s == t or _touch((lv[t], ix[t], iy[t]), (lv[s], ix[s], iy[s]))
            assert abs(int(lv[t]) - int(lv[s])) <= 1
            cover[t, s] += 1
        # (b) W list: subtrees
        for e in range(wl[0][t], wl[0][t + 1]):
            w = wl[1][e]
            assert blv[w] == lv[t] + 1
            for s in desc[w]:
                cover[t, s] += 1
        # (c),(d) ancestors
        a = leaf_box[t]
        while a >= 0:
            for e in range(xl[0][a], xl[0][a + 1]):
                cover[t, xl[1][e]] += 1
            for e in range(vl[0][a], vl[0][a + 1]):
                v = vl[1][e]
                assert blv[v] == blv[a]
                assert not _touch((blv[v], bix[v], biy[v]), (blv[a], bix[a], biy[a]))
                for s in desc[v]:
                    cover[t, s] += 1
            a = bpar[a]
    assert np.all(cover == 1), np.argwhere(cover != 1)[:5]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lists_cover_every_pair_once(hctx, seed):
    g = synth.gaussians(4, 500 + seed, wlog10=(-2.2, -1.0))
    lv, ix, iy = synth.geometric_leaves(g, kappa=1.0, max_level=6)
    tree = bc.Tree(hctx, lv, ix, iy)
    assert tree.stats()["nlevels"] >= 5
    _check_lists(tree)


def test_uniform_tree_counts(hctx):
    lv, ix, iy = synth.uniform_leaves(3)
    t = bc.Tree(hctx, lv, ix, iy)
    s = t.stats()
    assert s["nleaf"] == 64 and s["nbox"] == 85 and s["nlevels"] == 4
    assert s["n_w"] == 0 and s["n_x"] == 0
    # interior leaves have 9 near slots, edges 6, corners 4
    assert s["n_near"] == 36 * 9 + 24 * 6 + 4 * 4
    _check_lists(t)


def test_refine_resolves_and_balances(hctx):
    g = synth.gaussians(3, 9, wlog10=(-1.6, -1.0))
    t = bc.Tree.refine(hctx, g, eps=1e-9, max_level=10)
    lv, ix, iy = t.leaves()
    leaves = set(zip(lv.tolist(), ix.tolist(), iy.tolist()))
    assert synth.balance_leaves(leaves) == leaves        # already 2:1 balanced
    # every leaf resolves f: interpolation error at random points is small
    import oracle
    p = hctx.p
    geom = synth.leaf_geometry(lv, ix, iy)
    f = g(oracle.leaf_nodes(geom, p))
    rng = np.random.default_rng(0)
    worst = 0.0
    for b in rng.choice(len(lv), min(40, len(lv)), replace=False):
        q = rng.uniform(-1, 1, (16, 2))
        fi = oracle.interp(p, f[b], q)
        fe = g(geom[b, :2] + geom[b, 2] * q)
        worst = max(worst, np.abs(fi - fe).max())
    assert worst < 1e-6 * np.abs(f).max()


def test_nodes_match_independent_formula(hctx):
    import oracle
    lv, ix, iy = synth.geometric_leaves(synth.gaussians(2, 3, wlog10=(-1.5, -1.0)), max_level=5)
    t = bc.Tree(hctx, lv, ix, iy, x0=-0.5, y0=0.25, L=1.5)
    want = oracle.leaf_nodes(synth.leaf_geometry(lv, ix, iy, -0.5, 0.25, 1.5), hctx.p)
    assert np.abs(t.nodes() - want).max() < 1e-15


def _table_geometry(k):
    if k < 9:
        return (k % 3 - 1) * 2.0, (k // 3 - 1) * 2.0, 1.0, True
    if k < 25:
        i, j = (k - 9) % 4, (k - 9) // 4
        g2x, g2y = 2 * i - 3, 2 * j - 3
        return 0.5 * g2x, 0.5 * g2y, 0.5, not (abs(g2x) <= 1 and abs(g2y) <= 1)
    i, j = (k - 25) % 4, (k - 25) // 4
    gx, gy = 2 * i - 3, 2 * j - 3
    return float(gx), float(gy), 2.0, not (abs(gx) <= 1 and abs(gy) <= 1)


@pytest.mark.parametrize("p", [8, 16])
def test_near_table_row_sums_closed_form(p):
    ctx = bc.Context(p=p, device=-1, cache_dir=None)
    T = ctx.table(2).reshape(41, p * p, p * p)
    x = ctx.table(0)
    nvalid = 0
    for k in range(41):
        gx, gy, rho, valid = _table_geometry(k)
        if not valid:
            assert not T[k].any()
            continue
        nvalid += 1
        xi = gx + rho * np.tile(x, p)
        eta = gy + rho * np.repeat(x, p)
        ex = np.array([square_potential(a, b) for a, b in zip(xi, eta)])
        assert np.abs(T[k].sum(axis=1) - ex).max() < 4e-15 * max(1.0, np.abs(ex).max()), k
    assert nvalid == 33
    w = ctx.table(1)
    assert abs(w.sum() - 4.0) < 1e-14


def test_self_table_centre_value():
    """p odd puts a node at the centre: its self-table row sums to (2 ln 2 + pi - 6)/2pi."""
    p = 5
    ctx = bc.Context(p=p, device=-1, cache_dir=None)
    T = ctx.table(2).reshape(41, p * p, p * p)
    centre = (p // 2) * p + p // 2
    assert abs(T[4, centre].sum() - (2 * math.log(2) + math.pi - 6) / (2 * math.pi)) < 1e-14


def test_tables_reflection_symmetry():
    """Reflecting x -> -x maps the colleague table at offset g to the one at
    (-gx, gy) with the source and target node columns mirrored in x."""
    p = 8
    ctx = bc.Context(p=p, device=-1, cache_dir=None)
    T = ctx.table(2).reshape(41, p, p, p, p)           # [k][ty][tx][sy][sx]
    pairs = [(3, 5), (0, 2), (6, 8), (9 + 0, 9 + 3), (25 + 4, 25 + 7)]
    for a, b in pairs:
        ref = T[b][:, ::-1, :, ::-1]
        assert np.abs(T[a] - ref).max() < 2e-16 * 64 * max(1.0, np.abs(T[a]).max()), (a, b)


def test_far_operators_consistency():
    """P2M then L2P-free checks: M2M of a child's multipole equals the parent's
    multipole from the same density (P2M of the parent's interpolant) to
    rounding, and M2L(d) agrees with the direct local expansion formula."""
    p, P1 = 8, 24
    ctx = bc.Context(p=p, nterms=P1, device=-1, cache_dir=None)
    Q = ctx.table(3).view(complex).reshape(P1, p * p)
    M2M = ctx.table(5).view(complex).reshape(4, P1, P1)
    x = ctx.table(0)
    # density: polynomial of degree < p/2 so that it is exactly representable on a child
    rng = np.random.default_rng(4)
    c = rng.standard_normal((3, 3))
    poly = lambda X, Y: sum(c[i, j] * X ** i * Y ** j for i in range(3) for j in range(3))
    X, Y = np.meshgrid(x, x, indexing="xy")
    # parent = [-1,1]^2 (r=1), children r=1/2 at centres (+-1/2, +-1/2)
    A_par = Q @ poly(X, Y).ravel()
    A_sum = np.zeros(P1, complex)
    for q in range(4):
        cx, cy = (q & 1) - 0.5, (q >> 1) - 0.5
        A_child = 0.25 * (Q @ poly(cx + 0.5 * X, cy + 0.5 * Y).ravel())
        A_sum += M2M[q] @ A_child
    assert np.abs(A_sum - A_par).max() < 1e-14 * np.abs(A_par).max()


@pytest.mark.parametrize("nterms", [8, 24, 31])
def test_up_schedule_covers_each_term_once(nterms):
    """Host logic of the double-float climb's term schedule, both directions:
    the shifts are lower-triangular (output l reads inputs k <= l); the lane
    runs cover every term exactly once, with zero padding only after a lane's
    last partial sum; every partial-sum slot of an output is ended by exactly
    one lane; the entries are the operator's to double-float rounding; and
    the scheduled sums reproduce the dense shift."""
    P1 = nterms
    ctx = bc.Context(p=8, nterms=P1, device=-1, cache_dir=None)
    lib = bc._load()
    M2M = ctx.table(5).view(complex).reshape(4, P1, P1)
    L2L = ctx.table(6).view(complex).reshape(4, P1, P1)
    rng = np.random.default_rng(P1)
    for adj in (0, 1):
        # the operator in the schedule's layout up[q][k][l] (output l, input k):
        # forward M2M_q[l][k], adjoint conj(L2L_q[k][l])
        up = np.conj(L2L) if adj else np.transpose(M2M, (0, 2, 1))
        nz = np.abs(up).max(axis=0) != 0
        terms = {(l, k) for k in range(P1) for l in range(P1) if nz[k, l]}
        assert terms == {(l, k) for l in range(P1) for k in range(l + 1)}
        Tc, mc = ctypes.c_int32(), ctypes.c_int32()
        bc._check(lib.bc_debug_up_schedule(ctx.handle, adj, ctypes.byref(Tc), ctypes.byref(mc), None, None, None))
        T, maxp = Tc.value, mc.value
        assert T == -(-len(terms) // 32)
        code = np.zeros((T, 32), np.uint32)
        ops = np.zeros((4, T, 32, 4), np.float32)
        nps = np.zeros(P1, np.int32)
        bc._check(lib.bc_debug_up_schedule(ctx.handle, adj, ctypes.byref(Tc), ctypes.byref(mc),
                                           code.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                           ops.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           nps.ctypes.data_as(bc._I32P)))
        opv = (ops[..., 0].astype(np.float64) + ops[..., 1]) + 1j * (ops[..., 2].astype(np.float64) + ops[..., 3])
        seen, ends = [], {}
        for lane in range(32):
            run = []
            for t in range(T):
                c = int(code[t, lane])
                run.append((t, c & 255))
                if c >> 8:
                    slot = (c >> 8) - 1
                    l = slot // maxp
                    assert slot % maxp < nps[l], (lane, t, slot)
                    ends[slot] = ends.get(slot, 0) + 1
                    for tt, k in run:
                        seen.append((l, k))
                        err = np.abs(opv[:, tt, lane] - up[:, k, l])
                        assert np.all(err <= 2.0 ** -46 * np.abs(up[:, k, l])), (l, k)
                    run = []
            for tt, k in run:   # padding after the lane's last partial sum
                assert k == 0 and not ops[:, tt, lane].any()
        assert len(seen) == len(terms) and set(seen) == terms
        assert len(ends) == int(nps.sum())
        assert all(ends.get(l * maxp + j) == 1 for l in range(P1) for j in range(nps[l]))
        x = rng.standard_normal((4, P1)) + 1j * rng.standard_normal((4, P1))
        out = np.zeros(P1, complex)
        for q in range(4):
            for lane in range(32):
                acc = 0.0
                for t in range(T):
                    c = int(code[t, lane])
                    acc += opv[q, t, lane] * x[q, c & 255]
                    if c >> 8:
                        out[((c >> 8) - 1) // maxp] += acc
                        acc = 0.0
        ref = np.einsum("qkl,qk->l", up, x)
        assert np.abs(out - ref).max() < 1e-13 * np.abs(ref).max()
