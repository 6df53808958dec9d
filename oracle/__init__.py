"""CPU FP64 oracle for the 2D volume potential on a Chebyshev quadtree.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (``paper_2501_17967_gb300``) never imports it, and this module
never imports the product.

It evaluates (paper Sec. 3.2, eq. (vbulk); Phi as in Sec. 2)

    u(x) = (1/2pi) * sum_B int_B log|x - y| f_B(y) dy

by direct singular quadrature per (target, leaf); see ``oracle.c`` for the
method.  It also evaluates the glue layer potential S[sigma] - D[tau] of
Sec. 3.4 on a discretised curve by direct summation (``layer``).  Nodes are first-kind Chebyshev points, ascending; leaf values are
stored [leaf][jy][jx].

Parity status of each function is stated in its docstring; every one is
pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(src)):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c11",
                           "-D_GNU_SOURCE", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_potential.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64, dp,
                                         i64p, i64p, dp, ctypes.c_int]
        lib.oracle_potential.restype = ctypes.c_int
        lib.oracle_gradient.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64, dp,
                                        i64p, i64p, dp, ctypes.c_int]
        lib.oracle_gradient.restype = ctypes.c_int
        lib.oracle_layer.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int]
        lib.oracle_layer.restype = ctypes.c_int
        lib.oracle_nodes.argtypes = [ctypes.c_int, dp]
        lib.oracle_nodes.restype = None
        lib.oracle_s_rule.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.oracle_s_rule.restype = ctypes.c_int
        lib.oracle_interp.argtypes = [ctypes.c_int, dp, ctypes.c_int64, dp, dp]
        lib.oracle_interp.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def cheb_nodes(p: int) -> np.ndarray:
    """First-kind Chebyshev nodes -cos((2j+1)pi/(2p)), ascending (paper Sec. 3.2.1
    leaves; node kind is a reading, the paper is silent)."""
    x = np.empty(p, dtype=np.float64)
    _load().oracle_nodes(p, _dp(x))
    return x


def leaf_geometry(levels, ix, iy, x0=-1.0, y0=-1.0, L=2.0):
    """(cx, cy, r) of dyadic leaves (level, ix, iy) of the root [x0,x0+L]x[y0,y0+L]."""
    levels = np.asarray(levels, dtype=np.int64)
    r = L * 0.5 / (2.0 ** levels)
    cx = x0 + (2 * np.asarray(ix, dtype=np.float64) + 1.0) * r
    cy = y0 + (2 * np.asarray(iy, dtype=np.float64) + 1.0) * r
    return np.stack([cx, cy, r], axis=1)


def leaf_nodes(geom: np.ndarray, p: int) -> np.ndarray:
    """Physical node coordinates [nleaf, p*p, 2] (x fastest within a leaf)."""
    x = cheb_nodes(p)
    gx = np.tile(x, p)          # jx fastest
    gy = np.repeat(x, p)
    cx, cy, r = geom[:, 0:1], geom[:, 1:2], geom[:, 2:3]
    return np.stack([cx + r * gx[None, :], cy + r * gy[None, :]], axis=2)


def potential(p: int, geom: np.ndarray, f: np.ndarray, targets: np.ndarray,
              sources=None, nthreads: int = 0) -> np.ndarray:
    """u at ``targets`` from all leaves (or a per-target CSR list of source leaves).

    geom: [nleaf, 3] (cx, cy, r); f: [nleaf, p, p] node values; targets: [n, 2].
    sources: None, or (ptr[n+1], idx) int64 arrays restricting the source leaves
    of each target (used for near-only / far-only parity restrictions).
    Pinned by the closed-form, scipy and symmetry tests.
    """
    geom = np.ascontiguousarray(geom, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(geom.shape[0], p * p)
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 2)
    out = np.empty(t.shape[0], dtype=np.float64)
    if sources is None:
        ptr = idx = None
        pp = ip = None
    else:
        ptr = np.ascontiguousarray(sources[0], dtype=np.int64)
        idx = np.ascontiguousarray(sources[1], dtype=np.int64)
        if ptr.shape[0] != t.shape[0] + 1 or (idx.size and (idx.min() < 0 or idx.max() >= geom.shape[0])):
            raise ValueError("bad source list")
        pp, ip = _ip(ptr), _ip(idx)
    rc = _load().oracle_potential(p, geom.shape[0], _dp(geom), _dp(f), t.shape[0], _dp(t),
                                  pp, ip, _dp(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_potential failed ({rc})")
    return out


def gradient(p: int, geom: np.ndarray, f: np.ndarray, targets: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """grad u at ``targets`` [n, 2] -> [n, 2]: (1/2pi) sum_B int_B (x - y)/|x - y|^2 f_B(y) dy,
    the derivative of eq. (vbulk) (the glue step of Sec. 3.4 needs the normal
    derivative of v_bulk on the fictitious curve).  Direct quadrature as in
    ``potential``: tensor Gauss-Legendre on admissible rectangles, Duffy rays
    from targets inside a leaf (the 1/r singularity cancels the ray Jacobian).
    Pinned by the rectangle and Gaussian closed forms and by central
    differences of ``potential``.
    """
    geom = np.ascontiguousarray(geom, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(geom.shape[0], p * p)
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 2)
    out = np.empty((t.shape[0], 2), dtype=np.float64)
    rc = _load().oracle_gradient(p, geom.shape[0], _dp(geom), _dp(f), t.shape[0], _dp(t), None, None,
                                 _dp(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_gradient failed ({rc})")
    return out


def layer(src: np.ndarray, q: np.ndarray, m: np.ndarray, targets: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """The glue potential S[sigma] - D[tau] of Sec. 3.4 discretised on curve
    nodes src[n, 2] with q_j = w_j sigma_j and dipoles m[n, 2] = w_j tau_j n_j:
    -(1/2pi) sum_j [q_j log|x - y_j| + m_j . (x - y_j)/|x - y_j|^2] at targets
    [nt, 2] (direct sum; coincident pairs skipped).  Pinned by the circle's
    closed forms (single layer -R log R inside, -R log|x| outside; double
    layer: Gauss's identity, 1 inside and 0 outside)."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1, 2)
    t = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 2)
    if q.shape[0] != src.shape[0] or m.shape[0] != src.shape[0]:
        raise ValueError("q, m and src differ in length")
    out = np.empty(t.shape[0], dtype=np.float64)
    if _load().oracle_layer(src.shape[0], _dp(src), _dp(q), _dp(m), t.shape[0], _dp(t), _dp(out),
                            int(nthreads)) != 0:
        raise RuntimeError("oracle_layer failed")
    return out


def potential_at_nodes(p, geom, f, leaf_ids=None, sources=None, nthreads=0):
    """u at all nodes of the given leaves (default: every leaf), shape [k, p*p]."""
    nodes = leaf_nodes(geom, p)
    if leaf_ids is not None:
        nodes = nodes[np.asarray(leaf_ids)]
    u = potential(p, geom, f, nodes.reshape(-1, 2), sources=sources, nthreads=nthreads)
    return u.reshape(nodes.shape[0], p * p)


def adjoint_columns(p, geom, g, columns, nthreads=0, target_leaves=None):
    """(A^T g)_j for sampled columns j = (leaf, node) of the discrete operator
    A_ij = (1/2pi) int_{B(j)} log|x_i - y| l_j(y) dy, x_i the leaf nodes.

    Each column is the potential of the Lagrange basis function l_j on its leaf,
    evaluated at the nodes and contracted with g (plain definition of A^T).
    g: values at every node ([nleaf, p*p]).  target_leaves: optional leaf ids;
    the contraction then runs over the nodes of those leaves only, which is
    (A^T g)_j itself when g vanishes at every other node.
    Pinned by tests/test_oracle_pins.py (transpose of oracle columns, scipy).
    """
    nodes = leaf_nodes(geom, p)
    g = np.asarray(g, dtype=np.float64).reshape(nodes.shape[0], p * p)
    if target_leaves is not None:
        tl = np.asarray(target_leaves, dtype=np.int64)
        nodes, g = nodes[tl], g[tl]
    nodes = nodes.reshape(-1, 2)
    g = g.reshape(-1)
    out = []
    for (b, j) in columns:
        e = np.zeros((1, p * p))
        e[0, j] = 1.0
        col = potential(p, geom[b:b + 1], e, nodes, nthreads=nthreads)
        out.append(float(np.dot(col, g)))
    return np.array(out)


def s_rule(ns: int):
    """Nodes/weights of the Duffy-ray rule: (s, w for s*g(s), w for s*log(s)*g(s))."""
    s = np.empty(ns); wr = np.empty(ns); wl = np.empty(ns)
    if _load().oracle_s_rule(ns, _dp(s), _dp(wr), _dp(wl)) != 0:
        raise ValueError("bad ns")
    return s, wr, wl


def interp(p: int, fvals: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """The leaf interpolant f_B at reference points (for pins of the node->coefficient map)."""
    fvals = np.ascontiguousarray(fvals, dtype=np.float64).reshape(p * p)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    out = np.empty(pts.shape[0])
    if _load().oracle_interp(p, _dp(fvals), pts.shape[0], _dp(pts), _dp(out)) != 0:
        raise ValueError("bad p")
    return out


def strip_assemble(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """The strip system of Sec. 3.3 as one dense matrix: N element blocks on a
    closed strip, block row k coupling x_(k-1), x_k and x_(k+1) (indices mod
    N) through C[k], A[k] and B[k] ([N, m, m] each); with N = 1 or 2 the
    blocks that land on the same position add up."""
    A, B, C = (np.asarray(t, dtype=np.float64) for t in (A, B, C))
    N, m = A.shape[0], A.shape[1]
    M = np.zeros((N * m, N * m))
    for k in range(N):
        r = slice(k * m, (k + 1) * m)
        M[r, k * m:(k + 1) * m] += A[k]
        kp, km = (k + 1) % N, (k - 1) % N
        M[r, kp * m:(kp + 1) * m] += B[k]
        M[r, km * m:(km + 1) * m] += C[k]
    return M


def strip_solve(A: np.ndarray, B: np.ndarray, C: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with sum over the block row of (C[k] x_(k-1) + A[k] x_k + B[k] x_(k+1)) = b[k]
    (Sec. 3.3's block-tridiagonal strip system with its periodic corners), by
    a dense solve of the assembled matrix.  b: [N, m, r] -> x: [N, m, r].
    Pinned by block-circulant systems solved through the block DFT and by
    the scalar periodic second-difference closed form."""
    b = np.asarray(b, dtype=np.float64)
    N, m, r = b.shape
    x = np.linalg.solve(strip_assemble(A, B, C), b.reshape(N * m, r))
    return x.reshape(N, m, r)
