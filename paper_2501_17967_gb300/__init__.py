"""GB300 machine code: the free-space 2D Laplace volume potential on an adaptive
quadtree of p x p Chebyshev leaves (the bulk step v_bulk of arXiv 2501.17967,
Sec. 3.2, eq. (vbulk)).

This package is a thin binding over the C ABI in ``include/boxcode.h``
(``libboxcode.so``, built in-tree by :func:`build`).  Every step of the
computation runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch supplies device memory and streams.  There is no CPU
fallback: without the compiled library and a GPU the calls raise.

    u(x_i) = (1/2pi) sum_B int_B log|x_i - y| f_B(y) dy,   Laplace(u) = f
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

__all__ = ["build", "Context", "Tree", "Batch", "BoxCodeError", "FP64", "SPLIT_BF16", "SPLIT_BF16_ALL", "apply",
           "apply_adjoint", "eval_points", "eval_points_grad", "Layer", "strip_solve", "strip_workspace", "BoxCodeApply", "lib_path"]

# precision modes (bc_precision): FP64 everywhere; BF16 digit products for the
# fixed-operator contractions (near field, P2M, L2P, W and X lists) with the
# M2L, the shifts, the log terms and every sum in FP64; the same plus the M2L
# on BF16 digits and the shifts in double-float
FP64 = 0
SPLIT_BF16 = 1
SPLIT_BF16_ALL = 2
SPLIT_ORDERS = (8, 12, 16)    # orders p with a split-precision path
_STATUS = {0: "BC_OK", -1: "BC_ERR_ARG", -2: "BC_ERR_TREE", -3: "BC_ERR_CUDA", -4: "BC_ERR_OOM",
           -5: "BC_ERR_TIMEOUT", -6: "BC_ERR_UNSUPPORTED", -7: "BC_ERR_STATE"}
_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tables")

_lib = None


class BoxCodeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("nterms", ctypes.c_int), ("node_kind", ctypes.c_int),
                ("split_slices", ctypes.c_int), ("autotune", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("nleaf", "nbox", "nlevels", "n_near", "n_v", "n_w", "n_x",
                                               "n_nonleaf", "n_down")]


DENSITY_FN = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                              ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)

# (name, restype, argtypes) of every exported symbol
_VP, _I64, _I32P, _DP = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("bc_create", ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_int, ctypes.POINTER(_VP)]),
    ("bc_destroy", None, [_VP]),
    ("bc_last_error", ctypes.c_char_p, []),
    ("bc_tables_build", ctypes.c_int, [_VP, ctypes.c_char_p]),
    ("bc_tree_create", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I64, _I32P, _I32P,
                                      _I32P, ctypes.POINTER(_VP)]),
    ("bc_tree_refine", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, DENSITY_FN, _VP,
                                      ctypes.c_double, ctypes.c_int, ctypes.POINTER(_VP)]),
    ("bc_tree_refine_truncated", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, DENSITY_FN,
                                                _VP, ctypes.c_double, ctypes.c_int, _DP, _I64, _DP, _I64,
                                                ctypes.POINTER(_VP)]),
    ("bc_tree_leaf_class", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int8)]),
    ("bc_tree_node_mask", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint8)]),
    ("bc_tree_nleaf", _I64, [_VP]),
    ("bc_tree_leaves", ctypes.c_int, [_VP, _I32P, _I32P, _I32P]),
    ("bc_tree_nodes", ctypes.c_int, [_VP, _DP]),
    ("bc_tree_stats_get", ctypes.c_int, [_VP, ctypes.POINTER(_Stats)]),
    ("bc_tree_lists", ctypes.c_int, [_VP, ctypes.c_int, _I64P, _I64P, _I64P, _I64P, _I32P]),
    ("bc_tree_boxes", ctypes.c_int, [_VP, _I32P, _I32P, _I32P, _I32P, _I32P]),
    ("bc_tree_destroy", None, [_VP]),
    ("bc_apply", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    ("bc_apply_adjoint", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    ("bc_eval_points", ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _VP, _VP]),
    ("bc_eval_points_grad", ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    ("bc_layer_create", ctypes.c_int, [_VP, _DP, _I64, ctypes.POINTER(_VP)]),
    ("bc_layer_apply", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    ("bc_layer_info", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    ("bc_debug_log_inv", ctypes.c_int, [ctypes.c_int, _VP, _I64, _VP, _VP, _VP]),
    ("bc_layer_destroy", None, [_VP]),
    ("bc_strip_workspace", ctypes.c_int, [_I64, _I64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    ("bc_strip_solve", ctypes.c_int, [_I64, _I64, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                      _VP]),
    ("bc_batch_create", ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)]),
    ("bc_batch_destroy", None, [_VP]),
    ("bc_batch_nleaf", _I64, [_VP]),
    ("bc_batch_run", ctypes.c_int, [_VP, _VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int,
                                    _VP]),
    ("bc_batch_autotune", ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    ("bc_batch_shape", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    ("bc_table_export", ctypes.c_int, [_VP, ctypes.c_int, _I64P, _DP]),
    ("bc_set_option", ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_double]),
    ("bc_debug_set", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    ("bc_debug_stage_times", ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    ("bc_debug_up_schedule", ctypes.c_int, [_VP, ctypes.c_int, _I32P, _I32P, ctypes.POINTER(ctypes.c_uint32),
                                            ctypes.POINTER(ctypes.c_float), _I32P]),
    ("bc_debug_fp64_peak", ctypes.c_int, [ctypes.c_int, _DP]),
    ("bc_apply_noalloc", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    ("bc_sync", ctypes.c_int, [_VP, _VP]),
]


def build(force: bool = False) -> str:
    """Compile libboxcode.so for sm_103a (in-tree) and return its path."""
    return _build_mod.build(force=force)


def lib_path() -> str:
    return _build_mod.LIB


def _load():
    global _lib
    if _lib is None:
        path = _build_mod.build()
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status):
    if status != 0:
        msg = _load().bc_last_error()
        raise BoxCodeError(status, msg.decode() if msg else "")


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I32P)


class Context:
    """Order-p context on one CUDA device (device=-1: host-only, for inspection)."""

    def __init__(self, p: int = 16, nterms: int = 0, device: int = 0, split_slices: int = 0,
                 cache_dir: str | None = _DEFAULT_CACHE, build_tables: bool = True, autotune: bool = False):
        lib = _load()
        cfg = _Config(p, nterms, 1, split_slices, int(autotune))
        h = _VP()
        _check(lib.bc_create(ctypes.byref(cfg), device, ctypes.byref(h)))
        self._h = h
        self.p = p
        self.device = device
        self.nterms = nterms
        if build_tables:
            if cache_dir:
                os.makedirs(cache_dir, exist_ok=True)
            _check(lib.bc_tables_build(h, cache_dir.encode() if cache_dir else None))

    @property
    def handle(self):
        return self._h

    def table(self, which: int) -> np.ndarray:
        """Host copy of a table (see bc_table_export)."""
        lib = _load()
        n = ctypes.c_int64()
        _check(lib.bc_table_export(self._h, which, ctypes.byref(n), None))
        out = np.empty(n.value)
        _check(lib.bc_table_export(self._h, which, ctypes.byref(n), out.ctypes.data_as(_DP)))
        return out

    def set_option(self, name: str, value: float):
        """Runtime option (see bc_set_option), e.g. set_option("m2l_triangular", 1)."""
        _check(_load().bc_set_option(self._h, name.encode(), float(value)))

    def debug(self, pass_mask: int = 3, timing: bool = False):
        """Diagnostics: restrict applies to the near (1) / far (2) field; time stages."""
        _check(_load().bc_debug_set(self._h, pass_mask, int(timing)))

    STAGES = ("tensor_v", "clear", "upward", "m2l", "down_levels", "tensor_e", "leaf_output", "tensor_near")

    def stage_times(self, adjoint: bool = False):
        """Durations (ms) of the last forward/adjoint apply's stages (see STAGES)."""
        ms = np.zeros(len(self.STAGES))
        _check(_load().bc_debug_stage_times(self._h, int(adjoint), ms.ctypes.data_as(_DP)))
        return ms

    def close(self):
        if getattr(self, "_h", None):
            _load().bc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree:
    """A 2:1-balanced quadtree of leaves (level, ix, iy) of the root [x0,x0+L]^2."""

    def __init__(self, ctx: Context, level, ix, iy, x0=-1.0, y0=-1.0, L=2.0, _handle=None):
        lib = _load()
        self.ctx = ctx
        self.x0, self.y0, self.L = float(x0), float(y0), float(L)
        if _handle is None:
            lv, plv = _i32(level)
            ax, pix = _i32(ix)
            ay, piy = _i32(iy)
            if not (lv.shape == ax.shape == ay.shape) or lv.ndim != 1:
                raise ValueError("level, ix, iy must be 1-D arrays of equal length")
            h = _VP()
            _check(lib.bc_tree_create(ctx.handle, x0, y0, L, lv.shape[0], plv, pix, piy, ctypes.byref(h)))
            self._h = h
        else:
            self._h = _handle
        self.nleaf = int(lib.bc_tree_nleaf(self._h))

    @classmethod
    def refine(cls, ctx: Context, density, eps: float = 1e-11, max_level: int = 20, x0=-1.0, y0=-1.0, L=2.0):
        """Adaptive tree (Alg. 2 resolution criterion + 2:1 balance); density(xy[n,2]) -> f[n]."""
        lib = _load()
        err = []

        def cb(xy, n, out, user):
            try:
                pts = np.ctypeslib.as_array(xy, shape=(n, 2))
                vals = np.asarray(density(pts), dtype=np.float64).reshape(n)
                np.ctypeslib.as_array(out, shape=(n,))[:] = vals
            except Exception as exc:  # report after the call
                err.append(exc)
                np.ctypeslib.as_array(out, shape=(n,))[:] = np.nan

        cfn = DENSITY_FN(cb)
        h = _VP()
        st = lib.bc_tree_refine(ctx.handle, x0, y0, L, cfn, None, eps, max_level, ctypes.byref(h))
        if err:
            raise err[0]
        _check(st)
        return cls(ctx, None, None, None, x0, y0, L, _handle=h)

    @classmethod
    def refine_truncated(cls, ctx: Context, density, gamma, gamma_b, eps: float = 1e-11, max_level: int = 20,
                         x0=-1.0, y0=-1.0, L=2.0):
        """Truncated adaptive tree (Alg. 2 with both criteria, 2:1 balance): the domain
        bounded by the closed polygon gamma [n, 2], the bulk region by gamma_b [m, 2];
        density(xy[n,2]) -> f[n] is called at nodes inside the domain only."""
        lib = _load()
        err = []

        def cb(xy, n, out, user):
            try:
                pts = np.ctypeslib.as_array(xy, shape=(n, 2))
                vals = np.asarray(density(pts), dtype=np.float64).reshape(n)
                np.ctypeslib.as_array(out, shape=(n,))[:] = vals
            except Exception as exc:  # report after the call
                err.append(exc)
                np.ctypeslib.as_array(out, shape=(n,))[:] = np.nan

        g = np.ascontiguousarray(gamma, dtype=np.float64).reshape(-1, 2)
        gb = np.ascontiguousarray(gamma_b, dtype=np.float64).reshape(-1, 2)
        cfn = DENSITY_FN(cb)
        h = _VP()
        st = lib.bc_tree_refine_truncated(ctx.handle, x0, y0, L, cfn, None, eps, max_level, g.ctypes.data_as(_DP),
                                          g.shape[0], gb.ctypes.data_as(_DP), gb.shape[0], ctypes.byref(h))
        if err:
            raise err[0]
        _check(st)
        return cls(ctx, None, None, None, x0, y0, L, _handle=h)

    def leaf_class(self) -> np.ndarray:
        """0 outside the domain (discarded), 1 cut by its boundary, 2 inside."""
        out = np.empty(self.nleaf, np.int8)
        _check(_load().bc_tree_leaf_class(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))))
        return out

    def node_mask(self) -> np.ndarray:
        """[nleaf, p*p]: 1 where the node lies inside the domain (the zero extension of f)."""
        out = np.empty((self.nleaf, self.ctx.p * self.ctx.p), np.uint8)
        _check(_load().bc_tree_node_mask(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
        return out

    @property
    def handle(self):
        return self._h

    def leaves(self):
        n = self.nleaf
        lv, ix, iy = (np.empty(n, np.int32) for _ in range(3))
        _check(_load().bc_tree_leaves(self._h, lv.ctypes.data_as(_I32P), ix.ctypes.data_as(_I32P),
                                      iy.ctypes.data_as(_I32P)))
        return lv, ix, iy

    def nodes(self) -> np.ndarray:
        out = np.empty((self.nleaf, self.ctx.p * self.ctx.p, 2))
        _check(_load().bc_tree_nodes(self._h, out.ctypes.data_as(_DP)))
        return out

    def stats(self) -> dict:
        s = _Stats()
        _check(_load().bc_tree_stats_get(self._h, ctypes.byref(s)))
        return {n: int(getattr(s, n)) for n, _ in _Stats._fields_}

    def lists(self, kind: int):
        lib = _load()
        nr, nz = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.bc_tree_lists(self._h, kind, ctypes.byref(nr), ctypes.byref(nz), None, None, None))
        ptr = np.empty(nr.value + 1, np.int64)
        idx = np.empty(nz.value, np.int64)
        code = np.empty(nz.value, np.int32)
        _check(lib.bc_tree_lists(self._h, kind, ctypes.byref(nr), ctypes.byref(nz), ptr.ctypes.data_as(_I64P),
                                 idx.ctypes.data_as(_I64P), code.ctypes.data_as(_I32P)))
        return ptr, idx, code

    def boxes(self):
        lib = _load()
        nb = self.stats()["nbox"]
        arrs = [np.empty(nb, np.int32) for _ in range(5)]
        _check(lib.bc_tree_boxes(self._h, *[a.ctypes.data_as(_I32P) for a in arrs]))
        return tuple(arrs)   # level, ix, iy, parent, leaf

    def close(self):
        if getattr(self, "_h", None):
            _load().bc_tree_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp64_peak_tflops(device: int = 0) -> float:
    """Measured FP64 FMA throughput of the device (TFLOP/s)."""
    v = ctypes.c_double()
    _check(_load().bc_debug_fp64_peak(device, ctypes.byref(v)))
    return v.value


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_tensor(x, tree: Tree, name):
    import torch
    n = tree.nleaf * tree.ctx.p * tree.ctx.p
    if not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or x.numel() != n or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 tensor with {n} elements")


def apply(tree: Tree, f, out=None, precision: int = FP64, stream=None):
    """u = A f (device or pinned/host float64 tensors of shape [nleaf, p, p] or flat)."""
    import torch
    _check_tensor(f, tree, "f")
    if out is None:
        out = torch.empty_like(f)
    _check_tensor(out, tree, "out")
    _check(_load().bc_apply(tree.ctx.handle, tree.handle, ctypes.c_void_p(f.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), precision,
                            _stream_ptr(stream) if f.is_cuda else None))
    return out


def apply_adjoint(tree: Tree, g, out=None, precision: int = FP64, stream=None):
    """h = A^T g (exact transpose of the discrete operator of :func:`apply`)."""
    import torch
    _check_tensor(g, tree, "g")
    if out is None:
        out = torch.empty_like(g)
    _check_tensor(out, tree, "out")
    _check(_load().bc_apply_adjoint(tree.ctx.handle, tree.handle, ctypes.c_void_p(g.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), precision,
                                    _stream_ptr(stream) if g.is_cuda else None))
    return out


def eval_points(tree: Tree, u, xy, out=None, stream=None):
    """Interpolate leaf-node values u at points xy[n, 2] (device tensors)."""
    import torch
    _check_tensor(u, tree, "u")
    xy = xy.contiguous()
    n = xy.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=xy.device)
    _check(_load().bc_eval_points(tree.ctx.handle, tree.handle, ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(xy.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                  _stream_ptr(stream) if xy.is_cuda else None))
    return out


def eval_points_grad(tree: Tree, u, xy, stream=None):
    """Value and gradient of the leaf interpolant of u at points xy[n, 2]
    (device tensors): returns (val[n], grad[n, 2])."""
    import torch
    _check_tensor(u, tree, "u")
    xy = xy.contiguous()
    n = xy.shape[0]
    val = torch.empty(n, dtype=torch.float64, device=xy.device)
    grad = torch.empty((n, 2), dtype=torch.float64, device=xy.device)
    _check(_load().bc_eval_points_grad(tree.ctx.handle, tree.handle, ctypes.c_void_p(u.data_ptr()),
                                       ctypes.c_void_p(xy.data_ptr()), n, ctypes.c_void_p(val.data_ptr()),
                                       ctypes.c_void_p(grad.data_ptr()),
                                       _stream_ptr(stream) if xy.is_cuda else None))
    return val, grad


class Layer:
    """Point sources on a curve (the fictitious curve of Sec. 3.4) in the
    leaves of a tree, for the FMM evaluation of the glue potential
    S[sigma] - D[tau] at every leaf node: u = -(1/2pi) sum_j [q_j log|x - y_j|
    + m_j.(x - y_j)/|x - y_j|^2] with q_j = w_j sigma_j, m_j = w_j tau_j n_j.
    The layer keeps the tree alive and shares its workspaces."""

    def __init__(self, tree: Tree, xy):
        self.tree = tree
        pts = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self.n = pts.shape[0]
        h = _VP()
        _check(_load().bc_layer_create(tree.handle, pts.ctypes.data_as(_DP), self.n, ctypes.byref(h)))
        self._h = h

    def info(self) -> dict:
        c = (ctypes.c_int64 * 6)()
        _check(_load().bc_layer_info(self._h, c))
        return dict(zip(("sources", "n_v", "n_w", "n_x", "near_pairs", "leaves_with_sources"), (int(v) for v in c)))

    def apply(self, q, m, out=None, stream=None, precision: int = 0):
        """u at every leaf node ([nleaf * p * p]) from charges q[n] and dipoles
        m[n, 2]; device tensors (on `stream`) or host tensors.  precision FP64,
        or SPLIT_BF16: the L2P at every leaf on the tensor cores (p = 8, 12, 16)."""
        import torch
        q = q.contiguous()
        m = m.contiguous()
        if q.dtype != torch.float64 or m.dtype != torch.float64 or q.numel() != self.n or m.numel() != 2 * self.n:
            raise ValueError("q must be float64 [n] and m float64 [n, 2]")
        NP = self.tree.ctx.p ** 2
        if out is None:
            out = torch.empty(self.tree.nleaf * NP, dtype=torch.float64, device=q.device)
        _check(_load().bc_layer_apply(self.tree.ctx.handle, self._h, ctypes.c_void_p(q.data_ptr()),
                                      ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      int(precision), _stream_ptr(stream) if q.is_cuda else None))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _load().bc_layer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def strip_workspace(nsys: int, N: int, m: int, r: int, device=None):
    """A scratch tensor large enough for strip_solve of these shapes."""
    import torch
    nbytes = ctypes.c_int64()
    _check(_load().bc_strip_workspace(nsys, N, m, r, ctypes.byref(nbytes)))
    return torch.empty(max(1, (nbytes.value + 7) // 8), dtype=torch.float64, device=device)


def strip_solve(A, B, C, b, stream=None, return_status=False, out=None, work=None, status=None):
    """Batched strip systems of Sec. 3.3 (block tridiagonal with periodic
    corners): C[k] x[k-1] + A[k] x[k] + B[k] x[k+1] = b[k], indices mod N.
    A, B, C: float64 device tensors [nsys, N, m, m]; b: [nsys, N, m, r].
    Returns x (and the per-system status if asked: 1 = zero pivot).  With
    the same tensors (out, work and status passed in too) a large-block
    solve replays its captured launch graph."""
    import torch
    A, B, C, b = (t.contiguous() for t in (A, B, C, b))
    if b.dim() != 4 or A.shape != B.shape or A.shape != C.shape or A.shape[:3] != b.shape[:3] \
            or A.shape[2] != A.shape[3] or any(t.dtype != torch.float64 for t in (A, B, C, b)):
        raise ValueError("A, B, C must be float64 [nsys, N, m, m] and b float64 [nsys, N, m, r]")
    nsys, N, m, r = (int(v) for v in b.shape)
    lib = _load()
    if work is None:
        work = strip_workspace(nsys, N, m, r, b.device)
    x = torch.empty_like(b) if out is None else out
    if status is None:
        status = torch.zeros(max(1, nsys), dtype=torch.int32, device=b.device)
    _check(lib.bc_strip_solve(nsys, N, m, r, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                              ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(work.data_ptr()),
                              ctypes.c_void_p(status.data_ptr()), _stream_ptr(stream)))
    return (x, status[:nsys]) if return_status else x


class Batch:
    """Many trees of one context applied together (one launch per pass, CUDA graph)."""

    def __init__(self, ctx: Context, trees):
        self.ctx = ctx
        self.trees = list(trees)   # kept alive while the batch exists
        arr = (_VP * len(self.trees))(*[t.handle for t in self.trees])
        h = _VP()
        _check(_load().bc_batch_create(ctx.handle, arr, len(self.trees), ctypes.byref(h)))
        self._h = h

    @property
    def nleaf(self) -> int:
        return int(_load().bc_batch_nleaf(self._h))

    def run(self, ins, outs, precision: int = FP64, adjoint: bool = False, stream=None):
        n = len(self.trees)
        for t, x, y in zip(self.trees, ins, outs):
            _check_tensor(x, t, "input")
            _check_tensor(y, t, "output")
        ip = (_VP * n)(*[ctypes.c_void_p(x.data_ptr()) for x in ins])
        op = (_VP * n)(*[ctypes.c_void_p(y.data_ptr()) for y in outs])
        _check(_load().bc_batch_run(self.ctx.handle, self._h, ip, op, precision, int(adjoint), _stream_ptr(stream)))
        return outs

    def autotune(self, precision: int = FP64, stream=None):
        _check(_load().bc_batch_autotune(self.ctx.handle, self._h, precision, _stream_ptr(stream)))
        return {d: self.shape(precision, d) for d in (0, 1)}

    def shape(self, precision: int = FP64, adjoint: int = 0):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(_load().bc_batch_shape(self._h, precision, adjoint, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            _load().bc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class BoxCodeApply(torch.autograd.Function):
        """u = A f with dL/df = A^T dL/du (the hand-written adjoint kernels)."""

        @staticmethod
        def forward(ctx, f, tree, precision=FP64):
            ctx.tree = tree
            ctx.precision = precision
            return apply(tree, f.contiguous(), precision=precision)

        @staticmethod
        def backward(ctx, g):
            return apply_adjoint(ctx.tree, g.contiguous(), precision=ctx.precision), None, None

    return BoxCodeApply


def __getattr__(name):
    if name == "BoxCodeApply":
        cls = _autograd()
        globals()["BoxCodeApply"] = cls
        return cls
    raise AttributeError(name)
