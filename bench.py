"""Throughput of the GB300 machine code: leaf nodes per second for one forward plus
one adjoint volume-potential apply, on the 200-Gaussian adaptive workload.

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--precision split|split_all|fp64] [--workload adaptive200|adaptive20|batch64]
                    [--impl ours|reference]

Workload (default): root [-1,1]^2, p = 16, density = 200 Gaussians (centres
U[-0.5,0.5]^2, widths log-uniform in [1e-4, 1e-1], amplitudes N(0,1), seed
2), quadtree refined by the library (Alg. 2 resolution criterion,
eps = 1e-11) and 2:1 balanced: 14,191 leaves, 15 levels, 3.63M leaf nodes.
A step is one forward apply u = A f and one adjoint apply h = A^T g of the
whole tree; value = leaf nodes / (time of a step).  The headline precision
("split") takes the fixed-operator products (near field, P2M, L2P, W and X
lists) on BF16 tensor cores as exact digit products and keeps the
multipole-to-local translations, the M2M/L2L shifts, the log terms and
every sum in native FP64.  The same JSON line carries the native FP64 path,
the all-tensor split variant and the 20-Gaussian workload as extra keys, and
the error against the oracle per level, forward and adjoint.
With --gpus N every rank runs its own replica (the path does not shard; no
collective on the data path) and value is the total over ranks.
--impl reference times the CPU FP64 oracle (direct quadrature) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "leaf nodes/sec (p=16, <=1e-10 rel err) fwd+adjoint"
UNIT = "leaf nodes/s"
P = 16

WORKLOADS = {
    "adaptive200": (3, "adaptive 200-Gaussian quadtree (widths 1e-4..1e-1), p=16, eps=1e-11"),
    "adaptive20": (2, "adaptive 20-Gaussian quadtree (widths 1e-3..1e-1), p=16, eps=1e-11"),
    "batch64": (None, "64 adaptive trees (about 2e2..2e4 leaves, log-uniform), p in {8,12,16}, batched"),
    "layer": (None, "glue layer potential at every node of the star-shaped domain's truncated 200-Gaussian tree"),
    "strip": (None, "strip solve: batched block-tridiagonal systems with periodic corners"),
}
PRECISIONS = {"fp64": 0, "split": 1, "split_all": 2}
DTYPES = {
    0: "f64",
    1: "bf16 digits (5 slices, exact FP32 accumulation) for the near field, P2M, L2P, W and X lists; "
       "f64 for M2L, M2M/L2L, log terms and sums",
    2: "bf16 digits for every fixed-operator product including M2L; double-float (2 x f32) M2M/L2L; "
       "f64 log terms and sums",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="split", choices=list(PRECISIONS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adaptive200", choices=list(WORKLOADS))
    ap.add_argument("--nterms", type=int, default=24,
                    help="far-field expansion terms P+1: 24 keeps the truncation near 1e-12, inside the "
                         "1e-10 target of the metric (30 reaches FP64 rounding)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: no FP64 / all-tensor / 20-Gaussian lines, no oracle checks")
    ap.add_argument("--no-overlap", dest="overlap", action="store_false",
                    help="run the near-field tensor launch in line instead of beside the far-field passes "
                         "(the library's default, on an internal stream)")
    ap.add_argument("--profile-run", action="store_true",
                    help="only the warm-up and timed steps of the chosen precision (for profiler captures)")
    return ap.parse_args()


def density(workload):
    from paper_2501_17967_gb300 import synth
    return synth.config_density(WORKLOADS[workload][0])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle samples
def touching(lv, ix, iy, t):
    """Leaves touching leaf t (edge or corner), t included, from the dyadic indices."""
    L = int(lv.max())
    s = L - lv
    x0, x1 = ix << s, (ix + 1) << s
    y0, y1 = iy << s, (iy + 1) << s
    ok = (x0 <= x1[t]) & (x0[t] <= x1) & (y0 <= y1[t]) & (y0[t] <= y1)
    return np.nonzero(ok)[0]


def oracle_forward_sample(leaves, fvals, per_level, seed=11):
    """Oracle u at every node of per_level leaves of every level (timed)."""
    import oracle
    from paper_2501_17967_gb300 import synth
    lv, ix, iy = leaves
    geom = synth.leaf_geometry(lv, ix, iy)
    pick = synth.sample_leaves_per_level(lv, per_level, seed=seed)
    t0 = time.perf_counter()
    ref = oracle.potential_at_nodes(P, geom, fvals, leaf_ids=pick)
    return pick, ref, time.perf_counter() - t0


def adjoint_sample(leaves, seed=13, per_level=1, k_cols=3, n_rand=24):
    """g random on S (sampled column leaves, their neighbours, random leaves),
    zero elsewhere; columns on every level near and far from S."""
    from paper_2501_17967_gb300 import synth
    lv, ix, iy = leaves
    rng = np.random.default_rng(seed)
    near_cols = synth.sample_leaves_per_level(lv, per_level, seed=seed)
    far_cols = synth.sample_leaves_per_level(lv, per_level, seed=seed + 1)
    S = set()
    for b in near_cols:
        S.update(touching(lv, ix, iy, int(b)).tolist())
    S.update(rng.choice(len(lv), size=min(n_rand, len(lv)), replace=False).tolist())
    S = np.array(sorted(S), dtype=np.int64)
    cols = [(int(b), int(j)) for b in np.concatenate([near_cols, far_cols])
            for j in rng.choice(P * P, size=k_cols, replace=False)]
    g = np.zeros((len(lv), P * P))
    g[S] = rng.standard_normal((len(S), P * P))
    return S, cols, g


def per_level(levels, errs, scale):
    out = {}
    for lvl, e in zip(levels, errs):
        out[str(int(lvl))] = max(out.get(str(int(lvl)), 0.0), float(e) / scale)
    return {k: float(f"{v:.3e}") for k, v in sorted(out.items(), key=lambda kv: int(kv[0]))}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import paper_2501_17967_gb300 as bc
    from paper_2501_17967_gb300 import synth
    g = density(args.workload if args.workload != "batch64" else "adaptive200")
    hctx = bc.Context(p=P, device=-1, cache_dir=None, build_tables=False)
    tree = bc.Tree.refine(hctx, g, eps=1e-11, max_level=18)
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    geom = synth.leaf_geometry(lv, ix, iy)
    fvals = g(oracle.leaf_nodes(geom, P))
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    rng = np.random.default_rng(17)
    order = rng.permutation(len(lv))
    pos = 0

    def sample(seconds):
        nonlocal pos
        done, used, k = 0, 0.0, 1
        while used < seconds:
            ids = order[pos % len(order):pos % len(order) + k]
            pos += len(ids)
            t0 = time.perf_counter()
            oracle.potential_at_nodes(P, geom, fvals, leaf_ids=ids)
            used += time.perf_counter() - t0
            done += len(ids)
            k = min(2 * k, 16)
        return done * P * P, used

    for _ in range(args.warmup):
        sample(per_step / 4)
    nodes_tot, t_tot = 0, 0.0
    for _ in range(args.steps):
        n, t = sample(per_step)
        nodes_tot += n
        t_tot += t
    value = nodes_tot / t_tot / 2.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1], "nleaf": int(len(lv)),
                       "leaf_nodes": int(len(lv)) * P * P, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{nodes_tot} target nodes of randomly drawn leaves of the same tree over "
                                       f"{args.steps} steps (~{per_step:.0f}s each); forward rate halved for "
                                       f"fwd+adjoint (the transposed operator costs the same per entry)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
STAGES = ("tensor_v", "clear", "upward", "m2l", "down_levels", "tensor_e", "leaf_output", "tensor_near")
STAGE_KERNELS = {
    "tensor_v": "k_split_vec + k_split_gemm<256> (leaf-to-expansion; X list and near field too in line)",
    "clear": "k_clear_flags",
    "upward": "k_up_levels",
    "m2l": "k_m2l_boxes (FP64 M2L per target box; FP64 path also k_x_entries) | "
           "k_split_exp + k_split_gemm<64> (all-tensor split)",
    "down_levels": "k_down_warps | k_down_levels<double-float> (all-tensor split)",
    "tensor_e": "k_split_exp + k_split_gemm<64> (L2P and W list)",
    "leaf_output": "k_leaf_out",
    "tensor_near": "k_split_gemm<256> (X list, then near field, on the internal stream)",
}
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of each stage's
# kernel in the bench configuration, keyed by (workload, nterms, precision):
# filled from the ncu captures of the unchanged kernels, null otherwise
# (the FP64 M2L: mean of one forward and one adjoint launch)
TRAFFIC = {("adaptive200", 24, "split"): {"m2l": 10043776}}


def stage_work(st, nleaf, nleaf_far, P1, NP, prec):
    """Algorithmic work of each stage of one apply, counted from the tree's
    lists: (amount, kind), kind "tensor" (BF16 flops of the 15 digit products,
    rows x K x columns of the real operators), "fp64" (FP64 flops; a real x
    complex term counts 4, a complex x complex term 8) or "bytes"."""
    R = 2 * P1
    m2l64 = (4.0 * P1 * P1 + 14.0 * P1) * st["n_v"]          # factored form, per V pair
    shift64 = 4.0 * (P1 * (P1 + 1) / 2) + 12.0 * P1           # factored shift per child: binomial + diagonals
    up64 = 4 * shift64 * st["n_nonleaf"]
    down64 = shift64 * st["n_down"] + 2.0 * P1 * st["n_x"]
    if prec == 0:
        return {
            "tensor_v": (0.0, "tensor"), "tensor_near": (0.0, "tensor"), "clear": (0.0, "fp64"),
            "upward": (4.0 * P1 * NP * nleaf + up64, "fp64"),
            "m2l": (m2l64 + 4.0 * P1 * NP * st["n_x"], "fp64"),
            "down_levels": (down64, "fp64"),
            "tensor_e": (0.0, "tensor"),
            "leaf_output": (2.0 * NP * NP * st["n_near"] + 4.0 * P1 * NP * (nleaf_far + st["n_w"]), "fp64"),
        }
    w = {
        "tensor_v": (15 * 2.0 * NP * R * (nleaf + st["n_x"]), "tensor"),
        "tensor_near": (15 * 2.0 * NP * NP * st["n_near"], "tensor"),
        "clear": (0.0, "fp64"),
        "upward": (up64, "fp64"),
        "m2l": (m2l64, "fp64"),
        "down_levels": (down64, "fp64"),
        "tensor_e": (15 * 2.0 * R * NP * (nleaf_far + st["n_w"]), "tensor"),
        "leaf_output": (8.0 * NP * (st["n_near"] + st["n_w"] + nleaf_far + nleaf), "bytes"),
    }
    if prec == 2:
        w["m2l"] = (15 * 2.0 * R * R * st["n_v"], "tensor")
    return w


def launches_per_apply(prec, overlap, st):
    """Kernels of one apply (trees of more than three levels), as the launch
    list of the profiles shows them."""
    if prec == 0:
        return 1 + 1 + 1 + (1 if st["n_x"] > 0 else 0) + 1 + 2   # clear, up, M2L, X, down, leaf logs + leaf
    if prec == 1:
        # digits + P2M tiles, clear, up, FP64 M2L, down, L2P digits + tiles, logs + leaf; beside the M2L:
        # X tiles, multipole digits + W tiles, near field
        return 2 + 1 + 1 + 1 + 1 + 2 + 2 + (4 if overlap else 0)
    # all-tensor: digits + group V, clear, up, M2L digits + tiles, down, E digits + tiles, logs + leaf;
    # X tiles and near field on the internal stream
    return 2 + 1 + 1 + 2 + 1 + 2 + 2 + (2 if overlap else 0)


def run_batch64(args):
    import torch
    print(json.dumps(batch64_line(args, torch.cuda.current_device())))


def batch64_line(args, dev):
    """64 independent Gaussian-sum densities on their own adaptive trees, p in
    {8, 12, 16} round-robin; one batch (union of trees, CUDA graph, autotuned
    launch shapes) per order.  A step = forward + adjoint of all 64."""
    import torch

    import paper_2501_17967_gb300 as bc
    from paper_2501_17967_gb300 import synth
    ctxs = {p: bc.Context(p=p, nterms=args.nterms, device=dev) for p in (8, 12, 16)}
    groups = {8: [], 12: [], 16: []}
    t0 = time.perf_counter()
    for k in range(64):
        g, p, eps = synth.batch_density(k)
        tree = bc.Tree.refine(ctxs[p], g, eps=eps, max_level=16)
        groups[p].append((tree, torch.from_numpy(g(tree.nodes())).to(dev)))
    t_tree = time.perf_counter() - t0
    batches = {p: bc.Batch(ctxs[p], [t for t, _ in groups[p]]) for p in groups}
    head = PRECISIONS[args.precision]
    prec = {p: (head if p in bc.SPLIT_ORDERS else bc.FP64) for p in groups}
    outs = {p: [torch.empty_like(f) for _, f in groups[p]] for p in groups}
    adjs = {p: [torch.empty_like(f) for _, f in groups[p]] for p in groups}
    for p in groups:
        batches[p].autotune(prec[p])
    stream = torch.cuda.current_stream()

    def step():
        for p in groups:
            ins = [f for _, f in groups[p]]
            batches[p].run(ins, outs[p], precision=prec[p], stream=stream)
            batches[p].run(outs[p], adjs[p], precision=prec[p], adjoint=True, stream=stream)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    nodes = sum(t.nleaf * p * p for p in groups for t, _ in groups[p])
    leaves = [t.nleaf for p in groups for t, _ in groups[p]]
    line = {"metric": METRIC + " (batched)", "value": nodes / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": f"{DTYPES[head]} (p=8,12,16)" if head else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["batch64"][1], "trees": 64, "leaves_min": min(leaves),
                       "leaves_max": max(leaves), "leaves_total": sum(leaves), "leaf_nodes": nodes,
                       "tree_build_s": round(t_tree, 2),
                       "launch_shapes": {str(p): batches[p].shape(prec[p], 0) for p in groups},
                       "l2": "flushed (256 MB write) between timed steps"},
            "clocks": clocks.summary()}
    return line


def layer_line(args, dev, steps, check=True):
    """The glue layer potential (S[sigma] - D[tau] on the fictitious curve,
    Sec. 3.4) by the FMM at every leaf node of the star-shaped domain's
    truncated tree of the 200-Gaussian density: 256 Gauss-Legendre panels of
    16 nodes, nterms 30 (point sources converge like 0.55^P).  Device
    arrays, L2 flushed between timed applies; error against the oracle's
    direct sum at every node of sampled leaves."""
    import torch

    import oracle
    import paper_2501_17967_gb300 as bc
    from paper_2501_17967_gb300 import synth
    ctx = bc.Context(p=P, nterms=30, device=dev)
    gamma, gamma_b = synth.star_domain()
    tree = bc.Tree.refine_truncated(ctx, synth.config_density(3), gamma, gamma_b, eps=1e-11, max_level=18)
    xy, w, nrm, t = synth.fictitious_curve_sources(256, 16)
    sig, tau = synth.glue_densities(t)
    qh, mh = w * sig, (w * tau)[:, None] * nrm
    layer = bc.Layer(tree, xy)
    q, m = torch.from_numpy(qh).to(dev), torch.from_numpy(mh).to(dev)
    u = torch.empty(tree.nleaf * P * P, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def timed(prec):
        for _ in range(3):
            layer.apply(q, m, out=u, stream=stream, precision=prec)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            layer.apply(q, m, out=u, stream=stream, precision=prec)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps, u.cpu().numpy().reshape(-1, P * P)

    # split: the L2P at every leaf on the tensor cores; FP64: all of it in FP64
    ms, un = timed(bc.SPLIT_BF16)
    if not check:
        return {"value": tree.nleaf * P * P / (ms * 1e-3), "ms": ms, "profile_run": True}
    ms64, un64 = timed(bc.FP64)
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    geom = synth.leaf_geometry(lv, ix, iy)
    pick = synth.sample_leaves_per_level(lv, 1, seed=4)
    ref = oracle.layer(xy, qh, mh, oracle.leaf_nodes(geom, P)[pick].reshape(-1, 2)).reshape(len(pick), P * P)

    def err(x):
        return float(np.abs(x[pick] - ref).max() / np.abs(ref).max())
    return {"value": tree.nleaf * P * P / (ms * 1e-3), "unit": "leaf nodes/s (layer potential at every node)",
            "ms": ms, "workload": "star-shaped domain, truncated 200-Gaussian tree; 4096 curve nodes "
                                  "(256 Gauss-Legendre panels x 16); nterms 30",
            "precision": "split: L2P at every leaf on the BF16 tensor cores (exact digit products); near sums, "
                         "W list, far field in FP64",
            "nleaf": int(tree.nleaf), "lists": layer.info(), "rel_err_vs_oracle": err(un),
            "fp64": {"value": tree.nleaf * P * P / (ms64 * 1e-3), "ms": ms64, "rel_err_vs_oracle": err(un64),
                     "split_vs_fp64_all_nodes": float(np.abs(un - un64).max() / np.abs(un64).max())},
            "sample": f"every node of {len(pick)} leaves (1 per level)", "l2": "flushed between applies",
            "dtype": "f64 + bf16 digit products"}


def strip_line(args, dev, steps, peak_fp64, check=True):
    """The strip solve of Sec. 3.3 at the paper's size: 56 elements of 16 x 24
    nodes (N = 56 blocks of m = 384, one right-hand side), block LU of the
    tridiagonal part plus the Woodbury corner correction, random block
    diagonally dominant blocks; and the batched small-block case (608
    systems of N = 256, m = 17, one warp each).  Algorithmic FP64 work per
    system N m^2 (14 m / 3 + 6 R), R = r + 2m."""
    import torch

    import oracle
    import paper_2501_17967_gb300 as bc

    def make(nsys, N, m, r, seed):
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((nsys, N, m, m)) + 3.0 * m * np.eye(m)
        B, C = rng.standard_normal((nsys, N, m, m)), rng.standard_normal((nsys, N, m, m))
        b = rng.standard_normal((nsys, N, m, r))
        return A, B, C, b

    def timed(arrs, nsteps):
        stream = torch.cuda.current_stream()
        t = [torch.from_numpy(a).to(dev) for a in arrs]
        nsys, N, m, r = arrs[3].shape
        x = torch.empty_like(t[3])
        bufs = {"out": x, "work": bc.strip_workspace(nsys, N, m, r, t[3].device),
                "status": torch.zeros(nsys, dtype=torch.int32, device=t[3].device)}
        for _ in range(2):
            bc.strip_solve(*t, stream=stream, **bufs)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        for k in range(nsteps):
            ev[k][0].record(stream)
            bc.strip_solve(*t, stream=stream, **bufs)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in ev) / nsteps, x

    def work(nsys, N, m, r):
        return nsys * N * m * m * (14.0 * m / 3.0 + 6.0 * (r + 2 * m))

    big = make(1, 56, 384, 1, 5)
    ms, x = timed(big, max(3, steps // 2))
    ach = work(1, 56, 384, 1) / (ms * 1e-3) / 1e12
    line = {"value": 1.0 / (ms * 1e-3), "unit": "strip solves/s", "ms": ms,
            "workload": "the paper's strip size: N = 56 elements of 16 x 24 nodes (m = 384), one right-hand side; "
                        "block LU + Woodbury, blocked LU per element over the whole GPU",
            "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak_fp64, 3), "unit": "TFLOP/s",
                         "frac": round(ach / peak_fp64, 4), "traffic": None,
                         "work": "N m^2 (14 m / 3 + 6 R) FP64 flop per system, R = r + 2m"},
            "dtype": "f64"}
    if check:
        A, B, C, b = big
        xs = x.cpu().numpy()[0]
        N = 56
        res = max(float(np.abs(A[0, k] @ xs[k] + B[0, k] @ xs[(k + 1) % N] + C[0, k] @ xs[(k - 1) % N]
                               - b[0, k]).max()) for k in range(N))
        rows = max(float((np.abs(A[0, k]).sum(1) + np.abs(B[0, k]).sum(1) + np.abs(C[0, k]).sum(1)).max())
                   for k in range(N))
        line["backward_error"] = res / (rows * float(np.abs(xs).max()))
    small = make(608, 256, 17, 1, 6)
    ms2, x2 = timed(small, steps)
    ach2 = work(608, 256, 17, 1) / (ms2 * 1e-3) / 1e12
    line["batched_small"] = {"value": 608 / (ms2 * 1e-3), "unit": "strip systems/s", "ms": ms2,
                             "workload": "608 systems, N = 256, m = 17, r = 1, one warp each",
                             "roofline_frac": round(ach2 / peak_fp64, 4)}
    if check:
        A, B, C, b = small
        ref = oracle.strip_solve(A[0], B[0], C[0], b[0])
        line["batched_small"]["rel_err_vs_oracle"] = float(np.abs(x2[0].cpu().numpy() - ref).max()
                                                           / np.abs(ref).max())
    return line


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over the ranks of the process group (x itself without
    one): the whole-job time of replicas that ran side by side."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_units(units_per_rank: float, world: int) -> float:
    """Units processed by the whole job: every replica does the same work."""
    return float(units_per_rank) * world


class Runner:
    """Timed forward + adjoint steps of one tree."""

    def __init__(self, bc, torch, ctx, tree, f, gin, dev, world, dist):
        self.bc, self.torch, self.ctx, self.tree = bc, torch, ctx, tree
        self.f, self.gin = f, gin
        self.u = torch.empty_like(f)
        self.h = torch.empty_like(f)
        self.dev, self.world, self.dist = dev, world, dist
        self.flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2 (129 MB)
        self.stream = torch.cuda.current_stream()

    def step(self, prec):
        self.bc.apply(self.tree, self.f, out=self.u, precision=prec, stream=self.stream)
        self.bc.apply_adjoint(self.tree, self.gin, out=self.h, precision=prec, stream=self.stream)

    def timed(self, prec, steps, warmup, sampler=None, stages=True):
        torch, bc = self.torch, self.bc
        for _ in range(max(3, warmup)):
            self.step(prec)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if self.world > 1:
            self.dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
            time.sleep(0.3)
        # the timed steps run as in production: no stage events, no host reads
        for k in range(steps):
            self.flush.zero_()
            ev[k][0].record(self.stream)
            self.step(prec)
            ev[k][1].record(self.stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.stop()
        if self.world > 1:
            self.dist.barrier()
        bc._check(bc._load().bc_sync(self.ctx.handle, None))
        total = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)), self.dist if self.world > 1 else None,
                               self.dev)
        st = np.zeros((2, len(STAGES)))
        if stages:
            # per-stage times from a separate pass with the library's stage
            # events on (they separate the kernels of the launch chain and are
            # read back every step, so they stay out of the timed steps)
            self.ctx.debug(timing=True)
            for k in range(steps):
                self.flush.zero_()
                self.step(prec)
                st[0] += self.ctx.stage_times(adjoint=False)
                st[1] += self.ctx.stage_times(adjoint=True)
            self.ctx.debug(timing=False)
            bc._check(bc._load().bc_sync(self.ctx.handle, None))
        return total / steps, st / max(1, steps)


def rooflines(stage_ms, wk, peaks, traffic):
    """Per-stage achieved rate against the measured peak of its bound."""
    out = {}
    for i, name in enumerate(STAGES):
        ms = float(stage_ms[:, i].mean())
        amount, kind = wk[name]
        if ms <= 0 or amount == 0:
            continue
        if kind == "bytes":
            ach, pk, bound, unit = amount / (ms * 1e-3) / 1e9, peaks["hbm"], "hbm", "GB/s"
        elif kind == "tensor":
            ach, pk, bound, unit = amount / (ms * 1e-3) / 1e12, peaks["bf16"], "tensor", "TFLOP/s"
        else:
            ach, pk, bound, unit = amount / (ms * 1e-3) / 1e12, peaks["fp64"], "alu", "TFLOP/s"
        out[name] = {"ms": round(ms, 4), "kernel": STAGE_KERNELS[name], "bound": bound, "achieved": round(ach, 4),
                     "unit": unit, "peak": round(pk, 3), "frac": round(ach / pk, 4), "traffic": traffic.get(name)}
    return out


# FP64 pipe: 1.25 TFLOP/s nominal over 152 SMs at 2070 MHz is 4 flop per clock
# per SM (one 32-lane DFMA warp instruction per 16 clocks per SM)
FP64_FLOP_PER_CLK_SM = 4.0
PEAK_SOURCE = {"tensor": "MEASURED_PEAKS.json bf16_tflops (burst), of measured",
               "alu": "FP64 pipe derived from unit rate and clock: SMs x 4 flop/clk/SM x max SM clock "
                      "(1.259 TFLOP/s at 152 SMs, 2070 MHz; nominal 1.25), of derived; the FMA probe of this "
                      "run is fp64_probe_tflops",
               "hbm": "MEASURED_PEAKS.json hbm_gbs, of measured"}


def dominant(per_stage):
    d = max(per_stage, key=lambda k: per_stage[k]["ms"])
    r = dict(per_stage[d])
    r["stage"] = d
    r["peak_source"] = PEAK_SOURCE[r["bound"]]
    return r


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload in ("layer", "strip"):
        # one extra workload alone (profiler captures: --profile-run keeps the
        # oracle check out)
        import torch
        dev = torch.cuda.current_device()
        if args.workload == "layer":
            line = layer_line(args, dev, args.steps, check=not args.profile_run)
        else:
            line = strip_line(args, dev, args.steps, FP64_FLOP_PER_CLK_SM * 152 * 2070e6 / 1e12,
                              check=not args.profile_run)
        print(json.dumps(line))
        return
    import torch
    import torch.distributed as dist

    import paper_2501_17967_gb300 as bc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    head = PRECISIONS[args.precision]

    g = density(args.workload)
    workload_name = WORKLOADS[args.workload][1]
    ctx = bc.Context(p=P, nterms=args.nterms, device=dev)
    ctx.set_option("split_overlap", 1 if args.overlap else 0)
    P1 = ctx.nterms or 30
    t0 = time.perf_counter()
    tree = bc.Tree.refine(ctx, g, eps=1e-11, max_level=18)
    t_tree = time.perf_counter() - t0
    st = tree.stats()
    N = tree.nleaf * P * P
    lv, ix, iy = (np.asarray(a) for a in tree.leaves())
    fvals = g(tree.nodes()).reshape(-1, P, P)
    f = torch.from_numpy(fvals).to(dev)
    gen = torch.Generator(device=dev).manual_seed(1)
    gin = torch.randn(f.shape, generator=gen, device=dev, dtype=torch.float64)
    run = Runner(bc, torch, ctx, tree, f, gin, dev, world, dist if world > 1 else None)

    if args.profile_run:
        ms_step, _ = run.timed(head, args.steps, args.warmup, stages=False)
        if rank == 0:
            print(json.dumps({"profile_run": True, "workload": workload_name, "nleaf": int(tree.nleaf),
                              "ms_per_step": ms_step}))
        if world > 1:
            dist.destroy_process_group()
        return

    clocks = ClockSampler(dev)
    ms_step, stage_ms = run.timed(head, args.steps, args.warmup, sampler=clocks)
    value = replica_units(N, world) / (ms_step * 1e-3)

    # end to end through the public API with pinned host buffers
    fh = f.cpu().pin_memory()
    gh = gin.cpu().pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    hh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        bc.apply(tree, fh, out=uh, precision=head)
        bc.apply_adjoint(tree, gh, out=hh, precision=head)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bc.apply(tree, fh, out=uh, precision=head)
        bc.apply_adjoint(tree, gh, out=hh, precision=head)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * N * 8,
           "d2h_bytes_per_step": 2 * N * 8}

    # rooflines (per apply, averaged over forward and adjoint)
    peaks_file = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh_:
            peaks_file = json.load(fh_)
    except OSError:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = clocks.summary().get("sm_max_mhz") or 2070.0
    fp64_probe = bc.fp64_peak_tflops(dev)
    peaks = {"fp64": FP64_FLOP_PER_CLK_SM * sms * sm_max * 1e6 / 1e12, "bf16": peaks_file.get("bf16_tflops", 1900.0),
             "hbm": peaks_file.get("hbm_gbs", 6800.0)}
    nleaf_far = int((lv >= 2).sum())

    def arrangement_work(prec, overlap=None):
        overlap = args.overlap if overlap is None else overlap
        wk = stage_work(st, tree.nleaf, nleaf_far, P1, P * P, prec)
        if prec and not overlap:
            wk["tensor_v"] = (wk["tensor_v"][0] + wk["tensor_near"][0], "tensor")   # one group-V launch
            wk["tensor_near"] = (0.0, "tensor")
        elif prec:
            xw = 15 * 2.0 * P * P * 2 * P1 * st["n_x"]   # X-list tiles run on the internal stream
            wk["tensor_v"] = (wk["tensor_v"][0] - xw, "tensor")
            wk["tensor_near"] = (wk["tensor_near"][0] + xw, "tensor")
        return wk

    per_stage = rooflines(stage_ms, arrangement_work(head), peaks,
                          TRAFFIC.get((args.workload, P1, args.precision), {}))
    roofline = dominant(per_stage)
    roofline["fp64_probe_tflops"] = round(fp64_probe, 4)
    roofline["stages"] = per_stage

    pname = {v: k for k, v in PRECISIONS.items()}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
            "config": {"workload": workload_name, "precision": pname[head], "nleaf": int(tree.nleaf),
                       "leaf_nodes": int(N), "nlevels": st["nlevels"], "nterms": P1, "n_v": st["n_v"],
                       "n_near": st["n_near"], "tree_build_s": round(t_tree, 3),
                       "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
            "clocks": clocks.summary(), "e2e": e2e,
            "gpu_launches": 2 * launches_per_apply(head, args.overlap, st) * args.steps,
            "roofline": roofline}

    if not args.no_extras:
        # the same precision with the tensor launches in line (nothing beside
        # them): each kernel's rate alone
        if head and args.overlap:
            ctx.set_option("split_overlap", 0)
            ms_i, stage_i = run.timed(head, max(3, args.steps // 2), args.warmup)
            ctx.set_option("split_overlap", 1)
            ps_i = rooflines(stage_i, arrangement_work(head, overlap=False), peaks, {})
            line["inline"] = {"value": world * N / (ms_i * 1e-3), "ms_per_step": ms_i,
                              "note": "tensor launches in line on the apply's stream (option split_overlap 0): "
                                      "each stage alone; tensor_v = digits + the one group-V launch (near field, "
                                      "P2M, X list)",
                              "stages": {k: {kk: v[kk] for kk in ("ms", "achieved", "unit", "peak", "frac")}
                                         for k, v in ps_i.items()}}
        # the other precisions on the same tree, with their own rooflines
        for other in (p for p in (0, 1, 2) if p != head):
            ms_o, stage_o = run.timed(other, max(3, args.steps // 2), args.warmup)
            ps = rooflines(stage_o, arrangement_work(other), peaks,
                           TRAFFIC.get((args.workload, P1, pname[other]), {}))
            line[pname[other]] = {"value": world * N / (ms_o * 1e-3), "ms_per_step": ms_o, "dtype": DTYPES[other],
                                  "roofline": dominant(ps),
                                  "stage_ms": {k: v["ms"] for k, v in ps.items()}}
        # the 20-Gaussian workload in the headline precision
        if args.workload != "adaptive20":
            g2 = density("adaptive20")
            tree2 = bc.Tree.refine(ctx, g2, eps=1e-11, max_level=18)
            f2 = torch.from_numpy(g2(tree2.nodes()).reshape(-1, P, P)).to(dev)
            gin2 = torch.randn(f2.shape, generator=gen, device=dev, dtype=torch.float64)
            run2 = Runner(bc, torch, ctx, tree2, f2, gin2, dev, world, dist if world > 1 else None)
            ms2, _ = run2.timed(head, args.steps, args.warmup, stages=False)
            line["adaptive20"] = {"workload": WORKLOADS["adaptive20"][1], "nleaf": int(tree2.nleaf),
                                  "value": world * tree2.nleaf * P * P / (ms2 * 1e-3), "ms_per_step": ms2}
        # the 64-tree batch (p = 8, 12, 16) in the headline precision
        b64 = batch64_line(args, dev)
        line["batch64"] = {k: b64[k] for k in ("value", "unit", "ms_per_step", "dtype", "config", "clocks")}
        line["batch64"]["value"] *= world
        # the glue layer potential at every node (FMM, point sources)
        if rank == 0:
            line["layer"] = layer_line(args, dev, args.steps)
            line["strip"] = strip_line(args, dev, args.steps, peaks["fp64"])

    if rank == 0 and not args.no_extras:
        # error against the oracle per level, forward (every node of 2 leaves
        # per level) and adjoint (columns near and far on every level); the
        # forward sample's oracle time is the CPU baseline
        import oracle
        from paper_2501_17967_gb300 import synth
        leaves = (lv, ix, iy)
        u = bc.apply(tree, f, precision=head).cpu().numpy().reshape(-1, P * P)
        pick, ref, t_or = oracle_forward_sample(leaves, fvals.reshape(-1, P * P), per_level=2)
        scale = np.abs(ref).max()
        fwd_err = np.abs(u[pick] - ref).max(axis=1)
        S, cols, gs = adjoint_sample(leaves)
        hs = bc.apply_adjoint(tree, torch.from_numpy(gs).to(dev), precision=head).cpu().numpy()
        hs = hs.reshape(-1, P * P)
        geom = synth.leaf_geometry(lv, ix, iy)
        href = oracle.adjoint_columns(P, geom, gs, cols, target_leaves=S)
        hgot = np.array([hs[b, j] for b, j in cols])
        hscale = np.abs(href).max()
        line["per_level_error"] = {
            "forward": per_level(lv[pick], fwd_err, scale),
            "adjoint": per_level([lv[b] for b, _ in cols], np.abs(hgot - href), hscale),
            "forward_max": float(fwd_err.max() / scale),
            "adjoint_max": float(np.abs(hgot - href).max() / hscale),
            "sample": f"forward: every node of {len(pick)} leaves (2 per level); adjoint: {len(cols)} columns "
                      f"(3 nodes of 2 leaves per level), g random on {len(S)} leaves and zero elsewhere; "
                      f"metric max|x - x*| / max|x*| over the sample"}
        nodes = len(pick) * P * P
        line["cpu_baseline"] = {"value": nodes / t_or / 2.0, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{nodes} target nodes ({len(pick)} leaves, 2 per level) of the same tree "
                                          f"in {t_or:.1f}s; forward rate halved for fwd+adjoint"}
        bc._check(bc._load().bc_sync(ctx.handle, None))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
