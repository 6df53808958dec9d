"""Throughput of the GB300 machine code: leaf nodes per second for one forward plus
one adjoint volume-potential apply on the adaptive 20-Gaussian workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split]
                    [--impl ours|reference]

Workload: root [-1,1]^2, p = 16, density = 20 Gaussians (centres U[-0.5,0.5]^2,
widths log-uniform in [1e-3, 1e-1], amplitudes N(0,1), seed 1), quadtree
refined by the library (Alg. 2 resolution criterion, eps = 1e-11) and 2:1
balanced.  A step is one forward apply u = A f and one adjoint apply
h = A^T g of the whole tree; value = leaf nodes / (time of a step).
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

WORKLOAD = "adaptive 20-Gaussian quadtree (widths 1e-3..1e-1), p=16, eps=1e-11"
METRIC = "leaf nodes/sec (p=16, <=1e-10 rel err) fwd+adjoint"
UNIT = "leaf nodes/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "split"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def density():
    from paper_2501_17967_gb300 import synth
    return synth.config_density(2)


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


# ---------------------------------------------------------------- oracle arm
def oracle_rate(tree_leaves, fvals, seconds, seed=11):
    """Oracle forward throughput (target nodes/s) on sampled leaves, bounded in time.
    The oracle's transposed operator costs the same per entry, so a fwd+adjoint
    step is twice the forward cost."""
    import oracle
    from paper_2501_17967_gb300 import synth
    lv, ix, iy = tree_leaves
    p = 16
    geom = synth.leaf_geometry(lv, ix, iy)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(lv))
    done, t_used, vals = 0, 0.0, {}
    k = 1
    while t_used < seconds and done < len(order):
        ids = order[done:done + k]
        t0 = time.perf_counter()
        u = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=ids)
        t_used += time.perf_counter() - t0
        for i, b in enumerate(ids):
            vals[int(b)] = u[i]
        done += len(ids)
        k = min(2 * k, 64)
    nodes = done * p * p
    return nodes / t_used / 2.0, nodes, t_used, vals


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import paper_2501_17967_gb300 as bc
    import oracle
    from paper_2501_17967_gb300 import synth
    g = density()
    hctx = bc.Context(p=16, device=-1, cache_dir=None, build_tables=False)
    tree = bc.Tree.refine(hctx, g, eps=1e-11, max_level=18)
    leaves = tree.leaves()
    geom = synth.leaf_geometry(*leaves)
    fvals = g(oracle.leaf_nodes(geom, 16)).reshape(-1, 16, 16)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rate(leaves, fvals, per_step / 4)
    rates, nodes_tot, t_tot = [], 0, 0.0
    for s in range(args.steps):
        r, n, t, _ = oracle_rate(leaves, fvals, per_step, seed=100 + s)
        rates.append(r)
        nodes_tot += n
        t_tot += t
    value = nodes_tot / t_tot / 2.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nleaf": int(tree.nleaf), "leaf_nodes": int(tree.nleaf) * 256,
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{nodes_tot} target nodes of randomly sampled leaves over {args.steps} steps "
                                       f"(~{per_step:.0f}s each), forward oracle rate halved for fwd+adjoint"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_2501_17967_gb300 as bc
    import oracle
    from paper_2501_17967_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    precision = {"fp64": bc.FP64, "split": bc.SPLIT_BF16}.get(args.precision)
    if precision is None:
        precision = bc.SPLIT_BF16 if getattr(bc, "SPLIT_AVAILABLE", False) else bc.FP64
    pname = "split-bf16" if precision == bc.SPLIT_BF16 else "fp64"

    g = density()
    ctx = bc.Context(p=16, device=dev)
    t0 = time.perf_counter()
    tree = bc.Tree.refine(ctx, g, eps=1e-11, max_level=18)
    t_tree = time.perf_counter() - t0
    st = tree.stats()
    N = tree.nleaf * 256
    nodes = tree.nodes()
    fvals = g(nodes).reshape(-1, 16, 16)
    f = torch.from_numpy(fvals).to(dev)
    gen = torch.Generator(device=dev).manual_seed(1)
    gin = torch.randn(f.shape, generator=gen, device=dev, dtype=torch.float64)
    u = torch.empty_like(f)
    h = torch.empty_like(f)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step():
        bc.apply(tree, f, out=u, precision=precision, stream=stream)
        bc.apply_adjoint(tree, gin, out=h, precision=precision, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ctx.debug(timing=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stages = np.zeros((2, 4))
    clocks = ClockSampler(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        stages[0] += ctx.stage_times(adjoint=False)
        stages[1] += ctx.stage_times(adjoint=True)
    torch.cuda.synchronize()
    clocks.stop()
    if world > 1:
        dist.barrier()
    ctx.debug(timing=False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    t_max = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms = float(t_max.item())
    ms_per_step = total_ms / args.steps
    value = world * N / (ms_per_step * 1e-3)

    # end to end through the public API with pinned host buffers
    fh = f.cpu().pin_memory()
    gh = gin.cpu().pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    hh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        bc.apply(tree, fh, out=uh, precision=precision)
        bc.apply_adjoint(tree, gh, out=hh, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bc.apply(tree, fh, out=uh, precision=precision)
        bc.apply_adjoint(tree, gh, out=hh, precision=precision)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": 2 * N * 8}

    # roofline of the dominant stage (leaf output: L2P + W list + near-field tables)
    stage_ms = stages / args.steps          # [dir][stage], per apply
    dom_dir, dom_stage = np.unravel_index(np.argmax(stage_ms), stage_ms.shape)
    NP, P1 = 256, ctx.nterms or 40
    n_l2p_leaves = tree.nleaf   # upper bound: leaves at level >= 2
    flops = {3: 2.0 * NP * NP * st["n_near"] + 8.0 * P1 * NP * (n_l2p_leaves + st["n_w"]),
             2: 8.0 * P1 * P1 * (st["n_v"] + st["n_nonleaf"]) + 8.0 * P1 * NP * st["n_x"],
             1: 8.0 * P1 * P1 * st["n_nonleaf"],
             0: 4.0 * P1 * NP * tree.nleaf}[int(dom_stage)]
    peak = bc.fp64_peak_tflops(dev)
    achieved = flops / (stage_ms[dom_dir, dom_stage] * 1e-3) / 1e12
    names = ["leaf_to_expansion", "upward", "downward", "leaf_output"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"{names[dom_stage]} ({'adjoint' if dom_dir else 'forward'})",
                "peak_source": "measured FP64 FMA throughput (bc_debug_fp64_peak)",
                "stage_ms": {("adj_" if d else "fwd_") + names[s]: round(float(stage_ms[d, s]), 4)
                             for d in range(2) for s in range(4)}}

    launches_per_apply = 2 + max(0, st["nlevels"] - 3) + max(0, st["nlevels"] - 2)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if precision == bc.FP64 else "bf16x-split+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": pname, "nleaf": int(tree.nleaf), "leaf_nodes": int(N),
                       "nlevels": st["nlevels"], "nterms": P1, "tree_build_s": round(t_tree, 3),
                       "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
            "clocks": clocks.summary(), "e2e": e2e, "gpu_launches": 2 * launches_per_apply * args.steps,
            "roofline": roofline}

    if rank == 0 and not args.no_cpu_baseline:
        rate, nn, tt, vals = oracle_rate(tree.leaves(), fvals, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{nn} target nodes ({nn // 256} random leaves) of the same tree in "
                                          f"{tt:.1f}s; forward rate halved for fwd+adjoint"}
        uu = u.cpu().numpy().reshape(-1, 256)
        got = np.stack([uu[b] for b in vals])
        ref = np.stack([vals[b] for b in vals])
        line["rel_err_vs_oracle_sample"] = float(np.abs(got - ref).max() / np.abs(ref).max())
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
