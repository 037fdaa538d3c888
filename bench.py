"""Benchmark of the Monte Carlo DtN hot path on B300.

One step = the whole hot path on one synthetic workload: BVH build, rows,
tangent balls, walks (+ killing walks), histograms, assembly of Lambda and
the Steklov eigensolve.  Default workload: two icosphere-s4 spheres
(R = 0.5, centres 1.5 apart; 5124 vertices, 10240 triangles), exterior
estimator with killing walks (N0 = 64 W), FP32 walks, W = 1024 walks per
vertex, eps = 1e-3, k = 64 Steklov pairs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs its own replica (seed = rank), no
collective on the data path (weak scaling); the step time is the max over
ranks.  --impl reference times the CPU oracle (plain C, brute-force closest
point) on a bounded sample of the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walk steps/s and DtN rows/s at fixed walks/row; FP32-batched vs FP64-plain at equal error"
UNIT = "walk steps/s"
# FP32 operations (add, mul, min, max, compare) of one BVH node visit (two
# child boxes) and one point-triangle test on the interior-region path
OPS_PER_NODE = 36
OPS_PER_TRI = 90


def workload_config(args):
    return dict(workload="two_spheres_s4_exterior", mesh="two icospheres s4, R=0.5, centres 1.5 apart",
                nv=5124, nf=10240, walks_per_row=args.walks, eps=1e-3, domain="exterior",
                killing_walks=64 * args.walks, prec=f"fp{args.prec}", steklov_k=args.k, seed="rank",
                rows="all vertices", l2="flushed between steps (512 MiB write)")


def make_mesh():
    import meshgen
    return meshgen.two_spheres(4, 0.5, 1.5)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch
    import paper_2606_05581_b300 as mcs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    m = make_mesh()
    V_h = torch.from_numpy(m.V).pin_memory()
    F_h = torch.from_numpy(m.F).pin_memory()
    V_d, F_d = V_h.to(dev), F_h.to(dev)
    W = args.walks
    params = mcs.default_params(walks_per_row=W, prec=args.prec, domain=1, killing_walks=64 * W, seed=rank,
                                timing=1)
    ws = mcs.Workspace()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    has_eig = hasattr(mcs, "steklov_modes")

    eig_ws = mcs.Workspace()

    def step(V, F, keep=False):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh = mcs.Mesh(V, F)
        rows = mcs.vertex_rows(mesh)
        e1.record(stream)
        res = mcs.estimate_dtn(mesh, rows, params, workspace=ws)
        ev = None
        e2.record(stream)
        if has_eig:
            ev = mcs.steklov_modes(res["Lambda"], rows["area"], args.k, vectors=True, workspace=eig_ws)
        e3 = torch.cuda.Event(enable_timing=True)
        e3.record(stream)
        e3.synchronize()
        st = dict(res["stats"])
        st["build_ms"] = e0.elapsed_time(e1)
        st["eig_ms"] = e2.elapsed_time(e3)
        if ev is not None:
            st["eig"] = ev[2]
        out = (mesh, rows, res, ev)
        return out if keep else (st, ev)

    # warm-up
    for _ in range(args.warmup):
        step(V_d, F_d)
    torch.cuda.synchronize()

    def timed(k, e2e=False):
        times, stats = [], []
        h2d = d2h = 0
        for _ in range(k):
            flush.fill_(1)
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            if e2e:
                V = V_h.to(dev, non_blocking=True)
                F = F_h.to(dev, non_blocking=True)
                mesh, rows, res, ev = step(V, F, keep=True)
                L_h = torch.empty(res["Lambda"].shape, dtype=torch.float64, pin_memory=True)
                L_h.copy_(res["Lambda"], non_blocking=True)
                h2d = V_h.numel() * 8 + F_h.numel() * 4
                d2h = L_h.numel() * 8
                if ev is not None:
                    lam_h = ev[0].to("cpu", non_blocking=True)
                    d2h += lam_h.numel() * 8
                st = dict(res["stats"])
            else:
                st, _ = step(V_d, F_d)
            s1.record(stream)
            s1.synchronize()
            times.append(s0.elapsed_time(s1))
            stats.append(st)
        return times, stats, h2d, d2h

    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index) if rank == 0 else None
    if clk:
        clk.start()
    times, stats, _, _ = timed(args.steps)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop() if clk else None
    ms = float(np.sum(times)) / args.steps
    ms_max = allreduce_max(ms, world)
    steps_total = sum(s["steps"] + s["killing_steps"] for s in stats) / args.steps  # per replica per step
    R = m.nv
    value = steps_total * world / (ms_max / 1e3)
    # end to end: host buffers in, Lambda (+ eigenvalues) out
    e2e_times, _, h2d, d2h = timed(max(1, min(args.steps, 3)), e2e=True)
    e2e_ms = allreduce_max(float(np.mean(e2e_times)), world)
    if rank != 0:
        return None
    # work counts of the same walks (identical seed -> identical walks), untimed
    p2 = mcs.default_params(walks_per_row=W, prec=args.prec, domain=1, killing_walks=64 * W, seed=rank,
                            timing=1, count_work=1)
    mesh = mcs.Mesh(V_d, F_d)
    rows = mcs.vertex_rows(mesh)
    cres = mcs.estimate_dtn(mesh, rows, p2, workspace=ws)
    cst = cres["stats"]
    walk_ms = float(np.mean([s["phase_ms"][1] for s in stats]))
    ops = OPS_PER_NODE * cst["nodes_visited"] + OPS_PER_TRI * cst["tris_tested"]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = 148 * 128 * sm_max * 1e6 / 1e12  # FP32 lanes x clock, T op/s
    achieved = ops / (walk_ms / 1e3) / 1e12
    phase = np.mean([s["phase_ms"] for s in stats], axis=0).tolist()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"f{args.prec}", "data": "synthetic",
        "config": dict(workload_config(args), parallelism=f"replicas{world}"),
        "rows_per_s": R * world / (ms_max / 1e3),
        "walks_per_s": (R * W + 64 * W) * world / (ms_max / 1e3),
        "closest_point_queries_per_s": value,
        "walk_steps_per_step": steps_total,
        "phase_ms": {"bvh_build_and_vertex_rows": float(np.mean([s["build_ms"] for s in stats])),
                     "rows_and_tangent_balls": phase[0], "walks": phase[1], "histogram": phase[2],
                     "assembly": phase[3], "steklov_modes": float(np.mean([s["eig_ms"] for s in stats]))},
        "steklov": stats[-1].get("eig"),
        "e2e": {"value": steps_total * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
        "gpu_launches": GPU_LAUNCHES_PER_STEP * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Top/s",
                     "frac": achieved / alu_peak, "traffic": None, "kernel": "k_walks (FP32, exterior)",
                     "ops_per_node": OPS_PER_NODE, "ops_per_tri": OPS_PER_TRI,
                     "nodes_per_query": cst["nodes_visited"] / max(1, cst["steps"] + cst["killing_steps"]),
                     "tris_per_query": cst["tris_tested"] / max(1, cst["steps"] + cst["killing_steps"]),
                     "peak_note": "148 SMs x 128 FP32 lanes x max SM clock (derived)"},
        "clocks": clocks,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, samples=1)[0]
    return line


# own kernels launched per step (BVH build 10, vertex rows 1, exterior
# estimate with automatic origin and killing 14); CUB sort kernels not counted
GPU_LAUNCHES_PER_STEP = 25


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- the oracle as baseline
def cpu_baseline(args, samples=1):
    """Oracle (plain C, brute force) on a bounded sample of the workload: a set of
    rows of the same exterior estimate, W walks each, in the same precision."""
    from oracle import oracle as O
    m = make_mesh()
    rows = O.vertex_rows(m.V, m.F)
    nthr = O.num_threads()
    origin = np.zeros(3)  # the inversion centre the estimate uses (sphere A's tangent-ball centre)
    t0 = time.time()
    origin = O.interior_origin(m.V, m.F, rows)
    t_origin = time.time() - t0
    nrows = max(2, nthr)
    rng = np.random.default_rng(0)
    out = []
    for s in range(samples):
        rl = np.sort(rng.choice(m.nv, nrows, replace=False)).astype(np.int32)
        t0 = time.time()
        est = O.estimate(m.V, m.F, rows, args.walks, 1e-3, exterior=True, origin=origin, seed=0, prec=args.prec,
                         row_list=rl)
        dt = time.time() - t0
        steps = int(est["steps"].sum())
        out.append({"value": steps / dt, "unit": UNIT, "cores": nthr, "kind": "oracle",
                    "sample": f"{nrows} rows x {args.walks} walks of the same exterior estimate "
                              f"(fp{args.prec}, brute-force closest point over {m.nf} triangles); "
                              f"{steps} walk steps in {dt:.1f} s (+{t_origin:.1f} s interior pass for the origin)",
                    "rows_per_s": nrows / dt})
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    res = cpu_baseline(args, samples=args.steps)
    vals = [r["value"] for r in res]
    value = float(np.mean(vals))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"f{args.prec}", "data": "synthetic",
            "config": dict(workload_config(args), parallelism="host cores"),
            "cpu_baseline": dict(res[0], value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--walks", type=int, default=1024)
    ap.add_argument("--prec", type=int, default=32, choices=[32, 64])
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world) if args.impl == "ours" else run_reference(args, rank, world)
    if line is not None:
        print(json.dumps(line))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
