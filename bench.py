"""Benchmark of the Monte Carlo DtN hot path on B300.

One step = the whole hot path on one synthetic workload.  Workloads
(--workload):

  two_spheres_s4_exterior  two icosphere-s4 spheres (R = 0.5,
      centres 1.5 apart; 5124 vertices, 10240 triangles), exterior estimator
      with killing walks (N0 = 64 W), FP32 walks, W = 1024 per vertex,
      eps = 1e-3, k = 64 Steklov pairs.  Step: BVH build, vertex rows,
      tangent balls, walks, histograms, assembly, Steklov eigensolve.
  wild_2m   a ~2.0M-face union of 300 ellipsoids / tori (noise, flipped
      faces, slivers), 10,000 farthest-point sample rows, W = 4096, FP32,
      interior, k = 64.  Same step with sample rows instead of vertex rows.
  batch (default)  --meshes (512) unions with 5k-200k faces each (mesh i:
      seed 1000 + i, exterior when i is odd), 1024 sample rows x 512 walks
      each, FP32, killing walks 64 W on exterior meshes, autotuned launch;
      step = one replay of the graph-captured batched estimate (all meshes'
      setup, ONE persistent walk launch, histograms, assembly).  BVH builds
      and sample rows are preprocessing, timed apart; the end-to-end figure
      includes them with the host copies in and every Lambda out.
  precision FP32 vs FP64 walks on the two-sphere mesh at W = 1024, 4096,
      16384 (4 seeds each), k = 128, against an FP64 W = 65536 reference;
      per-eigenvalue errors, their standard errors and walks/s.
  variance  the quadratic form of f = z on the unit icosphere s3 by the
      importance-sampled tangent ball, the uniformly sampled ball (weighted
      walks) and the naive finite-difference estimator (Alg. 1), over seeds at
      W = 8, 32, 128: means and variances.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

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


WORKLOADS = ("two_spheres_s4_exterior", "wild_2m", "batch", "precision", "variance")


def workload_config(args):
    if args.workload == "wild_2m":
        return dict(workload="wild_2m", mesh="union of 300 ellipsoids/tori, ~2.0M faces, seed 0 (noise 1e-3, "
                    "5% flipped, 10% slivers)", rows="10000 farthest-point samples (face centroids, from face 0)",
                    walks_per_row=args.walks or 4096, eps=1e-3, domain="interior", prec=f"fp{args.prec}",
                    steklov_k=args.k, seed="rank + 1", l2="inputs larger than L2 (BVH + triangles ~170 MB) and "
                    "flushed between steps (512 MiB write)")
    if args.workload == "batch":
        return dict(workload="batch", meshes=args.meshes, mesh="unions of U{1..50} primitives, faces "
                    "log-uniform [5k, 200k], seed 1000 + i", rows="1024 farthest-point samples per mesh",
                    walks_per_row=args.walks or 512, eps=1e-3, domain="exterior for odd i, interior for even i",
                    killing_walks=64 * (args.walks or 512), prec=f"fp{args.prec}", seed="i",
                    launch="one graph replay: per-mesh setup, one persistent walk launch, per-mesh histogram and "
                           "assembly; autotuned launch shape and queue order",
                    l2="inputs larger than L2 (all meshes' BVHs) and flushed between steps (512 MiB write)")
    return dict(workload="two_spheres_s4_exterior", mesh="two icospheres s4, R=0.5, centres 1.5 apart",
                nv=5124, nf=10240, walks_per_row=args.walks or 1024, eps=1e-3, domain="exterior",
                killing_walks=64 * (args.walks or 1024), prec=f"fp{args.prec}", steklov_k=args.k, seed="rank",
                rows="all vertices", l2="flushed between steps (512 MiB write)")


def make_mesh(args):
    import meshgen
    if args.workload == "wild_2m":
        return meshgen.wild_union(300, 2_000_000, seed=0)
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
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


# Algorithmic work of one closest-point query (one walk step), per unit of
# the traversal (the scope table's measurement row): each visited node reads
# its children's boxes, 32 B each (binary node: 2, four-wide node: 4), and
# costs ~12 FP32 operations per box; each tested triangle reads 36 B (three
# FP32 vertices) and costs ~70 operations; the step itself (Philox block,
# direction, update) ~25 operations.
BOX_BYTES, TRI_BYTES = 32, 36
OPS_PER_BOX, OPS_PER_TRI, OPS_PER_STEP = 12, 70, 25


def _walk_roofline(cst, walk_ms, kernel, peaks, width=2):
    """Roofline of the walk kernel: queries (walk steps) of the timed launch x
    the algorithmic bytes and operations per query (node and triangle counts
    per query from an untimed counting run of the same walks) over the
    kernel's event-timed duration, against the L2 read bandwidth and the FP32
    instruction rate measured on this GPU by the library's probes.  The
    bound reported is the ceiling the kernel is closer to."""
    q = max(1, cst["steps"] + cst["killing_steps"])
    npq = cst["nodes_visited"] / q
    tpq = cst["tris_tested"] / q
    bytes_q = width * BOX_BYTES * npq + TRI_BYTES * tpq
    ops_q = width * OPS_PER_BOX * npq + OPS_PER_TRI * tpq + OPS_PER_STEP
    secs = walk_ms / 1e3
    gbs = q * bytes_q / secs / 1e9
    tops = q * ops_q / secs / 1e12
    l2, alu = peaks["l2_read_gbs"], peaks["fp32_fma_tinst_s"]
    l2_frac, alu_frac = gbs / l2, tops / alu
    if l2_frac >= alu_frac:
        head = {"bound": "l2", "achieved": gbs, "peak": l2, "unit": "GB/s", "frac": l2_frac}
    else:
        head = {"bound": "alu", "achieved": tops, "peak": alu, "unit": "Top/s", "frac": alu_frac}
    return dict(head, traffic=None, kernel=kernel, l2_frac=l2_frac, alu_frac=alu_frac,
                l2_achieved_gbs=gbs, l2_peak_gbs=l2, alu_achieved_tops=tops, alu_peak_tops=alu,
                queries=q, kernel_ms=walk_ms, nodes_per_query=npq, tris_per_query=tpq,
                bytes_per_query=bytes_q, ops_per_query=ops_q, node_width=width,
                per_unit={"box_bytes": BOX_BYTES, "tri_bytes": TRI_BYTES, "ops_per_box": OPS_PER_BOX,
                          "ops_per_tri": OPS_PER_TRI, "ops_per_step": OPS_PER_STEP},
                peak_note="of measured: L2 read bandwidth and FP32 FMA instruction rate from the library's "
                          "probes on this GPU before the timed region",
                traffic_note="DRAM bytes of this kernel come from ncu captures summarised with the profiles; "
                             "not measured in this run")


def _downstream(mcs, out, dev, reps=5):
    """Untimed by the headline: Steklov heat of a 16-channel field and heat
    kernel signatures at 16 log-spaced times from the step's eigenpairs, each
    timed with CUDA events (mean of `reps` after one warm-up).  Algorithmic
    bytes: psi read (n k 8) plus the outputs written (heat: psi twice, u0 in)."""
    import torch
    _, rows, _, ev = out
    evals, X = ev[0], ev[1]
    n, k = int(X.shape[0]), int(X.shape[1])
    times = torch.logspace(-3, 1, 16, dtype=torch.float64, device=dev)
    c = 16
    u0 = torch.randn(n, c, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    ws = mcs.Workspace()

    def clock(fn):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    heat_ms = clock(lambda: mcs.steklov_heat(evals, X, rows["area"], u0, times, workspace=ws))
    hks_ms = clock(lambda: mcs.hks(evals, X, times))
    nt = int(times.numel())
    heat_bytes = 2 * n * k * 8 + n * c * 8 + nt * n * c * 8
    hks_bytes = n * k * 8 + nt * n * 8
    peak = _peaks().get("hbm_gbs")
    gbs = lambda b, ms: b / (ms / 1e3) / 1e9
    # FP64 multiply-adds: projection n k c, synthesis nt n k c; HKS nt n k
    heat_tflops = 2.0 * (n * k * c + nt * n * k * c) / (heat_ms / 1e3) / 1e12
    hks_tflops = 2.0 * nt * n * k / (hks_ms / 1e3) / 1e12
    return {"n": n, "k": k, "channels": c, "times": nt, "heat_ms": heat_ms, "hks_ms": hks_ms,
            "heat_gbs": gbs(heat_bytes, heat_ms), "hks_gbs": gbs(hks_bytes, hks_ms), "hbm_peak_gbs": peak,
            "heat_fp64_tflops": heat_tflops, "hks_fp64_tflops": hks_tflops, "fp64_nominal_tflops": 1.25,
            "note": "psi (n x k FP64) fits in L2 at this size, so the passes are bound by FP64 arithmetic "
                    "(B300's nominal FP64 rate) rather than HBM"}


def _galerkin(mcs, V, F, params, ws, kill, k):
    """Untimed by the headline: the Galerkin estimator on the same walks
    (exit barycentrics recorded), K = k + 32 cotangent-Laplacian modes as the
    basis, and the point-based basis (Sec. 4.4) on the same walks; each phase
    timed with CUDA events after one warm-up."""
    import torch
    mesh = mcs.Mesh(V, F)
    vrows = mcs.vertex_rows(mesh)
    res = mcs.estimate_dtn(mesh, vrows, params, assemble=False, record_exits=True, record_bary=True, workspace=ws)
    K = k + 32
    gws = mcs.Workspace()

    def clock(fn, reps=3):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            r = fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps, r

    basis_ms, (_, Phi, est) = clock(lambda: mcs.steklov_modes(mcs.cotan_laplacian(mesh), vrows["area"], K), 1)
    gal_ms, S = clock(lambda: mcs.galerkin_dtn(mesh, vrows, res, Phi, exterior=True, killing_walks=kill, workspace=gws))
    modes_ms, (ev, _, _) = clock(lambda: mcs.galerkin_modes(S, k))
    walks = int(res["exit_tri"].numel())
    # the point-based basis on the same walks: the vertex rows as the points,
    # sigma = the mean point spacing sqrt(area / n), tau_n and k the paper's
    sigma = float(torch.sqrt(vrows["area"].sum() / vrows["area"].numel()))
    pws = mcs.Workspace()
    pb_ms, (PhiP, _, pst) = clock(lambda: mcs.point_basis(vrows, K, workspace=pws), 1)
    pl_ms, Lp = clock(lambda: mcs.point_galerkin_lambda(mesh, vrows, res, exterior=True, killing_walks=kill,
                                                        sigma=sigma, workspace=pws))
    pp_ms, SP = clock(lambda: mcs.galerkin_project(Lp, PhiP, workspace=gws))
    pev, _, _ = mcs.galerkin_modes(SP, k)
    point = {"points": int(vrows["area"].numel()), "sigma": sigma, "tau_n": mcs.KNN_TAU, "knn": mcs.KNN_K,
             "basis_ms": pb_ms, "lambda_ms": pl_ms, "project_ms": pp_ms, "basis_status": pst["status"],
             "walks_per_s": walks / (pl_ms / 1e3), "evals_head": [round(float(x), 4) for x in pev[:8].cpu()]}
    return {"K": K, "basis_ms": basis_ms, "galerkin_dtn_ms": gal_ms, "modes_ms": modes_ms,
            "walks": walks, "walks_per_s": walks / (gal_ms / 1e3), "basis_status": est["status"],
            "evals_head": [round(float(x), 4) for x in ev[:8].cpu()], "point_basis": point}


def run_variance(args, rank, world):
    """Variance study (Sec. 5, Fig. variance_comparison): the quadratic form of
    f = z on the unit icosphere s3 (1280 face sample rows) by the importance-
    sampled tangent ball (the estimator), the uniformly sampled tangent ball
    (weighted walks) and the naive finite-difference estimator (Alg. 1,
    h = 0.02), each over 8 x --seeds seeds at several walk counts; all on the GPU
    (walks, exit barycentrics, Galerkin assembly).  value = the naive
    estimator's variance over the importance sampler's at the largest N."""
    import torch
    import meshgen
    import paper_2606_05581_b300 as mcs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.sample_rows(mesh, m.nf, orient=False)
    f = torch.from_numpy(np.ascontiguousarray(m.V[:, 2])).cuda()
    Phi = torch.zeros((m.nv, 16), dtype=torch.float64, device=dev)
    Phi[:, 0] = f
    Ws, seeds = (8, 32, 128), range(8 * args.seeds)
    names = {0: "importance_ball", 1: "uniform_ball", 2: "naive_fd"}
    table = {}
    t0 = time.time()
    for mode in (0, 1, 2):
        for W in Ws:
            vals = []
            for sd in seeds:
                p = mcs.default_params(walks_per_row=W, prec=32, seed=sd, eps=1e-4 if mode == 2 else 1e-3)
                p.start_mode = mode
                if mode == 2:
                    p.inset = 0.02
                res = mcs.estimate_dtn(mesh, rows, p, assemble=False, record_exits=True, record_bary=True)
                _, Lb = mcs.galerkin_dtn(mesh, rows, res, Phi, want_lambda=True, start_mode=mode)
                vals.append(float(f @ Lb @ f))
            table.setdefault(names[mode], []).append(
                {"walks_per_row": W, "samples": m.nf * W, "mean": float(np.mean(vals)),
                 "variance": float(np.var(vals, ddof=1)), "variance_x_N": float(np.var(vals, ddof=1)) * m.nf * W})
    wall = time.time() - t0
    ratio = table["naive_fd"][-1]["variance"] / table["importance_ball"][-1]["variance"]
    return {"metric": "variance ratio naive / importance-sampled tangent ball, quadratic form of z on the unit sphere",
            "value": ratio, "unit": "x", "n_gpus": 1, "steps": len(Ws) * len(seeds) * 3, "warmup": 0,
            "ms_per_step": wall * 1e3 / (len(Ws) * len(seeds) * 3), "higher_is_better": True, "scaling": "none",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "variance", "mesh": "unit icosphere s3", "rows": "1280 face sample rows",
                       "seeds": len(seeds), "inset_h": 0.02, "exact_l1_form": 4 * math.pi / 3},
            "table": table}


def run_ours(args, rank, world):
    """One mesh per step: the default two-sphere exterior workload or wild_2m."""
    import torch
    import paper_2606_05581_b300 as mcs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wild = args.workload == "wild_2m"
    m = make_mesh(args)
    V_h = torch.from_numpy(m.V).pin_memory()
    F_h = torch.from_numpy(m.F).pin_memory()
    V_d, F_d = V_h.to(dev), F_h.to(dev)
    W = args.walks or (4096 if wild else 1024)
    n_rows = 10_000 if wild else m.nv
    kill = 0 if wild else 64 * W
    pkw = dict(walks_per_row=W, prec=args.prec, domain=0 if wild else 1, killing_walks=kill,
               seed=replica_seed(rank, 1 if wild else 0), bvh_layout=args.bvh_layout)
    params = mcs.default_params(timing=1, **pkw)
    ws = mcs.Workspace()
    rows_ws = mcs.Workspace()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    eig_ws = mcs.Workspace()

    def make_rows(mesh):
        if wild:
            return mcs.sample_rows(mesh, n_rows, orient=True, workspace=rows_ws)
        return mcs.vertex_rows(mesh)

    def step(V, F, keep=False, on_lambda=None):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh = mcs.Mesh(V, F)
        if args.bvh_layout == 4:
            mesh.build_wide()
        rows = make_rows(mesh)
        e1.record(stream)
        res = mcs.estimate_dtn(mesh, rows, params, workspace=ws)
        e2.record(stream)
        if on_lambda is not None:
            on_lambda(res["Lambda"], e2)
        ev = mcs.steklov_modes(res["Lambda"], rows["area"], args.k, vectors=True, workspace=eig_ws)
        e3.record(stream)
        e3.synchronize()
        st = dict(res["stats"])
        st["build_ms"] = e0.elapsed_time(e1)
        st["eig_ms"] = e2.elapsed_time(e3)
        st["eig"] = ev[2]
        out = (mesh, rows, res, ev)
        return out if keep else (st, ev)

    for _ in range(args.warmup):
        step(V_d, F_d)
    torch.cuda.synchronize()
    peaks = mcs.probe_peaks()  # the roofline's ceilings, measured before the timed region

    pinned = {}  # the host buffer Lambda is read into: allocated once, outside the timed region
    side = torch.cuda.Stream(device=dev)  # Lambda's device-to-host copy overlaps the eigensolve

    def timed(k, e2e=False):
        times, stats = [], []
        h2d = d2h = 0
        if e2e and "L" not in pinned:
            pinned["L"] = torch.empty((n_rows, n_rows), dtype=torch.float64, pin_memory=True)
        for _ in range(k):
            flush.fill_(1)
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            if e2e:
                V = V_h.to(dev, non_blocking=True)
                F = F_h.to(dev, non_blocking=True)
                L_h = pinned["L"]
                done = torch.cuda.Event()

                def copy_out(L, ready):
                    side.wait_event(ready)
                    with torch.cuda.stream(side):
                        L_h.copy_(L, non_blocking=True)
                        done.record(side)

                mesh, rows, res, ev = step(V, F, keep=True, on_lambda=copy_out)
                stream.wait_event(done)
                lam_h = ev[0].to("cpu", non_blocking=True)
                h2d = V_h.numel() * 8 + F_h.numel() * 4
                d2h = L_h.numel() * 8 + lam_h.numel() * 8
                st = dict(res["stats"])
            else:
                torch.cuda.nvtx.range_push("timed_step")
                st, _ = step(V_d, F_d)
                torch.cuda.nvtx.range_pop()
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
    l0 = mcs.launch_count()
    times, stats, _, _ = timed(args.steps)
    torch.cuda.synchronize()
    launches = mcs.launch_count() - l0
    barrier(world)
    clocks = clk.stop() if clk else None
    ms = float(np.sum(times)) / args.steps
    ms_max = allreduce_max(ms, world)
    steps_total = sum(s["steps"] + s["killing_steps"] for s in stats) / args.steps  # per replica per step
    value = steps_total * world / (ms_max / 1e3)
    # end to end: host buffers in, Lambda and the eigenvalues out
    e2e_times, _, h2d, d2h = timed(max(1, min(args.steps, 3)), e2e=True)
    e2e_ms = allreduce_max(float(np.mean(e2e_times)), world)
    if rank != 0:
        return None
    # work counts of the same walks (identical seed -> identical walks), untimed
    mesh = mcs.Mesh(V_d, F_d)
    if args.bvh_layout == 4:
        mesh.build_wide()
    rows = make_rows(mesh)
    cst = mcs.estimate_dtn(mesh, rows, mcs.default_params(timing=1, count_work=1, **pkw), workspace=ws)["stats"]
    walk_ms = float(np.mean([s["phase_ms"][1] for s in stats]))
    phase = np.mean([s["phase_ms"] for s in stats], axis=0).tolist()
    walks = n_rows * W + kill
    downstream = _downstream(mcs, step(V_d, F_d, keep=True), dev)
    if not wild:
        downstream["galerkin"] = _galerkin(mcs, V_d, F_d, params, ws, kill, args.k)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"f{args.prec}", "data": "synthetic",
        "config": dict(workload_config(args), parallelism=f"replicas{world}"),
        "rows_per_s": n_rows * world / (ms_max / 1e3),
        "walks_per_s": walks * world / (ms_max / 1e3),
        "closest_point_queries_per_s": value,
        "walk_steps_per_step": steps_total,
        "capped_walks_per_step": float(np.mean([s["capped"] + s["killing_capped"] for s in stats])),
        "discarded_rows": stats[-1]["discarded_rows"],
        "phase_ms": {"bvh_build_and_rows": float(np.mean([s["build_ms"] for s in stats])),
                     "row_setup_and_tangent_balls": phase[0], "walks": phase[1], "histogram": phase[2],
                     "assembly": phase[3], "steklov_modes": float(np.mean([s["eig_ms"] for s in stats]))},
        "steklov": stats[-1].get("eig"),
        "e2e": {"value": steps_total * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
        "gpu_launches": int(launches),
        "gpu_launches_note": "library kernels counted by the library (mcs_launch_count); CUB sort kernels excluded",
        "roofline": _walk_roofline(cst, walk_ms, f"k_walks (FP{args.prec}, {'interior' if wild else 'exterior'})",
                                   peaks, 4 if args.bvh_layout == 4 else 2),
        "peaks_measured": peaks,
        "clocks": clocks,
        "downstream": downstream,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, samples=1)[0]
    return line


def _batch_setup(args, dev, rank):
    """Meshes, BVHs and sample rows of the batch workload (preprocessing)."""
    import torch
    import meshgen
    import paper_2606_05581_b300 as mcs
    t0 = time.time()
    hosts = meshgen.batch_meshes(args.meshes, 1000)
    t_gen = time.time() - t0
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    items = []
    meshes = mcs.build_meshes([(h.V, h.F) for h in hosts])
    if args.bvh_layout != 2:
        for mesh in meshes:
            mesh.build_wide()  # the autotuner tries both layouts
    for i, (mesh, rows) in enumerate(zip(meshes, mcs.sample_rows_batched(meshes, 1024, orient=True))):
        rows = {k: v for k, v in rows.items() if k in ("pos", "nrm", "area", "tri2bin")}
        items.append(dict(mesh=mesh, rows=rows, domain=i % 2, seed=i + 1_000_000 * rank))
    e1.record()
    e1.synchronize()
    return hosts, items, t_gen, e0.elapsed_time(e1)


def run_batch(args, rank, world):
    """The 512-mesh batch: every step is one replay of the graph-captured
    batched estimate (all meshes' setup and tangent balls, ONE persistent walk
    launch over all meshes, histograms and assembly).  The graph records CUDA
    events around its phases at every replay, so the walk kernel's time is
    measured inside the timed steps."""
    import torch
    import paper_2606_05581_b300 as mcs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    W = args.walks or 512
    hosts, items, t_gen, prep_ms = _batch_setup(args, dev, rank)
    params = mcs.default_params(walks_per_row=W, prec=args.prec, killing_walks=64 * W, bvh_layout=args.bvh_layout)
    b = mcs.Batch(items, params, assemble=True)
    t0 = time.time()
    tuned, trials = b.autotune(sample_fraction=1.0 / 64)
    tune_s = time.time() - t0
    tuned.timing = 1  # phase events inside the captured graph
    b.params = tuned
    t0 = time.time()
    nodes = b.capture()
    capture_s = time.time() - t0
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.launch()
    torch.cuda.synchronize()
    peaks = mcs.probe_peaks()  # the roofline's ceilings, measured before the timed region
    barrier(world)
    clk = ClockSampler(dev.index) if rank == 0 else None
    if clk:
        clk.start()
    l0 = mcs.launch_count()
    times, phases = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")
        s0.record(stream)
        b.launch()
        s1.record(stream)
        torch.cuda.nvtx.range_pop()
        s1.synchronize()
        times.append(s0.elapsed_time(s1))
        phases.append(b.graph_stats()[1]["phase_ms"])  # this replay's phases (read after its end)
    launches = mcs.launch_count() - l0
    barrier(world)
    clocks = clk.stop() if clk else None
    status, tot, per = b.graph_stats()
    ms_max = allreduce_max(float(np.mean(times)), world)
    steps = tot["steps"] + tot["killing_steps"]
    value = steps * world / (ms_max / 1e3)
    n_rows = sum(int(it["rows"]["pos"].shape[0]) for it in items)
    walks = tot["walks"] + sum(64 * W for it in items if it["domain"] == 1)
    e2e = _batch_e2e(args, hosts, tuned, stream)
    if rank != 0:
        return None
    phase = np.mean(np.array(phases), axis=0).tolist()
    # node and triangle counts of the same walks (counter-based: identical walks), untimed
    cp = mcs.default_params(**{f: getattr(tuned, f) for f, _ in mcs.Params._fields_
                               if f not in ("origin", "domain", "seed", "origin_auto")})
    cp.timing = 0
    cp.count_work = 1
    _, cst, _ = b.run(cp)
    assert cst["steps"] + cst["killing_steps"] == steps
    width = 4 if tuned.bvh_layout == 4 else 2
    precision = _fp32_batched_vs_fp64_plain(mcs, items[:16], W, tuned)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"f{args.prec}", "data": "synthetic",
        "config": dict(workload_config(args), parallelism=f"replicas{world}",
                       total_faces=int(sum(h.nf for h in hosts))),
        "rows_per_s": n_rows * world / (ms_max / 1e3),
        "walks_per_s": walks * world / (ms_max / 1e3),
        "closest_point_queries_per_s": value,
        "walk_steps_per_step": steps, "capped_walks_per_step": tot["capped"] + tot["killing_capped"],
        "lost_walks_per_step": tot["lost"],
        "discarded_rows": tot["discarded_rows"], "status": status,
        "phase_ms": {"mesh_generation_host": t_gen * 1e3, "bvh_builds_and_sample_rows": prep_ms,
                     "setup_and_tangent_balls": phase[0], "walks": phase[1], "histogram_and_assembly": phase[2]},
        "autotune": {"seconds": tune_s, "chosen": {"threads_per_block": tuned.threads_per_block,
                                                   "blocks_per_sm": tuned.blocks_per_sm,
                                                   "queue_order": tuned.queue_order,
                                                   "bvh_layout": tuned.bvh_layout,
                                                   "lanes_per_query": tuned.lanes_per_query}, "trials": trials},
        "graph": {"nodes": nodes, "capture_and_instantiate_s": capture_s},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "gpu_launches_note": "library kernels per graph replay x steps (mcs_launch_count); CUB kernels excluded",
        "roofline": _walk_roofline(cst, phase[1], f"k_walks (FP{args.prec}, mixed batch, one launch)", peaks,
                                   width),
        "peaks_measured": peaks,
        "fp32_batched_vs_fp64_plain": precision,
        "clocks": clocks,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args, samples=1, hosts=hosts)[0]
    return line


def _fp32_batched_vs_fp64_plain(mcs, items, W, tuned):
    """The metric's comparison on the batch's first meshes, untimed by the
    headline: FP32 walks of all of them in one batched launch (the tuned
    shape) against FP64 walks estimated one mesh at a time (the plain path),
    each timed with CUDA events around the whole estimate.  Both precisions
    draw the same Philox counters, so at equal walks per row they reach the
    same error (the precision workload's table; the statistical GPU tests):
    the walk-step rates compare them at equal error.  Lambda's relative
    difference (Frobenius norm) and the share of equal hit-count entries
    show how close the two estimates are."""
    import torch
    dev_events = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    p32 = mcs.default_params(**{f: getattr(tuned, f) for f, _ in mcs.Params._fields_
                                if f not in ("origin", "domain", "seed", "origin_auto", "timing", "count_work")})
    b = mcs.Batch(items, p32, assemble=True)
    b.run()
    a, e = dev_events()
    a.record()
    _, t32, _ = b.run()
    e.record()
    e.synchronize()
    ms32 = a.elapsed_time(e)
    steps32 = t32["steps"] + t32["killing_steps"]
    ms64, steps64 = 0.0, 0
    num = den = 0.0
    same = total = 0
    ws = mcs.Workspace()
    for i, it in enumerate(items):
        p64 = mcs.default_params(walks_per_row=W, prec=64, killing_walks=64 * W, domain=it["domain"],
                                 seed=it["seed"])
        a, e = dev_events()
        a.record()
        r = mcs.estimate_dtn(it["mesh"], it["rows"], p64, workspace=ws)
        e.record()
        e.synchronize()
        ms64 += a.elapsed_time(e)
        steps64 += r["stats"]["steps"] + r["stats"]["killing_steps"]
        L32, L64 = b.outputs[i]["Lambda"], r["Lambda"]
        num += float(((L32 - L64) ** 2).sum())
        den += float((L64 ** 2).sum())
        R = int(it["rows"]["pos"].shape[0])
        H32, H64 = mcs.dense_hist(b.result(i), R), mcs.dense_hist(r, R)
        same += int((H32 == H64).sum())
        total += H32.numel()
    return {"meshes": len(items), "fp32_batched_steps_per_s": steps32 / (ms32 / 1e3),
            "fp64_plain_steps_per_s": steps64 / (ms64 / 1e3),
            "ratio": (steps32 / (ms32 / 1e3)) / (steps64 / (ms64 / 1e3)),
            "walk_steps": {"fp32": steps32, "fp64": steps64},
            "lambda_rel_diff_frobenius": (num / den) ** 0.5, "hit_count_entries_equal": same / total,
            "note": "same meshes, rows, seeds and walks per row; the two precisions share their Philox counters, "
                    "so equal walks per row is equal error"}


def _batch_e2e(args, hosts, params, stream):
    """The batch end to end through the public API: every mesh's V, F copied
    in from pinned host memory, BVH builds, sample rows, the batched estimate
    (plain enqueue: a new mesh set means new device pointers), and every
    mesh's Lambda copied out; timed on the stream."""
    import torch
    import paper_2606_05581_b300 as mcs
    VF = [(torch.from_numpy(h.V).pin_memory(), torch.from_numpy(h.F).pin_memory()) for h in hosts]
    # the host buffers every mesh's Lambda is read into: pinned once, outside the timed region
    hLs = [torch.empty((1024, 1024), dtype=torch.float64, pin_memory=True) for _ in hosts]
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    h2d = d2h = 0
    dev_vf = []
    for V, F in VF:
        dev_vf.append((V.to("cuda", non_blocking=True), F.to("cuda", non_blocking=True)))
        h2d += V.numel() * 8 + F.numel() * 4
    meshes = mcs.build_meshes(dev_vf)  # every BVH build enqueued before one synchronisation
    if params.bvh_layout == 4:
        for mesh in meshes:
            mesh.build_wide()
    items = [dict(mesh=mesh, rows=rows, domain=i % 2, seed=i)
             for i, (mesh, rows) in enumerate(zip(meshes, mcs.sample_rows_batched(meshes, 1024, orient=True)))]
    b = mcs.Batch(items, params, assemble=True)
    _, tot, _ = b.run()
    outs = []
    for o, hL in zip(b.outputs, hLs):
        assert tuple(o["Lambda"].shape) == tuple(hL.shape)
        hL.copy_(o["Lambda"], non_blocking=True)
        d2h += hL.numel() * 8
        outs.append(hL)
    s1.record(stream)
    s1.synchronize()
    ms = s0.elapsed_time(s1)
    return {"value": (tot["steps"] + tot["killing_steps"]) / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms}


def run_precision(args, rank, world):
    """FP32 vs FP64 walks on the same Philox counters: per-eigenvalue error
    against an FP64 reference estimate with many more walks."""
    import torch
    import paper_2606_05581_b300 as mcs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    m = make_mesh(args)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    k = 128
    ws, eig_ws = mcs.Workspace(), mcs.Workspace()

    def spectrum(prec, W, seed):
        p = mcs.default_params(walks_per_row=W, prec=prec, domain=1, killing_walks=64 * W, seed=seed, timing=1)
        res = mcs.estimate_dtn(mesh, rows, p, workspace=ws)
        ev, _, est = mcs.steklov_modes(res["Lambda"], rows["area"], k, vectors=False, workspace=eig_ws)
        st = res["stats"]
        return ev.cpu().numpy(), st["phase_ms"][1], st["steps"] + st["killing_steps"], est

    Wref = args.ref_walks
    t0 = time.time()
    ref, ref_ms, _, ref_eig = spectrum(64, Wref, 999)
    ref_s = time.time() - t0
    table = []
    for W in (1024, 4096, 16384):
        for prec in (32, 64):
            evs, ms, steps = [], [], []
            for seed in range(args.seeds):
                ev, wms, st, _ = spectrum(prec, W, seed)
                evs.append(ev)
                ms.append(wms)
                steps.append(st)
            evs = np.array(evs)
            rel = np.abs(evs - ref[None, :]) / np.abs(ref[None, :])
            se = evs.std(axis=0, ddof=1) / np.abs(ref) if args.seeds > 1 else np.zeros(k)
            table.append({"prec": prec, "walks_per_row": W, "seeds": args.seeds,
                          "mean_rel_err": float(rel.mean()), "median_rel_err": float(np.median(rel)),
                          "max_rel_err": float(rel.max()),
                          "rel_err_first16": rel.mean(axis=0)[:16].tolist(),
                          "rel_se_single_run_mean": float(se.mean()),
                          "walk_ms": float(np.mean(ms)), "walk_steps": float(np.mean(steps)),
                          "walk_steps_per_s": float(np.mean(steps) / (np.mean(ms) / 1e3)),
                          "fp32_fp64_spectrum_rel_diff": None})
    # FP32 vs FP64 on identical counters: how far apart the two spectra are
    for W in (1024, 4096, 16384):
        e32 = spectrum(32, W, 0)[0]
        e64 = spectrum(64, W, 0)[0]
        for row in table:
            if row["walks_per_row"] == W:
                row["fp32_fp64_spectrum_rel_diff"] = float(np.max(np.abs(e32 - e64) / np.abs(e64)))
    # equal error: the walks per row each precision needs for the FP32 error at
    # W = 16384, by log-log interpolation between the measured points (no
    # extrapolation beyond them), and the walk time that takes at the
    # measured walk steps per walk and walk steps per second
    def need(prec, target):
        rs = sorted((r for r in table if r["prec"] == prec), key=lambda r: r["walks_per_row"])
        lw = np.log([r["walks_per_row"] for r in rs])
        le = np.log([r["mean_rel_err"] for r in rs])
        # errors fall with W: interpolate W(err) on the decreasing sequence
        w = float(np.exp(np.interp(np.log(target), le[::-1], lw[::-1])))
        near = min(rs, key=lambda r: abs(math.log(r["walks_per_row"]) - math.log(w)))
        return w, near["walk_steps_per_s"], near["walk_steps"] / near["walks_per_row"]
    target = [r for r in table if r["prec"] == 32 and r["walks_per_row"] == 16384][0]["mean_rel_err"]
    w32, sps32, spw32 = need(32, target)
    w64, sps64, spw64 = need(64, target)
    t32 = w32 * spw32 / sps32
    t64 = w64 * spw64 / sps64
    fp32_best = max(r["walk_steps_per_s"] for r in table if r["prec"] == 32)
    return {"metric": METRIC, "value": fp32_best, "unit": UNIT, "n_gpus": 1, "steps": None, "warmup": None,
            "higher_is_better": True, "dtype": "f32 vs f64", "data": "synthetic",
            "config": dict(workload="precision", mesh="two icospheres s4, R=0.5, centres 1.5 apart",
                           domain="exterior", killing_walks="64 W", steklov_k=k, reference=f"FP64, W={Wref}",
                           seeds=args.seeds),
            "reference": {"walks_per_row": Wref, "walk_ms": ref_ms, "seconds": ref_s, "eig": ref_eig,
                          "first8": ref[:8].tolist()},
            "table": table,
            "equal_error": {"target_mean_rel_err": target, "fp32_walks_per_row": w32, "fp64_walks_per_row": w64,
                            "fp32_walk_seconds": t32, "fp64_walk_seconds": t64, "fp64_over_fp32_time": t64 / t32}}


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    """Max over the replicas (the job's step time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank, base=0):
    """Each replica estimates its own problem: the walk seed is offset by the rank."""
    return base + rank


# ---------------------------------------------------------------- the oracle as baseline
def cpu_baseline(args, samples=1, hosts=None):
    """Oracle (plain C, brute-force closest point over all triangles) on a
    bounded sample of the workload, in the same precision."""
    from oracle import oracle as O
    nthr = O.num_threads()
    rng = np.random.default_rng(0)
    out = []
    if args.workload == "batch":
        import meshgen
        hosts = hosts or [meshgen.batch_mesh(0), meshgen.batch_mesh(1)]
        W = args.walks or 512
        nr, nw = max(2, nthr), W // 2
        rows_of = []
        for i in range(2):  # mesh 0 (interior) and mesh 1 (exterior): the oracle's own rows and origin
            h = hosts[i]
            rows = O.fps_rows(h.V, h.F, 1024, orient=True)
            rows_of.append((rows, O.interior_origin(h.V, h.F, rows) if i % 2 else None))
        for s in range(samples):
            steps = 0
            dt = 0.0
            for i in range(2):
                h = hosts[i]
                rows, origin = rows_of[i]
                rl = np.sort(rng.choice(1024, nr, replace=False)).astype(np.int32)
                t0 = time.time()
                est = O.estimate(h.V, h.F, rows, W, 1e-3, exterior=bool(i % 2), origin=origin, seed=i,
                                 prec=args.prec, row_list=rl, params=dict(walk_limit=nw))
                dt += time.time() - t0
                steps += int(est["steps"].sum())
            out.append({"value": steps / dt, "unit": UNIT, "cores": nthr, "kind": "oracle",
                        "sample": f"meshes 0 (interior, {hosts[0].nf} faces) and 1 (exterior, {hosts[1].nf} "
                                  f"faces) of the batch: {nr} random sample rows x the first {nw} of their {W} "
                                  f"walks each (fp{args.prec}, brute-force closest point); {steps} walk steps in "
                                  f"{dt:.1f} s; walk steps/s is per-step work, so it carries over to the whole "
                                  f"batch unchanged"})
        return out
    m = make_mesh(args)
    if args.workload == "wild_2m":
        # rows at random face centroids with their face normals (the oracle's
        # farthest-point sampling over 2M faces alone takes minutes); every
        # face mapped to row 0 -- the walks and their queries are the same work
        n = max(2, nthr)
        f = rng.choice(m.nf, n, replace=False)
        a, b_, c = m.V[m.F[f, 0]], m.V[m.F[f, 1]], m.V[m.F[f, 2]]
        nrm = np.cross(b_ - a, c - a)
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        rows = dict(pos=(a + b_ + c) / 3.0, nrm=nrm / (2.0 * area[:, None]), area=area,
                    tri2bin=np.zeros(m.nf, np.int32))
        W = 4
        for s in range(samples):
            t0 = time.time()
            est = O.estimate(m.V, m.F, rows, W, 1e-3, exterior=False, seed=s, prec=args.prec)
            dt = time.time() - t0
            steps = int(est["steps"].sum())
            out.append({"value": steps / dt, "unit": UNIT, "cores": nthr, "kind": "oracle",
                        "sample": f"{n} rows at random face centroids x {W} walks, interior, fp{args.prec}, "
                                  f"brute-force closest point over {m.nf} triangles; {steps} walk steps in "
                                  f"{dt:.1f} s"})
        return out
    rows = O.vertex_rows(m.V, m.F)
    W = args.walks or 1024
    t0 = time.time()
    origin = O.interior_origin(m.V, m.F, rows)
    t_origin = time.time() - t0
    nrows = max(2, nthr)
    for s in range(samples):
        rl = np.sort(rng.choice(m.nv, nrows, replace=False)).astype(np.int32)
        t0 = time.time()
        est = O.estimate(m.V, m.F, rows, W, 1e-3, exterior=True, origin=origin, seed=0, prec=args.prec,
                         row_list=rl)
        dt = time.time() - t0
        steps = int(est["steps"].sum())
        out.append({"value": steps / dt, "unit": UNIT, "cores": nthr, "kind": "oracle",
                    "sample": f"{nrows} rows x {W} walks of the same exterior estimate "
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
    ap.add_argument("--workload", default="batch", choices=WORKLOADS)
    ap.add_argument("--walks", type=int, default=0, help="walks per row (0: the workload's)")
    ap.add_argument("--meshes", type=int, default=512, help="batch workload: number of meshes")
    ap.add_argument("--seeds", type=int, default=4,
                    help="precision workload: seeds per configuration (variance workload: 8x as many)")
    ap.add_argument("--ref-walks", type=int, default=65536, help="precision workload: reference walks per row")
    ap.add_argument("--prec", type=int, default=32, choices=[32, 64])
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--bvh-layout", type=int, default=0, choices=[0, 2, 4],
                    help="BVH node layout of the walk queries: 0 library default, 2 binary, 4 four-wide")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "batch":
        line = run_batch(args, rank, world)
    elif args.workload == "precision":
        line = run_precision(args, rank, world) if rank == 0 else None
    elif args.workload == "variance":
        line = run_variance(args, rank, world) if rank == 0 else None
    else:
        line = run_ours(args, rank, world)
    if line is not None:
        print(json.dumps(line))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
