#!/usr/bin/env python3
"""Benchmark of the SOR stress-majorization layout path on GB300.

Workload (graph-drawing benchmark stand-ins, 2-D, X^0 uniform in [0,1]^2):
Erdos-Renyi n=10,000 mean degree 6, Delaunay mesh of 20,000 uniform points,
random binary tree n=16,383.  One step lays out every graph of the workload:
ideal distances from the CSR (multi-source BFS), then Algorithm 2 to
convergence (relative displacement 1e-4, at most 1000 iterations) at each
omega of the step's sweep.  The default sweep is the classical factor 1.5
(the paper's omega = 0.5); ``--sweep`` runs the classical factors 1.0 .. 1.9.

Metric: unordered pair interactions per second over the whole step (every
all-pairs pass counts n(n-1)/2 pairs: each CG matvec, and each stress/RHS
evaluation of a candidate layout); SOR iterations per second beside it.
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

from paper_1711_01228_gb300 import synth  # noqa: E402

WORKLOAD = ("er10k", "delaunay20k", "tree16k")
FLOP_K2 = {1: 13, 2: 19, 3: 25}   # stress + L^X X per unordered pair per candidate
FLOP_MV = {1: 4, 2: 8, 3: 12}     # L^W p per unordered pair


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


KERNEL_SOURCES = ("fd_internal.cuh", "fd_solver.cuh", "fd_solver_d2.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fd_main_kernel_bench_traffic.txt")


def kernel_hash() -> str:
    """Hash of the layout kernel's sources: DRAM counters taken from another
    version of the kernel do not describe this one."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1711_01228_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes (read + write) per layout-kernel launch of this workload, from
    the committed ncu capture, or None when the kernel has changed since."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    with open(TRAFFIC_FILE) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_hash") != kernel_hash() or kv.get("workload") != workload:
        return None
    return float(kv["dram_bytes_per_launch"])


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, device, world):
    """Each value's maximum over the ranks (the slowest replica sets the job's time)."""
    if world <= 1:
        return list(values)
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: every rank processes units_per_rank in at most ms."""
    return units_per_rank * world / (ms / 1e3)


def make_inputs(names, dim=2, seed=0):
    out = []
    for nm in names:
        rp, ci = synth.workload(nm, seed)
        n = len(rp) - 1
        out.append((nm, rp, ci, synth.initial_layout(n, dim, seed)))
    return out


def omegas(sweep: bool):
    # classical SOR factor omega_c = 1 + omega (paper's omega)
    return [round(0.1 * k, 1) for k in range(10)] if sweep else [0.5]


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1711_01228_gb300 import api, build

    build.build()
    api.lib()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    inputs = make_inputs(args.workload.split(","), args.dim)
    oms = omegas(args.sweep)
    dev_inputs = [(nm, torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), torch.from_numpy(x0).to(dev))
                  for nm, rp, ci, x0 in inputs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    opts = dict(tol=1e-4, max_iter=args.max_iter, stop=api.STOP_REL_DISP)

    def one_step(acc, host=False):
        for (nm, rp, ci, x0), (_, rpd, cid, x0d) in zip(inputs, dev_inputs):
            if host:
                L = api.Layout(rp, ci, dim=args.dim, disconnected_policy=1)
            else:
                L = api.Layout(rpd, cid, dim=args.dim, disconnected_policy=1, stream=stream.cuda_stream)
            info = L.info()
            acc["apsp_ms"] += info["apsp_ms"]
            n_g, m2 = len(rp) - 1, int(rp[-1])
            # edge pass: per pass over the edge list 20 B per vertex (row_ptr, reached word, next word)
            # and 12 B per edge end (col_idx, the neighbour's frontier word); 1 B per pair written once
            acc["apsp_bytes"] += info["bfs_sweeps"] * (20.0 * n_g + 12.0 * m2) + 0.5 * n_g * (n_g - 1)
            acc["h2d"] += rp.nbytes + ci.nbytes
            for om in oms:
                if host:
                    X = x0.copy()
                    acc["h2d"] += X.nbytes
                else:
                    X = x0d.clone()
                r = L.run(X, omega=om, **opts)
                if host:
                    acc["d2h"] += X.nbytes + 8
                st = r.stats
                acc["pairs"] += st["pair_passes"] * st["pairs"]
                acc["iters"] += st["iterations"]
                acc["kernel_ms"] += st["kernel_ms"]
                acc["launches"] += 1
                acc["flops"] += st["pairs"] * (st["matvec_passes"] * FLOP_MV[args.dim] + st["stress_passes"] * FLOP_K2[args.dim])
                acc["cg"] += st["cg_steps"]
                acc["runs"].append((nm, om, st["iterations"], st["cg_steps"], st["final_stress"]))
            acc["n_launch_total"] += 3 + len(oms)  # BFS, fill, row sums (the launch list: one each), + one layout kernel per run
            L.close()

    def zero():
        return dict(pairs=0.0, iters=0, kernel_ms=0.0, apsp_ms=0.0, apsp_bytes=0.0, flops=0.0, cg=0, launches=0,
                    h2d=0, d2h=0, runs=[], n_launch_total=0)

    for _ in range(args.warmup):
        one_step(zero())
    torch.cuda.synchronize()
    # ----- device-resident timed region
    sampler = ClockSampler(local_rank)
    acc = zero()
    times = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between steps (outside the timed interval)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        one_step(acc)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = sum(times)
    # ----- end to end through the public API with host buffers
    acc_e = zero()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps if not args.no_e2e else 0):
        one_step(acc_e, host=True)
    torch.cuda.synchronize()
    e2e_ms = max((time.perf_counter() - t0) * 1e3, 1e-9)
    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], dev, world)
    value = job_rate(acc["pairs"], world, total_ms)
    e2e_value = job_rate(acc_e["pairs"], world, e2e_ms)
    peaks, src = _peaks()
    clk = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * clk * 1e6 / 1e12  # TFLOP/s at the maximum SM clock
    fp32_measured = {"fma_f32": api.fp32_peak(False), "fma_f32x2": api.fp32_peak(True)}
    achieved = acc["flops"] / (acc["kernel_ms"] / 1e3) / 1e12
    batched = run_batched(args, local_rank, fp32_peak) if (args.batch and rank == 0) else None
    differentiable = run_differentiable(args, local_rank) if (args.grad and rank == 0) else None
    direct = run_direct(args, local_rank, peaks, fp32_peak) if (args.direct_sec and rank == 0) else None
    vertex_omega = run_vertex_omega(args, local_rank) if (args.direct_sec and rank == 0) else None
    line = {
        "metric": "pair-interactions/s",
        "value": value,
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(args, inputs, world),
        "sor_iterations_per_s": acc["iters"] * world / (total_ms / 1e3),
        "cg_steps_per_sor_iteration": acc["cg"] / max(acc["iters"], 1),
        "gpu_launches": acc["n_launch_total"],
        "roofline": {"bound": "alu", "kernel": "fd_main_kernel", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": measured_traffic(",".join(args.workload.split(","))),
                     "traffic_unit": "DRAM bytes per launch (ncu, read + write)",
                     "peak_note": f"FP32 CUDA cores {sms} SMs x 128 x 2 flop at {clk:.0f} MHz ({src} max clock)",
                     "peak_measured_tflops": fp32_measured,
                     "peak_measured_note": "fd_fp32_peak: 16 independent FMA chains per thread, scalar and "
                                           "two-wide packed, best of 5 launches"},
        "apsp": {"kernel": "bfs_batch_kernel", "ms_per_step": acc["apsp_ms"] / args.steps,
                 "algorithmic_bytes_per_step": acc["apsp_bytes"] / args.steps,
                 "achieved_gbs": acc["apsp_bytes"] / (acc["apsp_ms"] / 1e3) / 1e9,
                 "peak_gbs": peaks.get("hbm_gbs", 6800.0),
                 "frac": acc["apsp_bytes"] / (acc["apsp_ms"] / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0),
                 "note": "bytes a pass over the edge list must move per 64-source search (row_ptr, reached and "
                         "next words, col_idx, neighbour frontier words) times the passes run, plus 1 B per "
                         "pair written; the per-search words are L2-resident, so this is not DRAM traffic"},
        "layout_kernel_ms_per_step": acc["kernel_ms"] / args.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": acc_e["h2d"] // args.steps,
                "d2h_bytes_per_step": acc_e["d2h"] // args.steps},
        "runs": acc["runs"][: len(inputs) * len(oms)],
    }
    if batched is not None:
        line["batched"] = batched
    if differentiable is not None:
        line["differentiable"] = differentiable
    if direct is not None:
        line["direct_solver"] = direct
    if vertex_omega is not None:
        line["vertex_omega"] = vertex_omega
    return line


def run_batched(args, local_rank, peak_tflops):
    """The batched form: 4096 independent graphs in one persistent launch,
    timed beside the single-graph path on an evenly spaced sample of the same
    graphs at the same accuracy (tolerance, iteration cap, omega)."""
    import torch

    from paper_1711_01228_gb300 import api

    dev = torch.device("cuda", local_rank)
    G = args.batch_graphs
    graphs = synth.batch_graphs(G, seed=0)
    sizes = np.array([len(rp) - 1 for rp, _ in graphs])
    X0 = synth.batch_initial_layout(sizes, 2, seed=0)
    stream = torch.cuda.Stream(dev)  # a capturable stream for the CUDA graph of the launch
    opts = dict(omega=0.5, tol=1e-4, max_iter=args.max_iter, stop=api.STOP_REL_DISP)
    B = api.Batch.from_graphs(graphs, dim=2, disconnected_policy=1, stream=stream.cuda_stream)
    Xd = torch.from_numpy(X0).to(dev)
    torch.cuda.synchronize()
    groups, stages = B.tune(Xd, probe_iter=5, repeats=2, **opts)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    X = Xd.clone()
    B.run(X, **opts)  # warm-up (captures the launch as a CUDA graph)
    times, res = [], None
    for _ in range(max(1, args.batch_steps)):
        X = Xd.clone()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        res = B.run(X, **opts)
        times.append(res.stats["kernel_ms"])
    ms = statistics.median(times)
    info = B.info()
    st = res.stats
    it = res.iterations
    pairs_s = st["pairs"] / (ms / 1e3)
    flops = 0.0
    for g in range(G):
        pg = 0.5 * sizes[g] * (sizes[g] - 1)
        flops += pg * (res.matvec_passes[g] * FLOP_MV[2] + res.stress_passes[g] * FLOP_K2[2])
    achieved = flops / (ms / 1e3) / 1e12
    Xb = X.cpu().numpy()
    B.close()
    # the single-graph path (fd_layout_create + fd_run per graph) on every k-th graph by size
    order = np.argsort(-sizes, kind="stable")
    sample = order[:: max(1, G // args.batch_sample)][: args.batch_sample]
    plain_ms, rel, iters_ok, batch_ms_sample = 0.0, [], 0, 0.0
    gp = np.concatenate([[0], np.cumsum(sizes)])
    for g in sample.tolist():
        rp, ci = graphs[g]
        x = torch.from_numpy(X0[gp[g]:gp[g + 1]].copy()).to(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with api.Layout(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), dim=2, disconnected_policy=1,
                        stream=torch.cuda.current_stream(dev).cuda_stream) as L:
            r = L.run(x, **opts)
        torch.cuda.synchronize()
        plain_ms += (time.perf_counter() - t0) * 1e3
        batch_ms_sample += float(res.graph_ms[g])
        rel.append(abs(r.stress - res.stress[g]) / max(abs(r.stress), 1e-30))
        iters_ok += int(abs(r.iterations - int(it[g])) <= max(1, int(np.ceil(0.02 * r.iterations))))
    del Xb
    return {
        "workload": f"{G} graphs, n log-uniform in [16, 2048] (seeded), even index Erdos-Renyi mean degree 4, "
                    "odd index random geometric (unit square, radius bisected to mean degree 6); 2-D, X0 U[0,1]^2, "
                    f"omega_c 1.5, rel-disp tol 1e-4, max {args.max_iter} iters, unreachable pairs at (largest d)+1",
        "graphs": G, "total_vertices": int(sizes.sum()), "ms": ms, "steps": len(times),
        "pairs_per_s": pairs_s, "sor_iterations_per_s": float(it.sum()) / (ms / 1e3), "graphs_per_s": G / (ms / 1e3),
        "converged": int((it < args.max_iter).sum()), "hit_max_iter": int((it >= args.max_iter).sum()),
        "launch": {"kernel": "fd_batch_kernel", "grid": info["grid"], "groups_per_cta": groups, "stages": stages,
                   "tuned": True, "cuda_graph": bool(info["graph_captured"]), "launches_per_run": 1},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops},
        "l2": "flushed before each timed run (256 MB write)",
        "plain_sample": {"graphs": len(sample), "selection": "every k-th graph in size order",
                         "plain_ms_total": plain_ms, "batched_device_ms_same_graphs": batch_ms_sample,
                         "plain_ms_per_graph": plain_ms / len(sample),
                         "max_rel_stress_diff": float(max(rel)), "iterations_within_2pct": iters_ok / len(sample),
                         "note": "plain = fd_layout_create + fd_run per graph (host wall time, includes the "
                                 "distance set-up); batched = device time its CTA spent on the graph"},
    }


def run_differentiable(args, local_rank):
    """The differentiable form: stress of a weighted random geometric graph in
    3-D with its two gradients (positions: the force kernel; edge lengths:
    shortest-path back-propagation), timed beside the plain stress pass."""
    import torch

    from paper_1711_01228_gb300 import api, autograd

    dev = torch.device("cuda", local_rank)
    # the largest connected component of a random geometric graph (derivatives in the
    # edge lengths need every pair connected)
    rp0, ci0, pts0 = synth.random_geometric(args.grad_n, 3, 6.0, seed=0)
    rp, ci, keep = _largest_component(rp0, ci0)
    pts = pts0[keep]
    n = len(rp) - 1
    s = 0
    rng = np.random.default_rng(s)
    w = np.empty(len(ci), dtype=np.float32)
    seen = {}
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            key = (min(u, int(ci[e])), max(u, int(ci[e])))
            seen.setdefault(key, np.float32(rng.uniform(0.5, 2.0)))
            w[e] = seen[key]
    X = torch.from_numpy((pts * 10.0).astype(np.float32)).to(dev)
    wt = torch.from_numpy(w).to(dev).requires_grad_(True)
    rpt, cit = torch.from_numpy(rp), torch.from_numpy(ci)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    L = api.Layout(rp, ci, dim=3, edge_len=w, disconnected_policy=0)
    F = torch.empty_like(X)
    G = torch.empty(len(ci), dtype=torch.float32, device=dev)
    ms_energy = timed(lambda: L.energy(X))
    ms_forces = timed(lambda: L.forces(X, out=F))
    ms_lgrad = timed(lambda: L.length_grad(X, out=G))
    create_ms = L.info()["apsp_ms"]
    L.close()

    def step():
        wt.grad = None
        f = autograd.stress_lengths(X, wt, rpt, cit)
        f.backward()

    ms_step = timed(step)

    # adjoint through K = 32 unrolled iterations (checkpoint every 8): fit lengths to target distances
    K, every = 32, 8
    rng2 = np.random.default_rng(1)
    Yt = torch.from_numpy((rng2.random((n, 3)) * 10.0).astype(np.float32)).to(dev)
    pi = torch.from_numpy(rng2.integers(0, n, 4096)).to(dev)
    pj = torch.from_numpy(rng2.integers(0, n, 4096)).to(dev)
    keep = pi != pj
    pi, pj = pi[keep], pj[keep]
    tgt = (Yt[pi] - Yt[pj]).norm(dim=1)
    X0 = X.clone()

    def unrolled_step():
        wt.grad = None
        XK = autograd.unrolled_layout(X0, wt, rpt, cit, K=K, omega=0.5, every=every)
        loss = ((XK[pi] - XK[pj]).norm(dim=1) - tgt).pow(2).sum()
        loss.backward()

    ms_unrolled = timed(unrolled_step, reps=2)

    def unrolled_step_direct():
        wt.grad = None
        XK = autograd.unrolled_layout(X0, wt, rpt, cit, K=K, omega=0.5, every=every, solver=api.SOLVER_DIRECT)
        loss = ((XK[pi] - XK[pj]).norm(dim=1) - tgt).pow(2).sum()
        loss.backward()

    ms_unrolled_direct = timed(unrolled_step_direct, reps=2)

    def unrolled_forward():
        with torch.no_grad():
            autograd.unrolled_layout(X0, wt.detach(), rpt, cit, K=K, omega=0.5, every=every)

    ms_unrolled_fwd = timed(unrolled_forward, reps=2)
    pairs = 0.5 * n * (n - 1)
    return {"workload": f"largest component (n={n}) of a random geometric graph of {args.grad_n} points in the "
                        "unit cube x 10, mean degree 6 (seed 0); edge lengths seeded in [0.5, 2]; 3-D",
            "stress_pass_ms": ms_energy, "position_grad_ms": ms_forces, "length_grad_ms": ms_lgrad,
            "weighted_apsp_ms": create_ms, "autograd_step_ms": ms_step,
            "unrolled": {"iterations": K, "checkpoint_every": every, "omega_c": 1.5,
                         "forward_ms": ms_unrolled_fwd, "forward_backward_ms": ms_unrolled,
                         "forward_backward_ms_direct_solver": ms_unrolled_direct,
                         "loss": "squared error of 4096 sampled pair distances of X^K against a seeded "
                                 "random layout's"},
            "stress_pairs_per_s": pairs / (ms_energy / 1e3), "position_grad_pairs_per_s": pairs / (ms_forces / 1e3),
            "note": "autograd step = fd_layout_create (weighted shortest paths) + stress + forces + length "
                    "gradient, through torch.autograd; every value from the CUDA library"}


def run_direct(args, local_rank, peaks, fp32_peak):
    """The direct solver of Eq. (2-5) beside CG on one graph of the workload:
    the factorisation (fd_factor: FP32 Gauss-Jordan inverse of the shifted
    L^W), then Algorithm 2 with each solver, same options as the headline
    runs.  The dense apply is a phase of the layout kernel; its duration comes
    from the kernel's %globaltimer marks (fd_timeline), the rest from CUDA
    events."""
    import ctypes

    import torch

    from paper_1711_01228_gb300 import api

    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    if args.direct_n:
        rp, ci = synth.delaunay(args.direct_n, seed=0)
        name = f"delaunay{args.direct_n}"
    else:
        name = "delaunay20k"
        rp, ci = synth.workload(name)
    n = len(rp) - 1
    x0 = synth.initial_layout(n, 2, seed=0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts = dict(omega=0.5, tol=1e-4, max_iter=args.max_iter, stop=api.STOP_REL_DISP)
    L = api.Layout(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), dim=2, disconnected_policy=1,
                   stream=stream.cuda_stream)
    X0 = torch.from_numpy(x0).to(dev)
    n_pad = L.info()["tile"] * ((n + L.info()["tile"] - 1) // L.info()["tile"])

    def runs(solver, reps):
        out = []
        for _ in range(reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            X = X0.clone()
            r = L.run(X, solver=solver, **opts)
            out.append(r.stats)
        return out

    runs(api.SOLVER_CG, 1)
    cg = runs(api.SOLVER_CG, 2)
    factor_ms = [L.factor() for _ in range(2)]
    runs(api.SOLVER_DIRECT, 1)
    dr = runs(api.SOLVER_DIRECT, 2)
    # phase durations of one direct run: tag 10 = the dense apply (ns between the barrier before it and its own)
    cap = 400000
    api.lib().fd_timeline_enable(L._h, cap)
    L.run(X0.clone(), solver=api.SOLVER_DIRECT, **opts)
    buf = np.zeros(2 * cap)
    cnt = ctypes.c_int32()
    api.lib().fd_timeline_read(L._h, buf.ctypes.data, cap, ctypes.byref(cnt))
    api.lib().fd_timeline_enable(L._h, 0)
    tl = buf[:2 * cnt.value].reshape(-1, 2)
    apply_ns = [b[1] - a[1] for a, b in zip(tl[:-1], tl[1:]) if int(b[0]) == 10]
    L.close()
    ms_cg = statistics.median(st["kernel_ms"] for st in cg)
    ms_dr = statistics.median(st["kernel_ms"] for st in dr)
    fac = min(factor_ms)
    nb = n_pad // 128
    # symmetric sweep: per block step, m (m + 1) / 2 trailing block products (lower blocks, m = nb - 1)
    # and m panel products of 2 * 128^3 flops each (the pivot blocks are not counted)
    m = nb - 1
    gj_flops = nb * (m * (m + 1) // 2 + m) * 2.0 * 128 ** 3
    apply_bytes = 4.0 * n_pad * n_pad
    apply_us = float(np.mean(apply_ns)) / 1e3 if apply_ns else float("nan")
    hbm = peaks.get("hbm_gbs", 6800.0)
    st_cg, st_dr = cg[0], dr[0]
    return {"workload": f"{name} (n={n}), 2-D, X0 U[0,1]^2 seed 0, omega_c 1.5, rel-disp tol 1e-4, "
                        f"max {args.max_iter} iters; L2 flushed before each run",
            "cg": {"kernel_ms": ms_cg, "iterations": st_cg["iterations"], "solver_steps": st_cg["cg_steps"],
                   "matvec_passes": st_cg["matvec_passes"], "final_stress": st_cg["final_stress"],
                   "pairs_per_s": st_cg["pair_passes"] * st_cg["pairs"] / (ms_cg / 1e3)},
            "direct": {"kernel_ms": ms_dr, "iterations": st_dr["iterations"], "solver_steps": st_dr["cg_steps"],
                       "matvec_passes": st_dr["matvec_passes"], "dense_applies": st_dr["cg_steps"],
                       "final_stress": st_dr["final_stress"],
                       "pairs_per_s": st_dr["pair_passes"] * st_dr["pairs"] / (ms_dr / 1e3)},
            "factor": {"kernel": "sw_update_kernel (+ sw_pivot/panel/finish, dense_build)", "ms": fac,
                       "flops": gj_flops, "achieved_tflops": gj_flops / (fac / 1e3) / 1e12,
                       "peak_tflops": fp32_peak, "frac": gj_flops / (fac / 1e3) / 1e12 / fp32_peak,
                       "bound": "alu", "bytes_resident": apply_bytes},
            "dense_apply": {"bound": "hbm", "bytes": apply_bytes, "us": apply_us,
                            "achieved_gbs": apply_bytes / (apply_us * 1e-6) / 1e9 if apply_ns else None,
                            "peak_gbs": hbm,
                            "frac": apply_bytes / (apply_us * 1e-6) / 1e9 / hbm if apply_ns else None,
                            "note": "one read of the FP32 inverse (4 n_pad^2 bytes) per application; duration "
                                    "from the layout kernel's %globaltimer marks, grid barrier included"},
            "speedup_per_run": ms_cg / ms_dr,
            "break_even_runs": fac / (ms_cg - ms_dr) if ms_cg > ms_dr else None}


def run_vertex_omega(args, local_rank):
    """Per-vertex relaxation factors (omega_i = omega m_i, Sec. 6) on the
    Delaunay 20,000 graph with the headline options: no factors, m = 1 (the
    same trajectory: the cost of forming omega_i per vertex) and seeded
    m_i uniform in [0, 2] (the paper gives no rule for choosing them)."""
    import torch

    from paper_1711_01228_gb300 import api

    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    rp, ci = synth.workload("delaunay20k")
    n = len(rp) - 1
    X0 = torch.from_numpy(synth.initial_layout(n, 2, seed=0)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    L = api.Layout(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), dim=2, disconnected_policy=1,
                   stream=stream.cuda_stream)
    cases = {"none": None, "ones": np.ones(n, np.float32),
             "uniform_0_2": np.random.default_rng(0).uniform(0.0, 2.0, n).astype(np.float32)}
    out = {}
    for name, m in cases.items():
        L.set_vertex_omega(m)
        stats = []
        for rep in range(3):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            r = L.run(X0.clone(), omega=0.5, tol=1e-4, max_iter=args.max_iter, stop=api.STOP_REL_DISP)
            if rep > 0:
                stats.append(r.stats)
        ms = statistics.median(st["kernel_ms"] for st in stats)
        st = stats[0]
        out[name] = {"kernel_ms": ms, "iterations": st["iterations"], "accepted": st["accepted"],
                     "final_stress": st["final_stress"], "ms_per_iteration": ms / max(st["iterations"], 1),
                     "pairs_per_s": st["pair_passes"] * st["pairs"] / (ms / 1e3)}
    L.close()
    return {"workload": "delaunay20k (n=20000), 2-D, X0 U[0,1]^2 seed 0, omega 0.5 (classical 1.5) times "
                        "per-vertex factors m, rel-disp tol 1e-4; L2 flushed before each run; median of 2",
            "cases": out,
            "overhead_ones_vs_none": out["ones"]["ms_per_iteration"] / out["none"]["ms_per_iteration"] - 1.0}


def _largest_component(rp, ci):
    """CSR of the largest connected component (vertices renumbered in order)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    n = len(rp) - 1
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    _, lab = connected_components(A, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    sub = A[keep][:, keep].tocsr()
    sub.sort_indices()
    return sub.indptr.astype(np.int32), sub.indices.astype(np.int32), keep


def run_scale(args, local_rank):
    """The method at scale: Barabasi-Albert n = 200,000 (m = 3), 2-D and 3-D,
    200 iterations of Algorithm 2 at omega = 0.5 (classical 1.5).  Reports
    throughput, the L^W passes' streaming rate against HBM (the 20 GB of
    distance codes do not fit in L2), and the error against the FP64 oracle
    on sampled vertices (distance rows, force rows at X^0)."""
    import torch

    import oracle
    from paper_1711_01228_gb300 import api

    rp, ci = synth.workload("ba200k")
    n = len(rp) - 1
    peaks, _ = _peaks()
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 14, replace=False)]))
    out = {"workload": f"Barabasi-Albert n={n}, m=3 ({int(rp[-1]) // 2} edges), X0 U[0,1]^d seed 0, "
                       "200 iterations at omega_c 1.5 (tolerance 0)", "dims": {}}
    for dim in (2, 3):
        X0 = synth.initial_layout(n, dim, 0)
        with api.Layout(rp, ci, dim=dim) as L:
            info = L.info()
            F = L.forces(X0).astype(np.float64)[rows]
            Xd = torch.from_numpy(X0).cuda()
            r = L.run(Xd, omega=0.5, tol=0.0, max_iter=200)
            st = r.stats
        Fr = []
        for i in rows:
            d = oracle.bfs_row(rp, ci, int(i)).astype(np.float64)
            Fr.append(oracle.force_row(X0, int(i), d))
        Fr = np.stack(Fr)
        pairs = st["pairs"]
        code_bytes = info["distance_bytes"]
        out["dims"][str(dim)] = {
            "distance_bytes": code_bytes, "apsp_ms": info["apsp_ms"], "iterations": st["iterations"],
            "cg_steps": st["cg_steps"], "kernel_ms": st["kernel_ms"],
            "pair_interactions_per_s": st["pair_passes"] * pairs / (st["kernel_ms"] / 1e3),
            "fp32_tflops": pairs * (st["matvec_passes"] * FLOP_MV[dim] + st["stress_passes"] * FLOP_K2[dim])
            / (st["kernel_ms"] / 1e3) / 1e12,
            "code_stream_gbs": (st["matvec_passes"] + st["stress_passes"] / 2.0) * code_bytes / (st["kernel_ms"] / 1e3) / 1e9,
            "hbm_peak_gbs": peaks.get("hbm_gbs", 6800.0),
            "final_stress": r.stress,
            "force_rel_err_sampled": float(np.linalg.norm(F - Fr) / np.linalg.norm(Fr)),
            "sampled_vertices": int(len(rows)),
        }
    out["note"] = ("code_stream_gbs counts one read of the distance codes per pass (two-candidate passes read "
                   "them once for both candidates); force error is Frobenius over the sampled rows, FP32 vs "
                   "the FP64 oracle")
    return out


TABLE1_AVG = {"iters": {"0": 100.0, "0.5": 67.5, "1.0": 50.4, "1.5": 44.9, "auto": 47.2, "enum": 41.8},
              "time": {"0": 100.0, "0.5": 100.1, "1.0": 74.8, "1.5": 66.7, "auto": 70.2, "enum": 140.9}}


def best_omega_stats(traces):
    """The two observations of Sec. 5.2.2 on the enumerated best omega of
    every iteration: the share of iterations whose best omega lies in
    [0.5, 2], and the zigzag: among the moves of the best omega, the share
    of turning points (the move reverses the previous one; an independent
    sequence gives 2/3), and the lag-1 autocorrelation of the moves
    (negative for a zigzag; -1/2 for an independent sequence's increments)."""
    inside, turns, moves, ac = [], 0, 0, []
    for om in traces:
        if len(om) == 0:
            continue
        inside.append(float(np.mean((om >= 0.5) & (om <= 2.0))))
        d = np.diff(om)
        d = d[d != 0.0]
        if len(d) >= 2:
            turns += int(np.sum(np.sign(d[1:]) != np.sign(d[:-1])))
            moves += len(d) - 1
            if np.std(d[1:]) > 0 and np.std(d[:-1]) > 0:
                ac.append(float(np.corrcoef(d[:-1], d[1:])[0, 1]))
    return {"in_0.5_2": float(np.mean(inside)) if inside else float("nan"),
            "turning_points": turns / moves if moves else float("nan"),
            "lag1_autocorr": float(np.mean(ac)) if ac else float("nan")}


def run_table1(args, local_rank):
    """Iterations and device time of every omega strategy of Sec. 5.2 on
    synthetic stand-ins at the sizes of Table 1 (band-46 ... net-2305), with
    the table's relative-error tolerances (stress decrease), averaged over
    seeded initial layouts; ratios against omega = 0 beside the table's
    average row."""
    from paper_1711_01228_gb300 import api

    cases = [("rgg46", 46, 1e-6), ("rgg62", 62, 1e-6), ("rgg86", 86, 1e-6), ("rgg156", 156, 1e-5),
             ("rgg303", 303, 1e-5), ("rgg516", 516, 1e-5), ("grid33x34", 1122, 1e-4), ("grid34x34", 1156, 1e-4),
             ("ba2305", 2305, 1e-4)]
    strategies = [("0", dict(omega=0.0)), ("0.5", dict(omega=0.5)), ("1.0", dict(omega=1.0)),
                  ("1.5", dict(omega=1.5)), ("auto", dict(strategy=api.OMEGA_PROB)),
                  ("enum", dict(strategy=api.OMEGA_ENUM))]
    out = {}
    for name, n, tol in cases:
        if name.startswith("rgg"):
            rp, ci, _ = synth.random_geometric(n, 2, 6.0, seed=1)
        elif name.startswith("grid"):
            a, b = (int(v) for v in name[4:].split("x"))
            rp, ci = synth.grid(a, b)
        else:
            rp, ci = synth.barabasi_albert(n, 3, seed=1)
        n = len(rp) - 1
        res = {}
        traces = []
        with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
            for key, kw in strategies:
                its, ms = [], []
                for seed in range(args.table1_seeds):
                    X = synth.initial_layout(n, 2, seed)
                    r = L.run(X, tol=tol, max_iter=5000, stop=api.STOP_REL_STRESS, seed=seed, trace=(key == "enum"),
                              **kw)
                    its.append(r.iterations)
                    ms.append(r.stats["kernel_ms"])
                    if key == "enum":
                        traces.append(np.asarray(r.omega, dtype=np.float64))
                res[key] = {"iterations": float(np.mean(its)), "ms": float(np.mean(ms))}
        out[name] = {"n": n, "tol": tol, "strategies": res, "enum_best_omega": best_omega_stats(traces)}
    ratio = {k: float(np.mean([100.0 * v["strategies"][k]["iterations"] / v["strategies"]["0"]["iterations"]
                               for v in out.values()])) for k, _ in strategies}
    tratio = {k: float(np.mean([100.0 * v["strategies"][k]["ms"] / v["strategies"]["0"]["ms"]
                                for v in out.values()])) for k, _ in strategies}
    zig = {k: float(np.mean([v["enum_best_omega"][k] for v in out.values()]))
           for k in ("in_0.5_2", "turning_points", "lag1_autocorr")}
    return {"table1_synthetic": out, "avg_iterations_pct_of_omega0": ratio, "avg_time_pct_of_omega0": tratio,
            "enum_best_omega_mean_over_cases": zig,
            "paper_table1_average_row": TABLE1_AVG,
            "note": "omega is the paper's (0 = Algorithm 1); auto = probabilistic strategy, enum = enumerating; "
                    "stop when the relative stress decrease falls below the tolerance; "
                    f"{args.table1_seeds} seeded X0 per case; synthetic graphs stand in for the paper's data sets"}


def cpu_sample(budget_s: float):
    """The oracle, as it is, on a bounded sample of the workload: one pass each
    of stress, L^X X and L^W p over all pairs of the Erdos-Renyi graph
    (distances from the oracle's BFS, not timed), repeated to ~budget_s."""
    import oracle

    rp, ci = synth.workload("er10k")
    n = len(rp) - 1
    X = synth.initial_layout(n, 2, 0).astype(np.float64)
    st, D = oracle.apsp(rp, ci, policy=1)
    pairs = n * (n - 1) / 2
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.stress(X, D)
        oracle.rhs(X, D)
        oracle.lw_matvec(X, D)
        done += 3
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return {"value": done * pairs / el, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle stress + L^X X + L^W p, {done} single-thread FP64 passes over the {int(pairs)} "
                      f"pairs of ER n=10,000 ({el:.1f} s)"}


def workload_config(args, inputs, world):
    """The bench line's config: the workload both arms are quoted on."""
    return {"workload": "+".join(args.workload.split(",")) + f" {args.dim}-D, X0 U[0,1]^{args.dim} seed 0, omega_c "
            + ("1.0-1.9 sweep" if args.sweep else "1.5") + ", rel-disp tol 1e-4, max 1000 iters",
            "graphs": {nm: {"n": len(rp) - 1, "m": int(rp[-1]) // 2} for nm, rp, _, _ in inputs},
            "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    """The oracle, as it is, on the host cores: each step a bounded sample of
    the workload (see cpu_sample), on the GPU arm's config and metric."""
    if rank != 0:
        return None
    for _ in range(args.warmup):
        cpu_sample(1.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_sample(3.0))
    el = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    return {"impl": "reference", "metric": "pair-interactions/s", "value": v, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, make_inputs(args.workload.split(","), args.dim), world),
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=",".join(WORKLOAD))
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--max-iter", type=int, default=1000, help="iteration cap per run (1000 = the workload)")
    ap.add_argument("--dim", type=int, default=2, choices=[1, 2, 3], help="layout dimension (2 = the workload)")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batched-form section")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-sample", type=int, default=64, help="graphs timed through the single-graph path")
    ap.add_argument("--no-grad", dest="grad", action="store_false", help="skip the differentiable-form section")
    ap.add_argument("--table1", action="store_true", help="omega strategies on stand-ins at Table 1's sizes, then exit")
    ap.add_argument("--scale", action="store_true", help="Barabasi-Albert n=200,000, 2-D and 3-D, 200 iterations, then exit")
    ap.add_argument("--table1-seeds", type=int, default=5)
    ap.add_argument("--grad-n", type=int, default=4096, help="vertices of the differentiable workload (<= 4096)")
    ap.add_argument("--no-direct", dest="direct_sec", action="store_false",
                    help="skip the direct-solver and per-vertex omega sections")
    ap.add_argument("--direct", action="store_true", help="only the direct-solver section, then exit")
    ap.add_argument("--direct-n", type=int, default=0, help="Delaunay graph size of --direct (0 = delaunay20k)")
    args = ap.parse_args()
    rank, world, local_rank = _env_rank()
    if args.scale:
        import torch

        from paper_1711_01228_gb300 import build

        build.build()
        torch.cuda.set_device(local_rank)
        if rank == 0:
            print(json.dumps(run_scale(args, local_rank)), flush=True)
        return
    if args.direct:
        import torch

        from paper_1711_01228_gb300 import api, build

        build.build()
        api.lib()
        torch.cuda.set_device(local_rank)
        if rank == 0:
            peaks, src = _peaks()
            sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
            fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            print(json.dumps(run_direct(args, local_rank, peaks, fp32_peak)), flush=True)
            if not args.direct_n:
                print(json.dumps(run_vertex_omega(args, local_rank)), flush=True)
        return
    if args.table1:
        import torch

        from paper_1711_01228_gb300 import build

        build.build()
        torch.cuda.set_device(local_rank)
        if rank == 0:
            print(json.dumps(run_table1(args, local_rank)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_sample(10.0)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
