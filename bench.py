#!/usr/bin/env python3
"""Benchmark of the SOR stress-majorization layout path on GB300.

Headline workload (the largest single-GPU configuration): a Barabasi-Albert
graph, n = 200,000, m = 3 (about 6e5 edges), laid out in 2-D and in 3-D,
X^0 uniform in the unit square / cube (seed 0), 200 iterations of
Algorithm 2 at omega = 0.5 (classical 1.5).  Its distance codes take 20 GB
per layout, far more than the 129 MB L2, so every all-pairs pass streams them
from HBM (no L2 flush is needed between steps).

One step is ITERS_PER_STEP (10) iterations of each layout, continuing the
trajectory of the step before (fd_run resumed with first_iter), so that the
default 20 timed steps are exactly the configuration's 200 iterations.  The
ideal distances (multi-source BFS over the CSR) are computed once per layout
before the steps and reported beside them (``apsp``); the end-to-end figure
(``e2e``) includes them.

Metric: unordered pair interactions per second (every all-pairs pass counts
n(n-1)/2 pairs: each L^W matvec, and each stress/RHS evaluation of a
candidate layout); SOR iterations per second beside it.

Sections run once after the timed steps: the benchmark-set stand-ins (ER
n=10,000, Delaunay n=20,000, random binary tree n=16,383) at classical omega
1.0 ... 1.9, the batched form (4096 graphs), the differentiable form, the
direct solver and per-vertex omega; every result carries its error against
the FP64 oracle where the oracle can compute it.
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

WORKLOAD = ("er10k", "delaunay20k", "tree16k")   # benchmark-set stand-ins (sweep section)
HEADLINE = "ba200k"                               # Barabasi-Albert n=200,000, m=3
HEADLINE_DIMS = (2, 3)
HEADLINE_ITERS = 200
ITERS_PER_STEP = 10
FLOP_K2 = {1: 13, 2: 19, 3: 25}   # stress + L^X X per unordered pair per candidate
FLOP_MV = {1: 4, 2: 8, 3: 12}     # L^W p per unordered pair
FLOP_RHS = {1: 4, 2: 8, 3: 12}    # the L^X X part of FLOP_K2 (both endpoints), absent where a candidate's RHS is skipped
# enumerating strategy (stress only): per candidate Delta = Delta_z + omega (Delta_z - Delta_x) 2d, r^2 2d,
# r/d - 1 3, square-accumulate 2; per pair once Delta_z, Delta_x and their difference 3d
FLOP_ENUM_CAND = {1: 9, 2: 13, 3: 17}
FLOP_ENUM_SHARED = {1: 3, 2: 6, 3: 9}
NENUM = 19


def algorithmic_flops(st: dict, dim: int) -> float:
    """Algorithmic FP32 FLOPs of a layout-kernel call from its fd_stats: L^W
    passes, stress/RHS passes per candidate, and the enumeration passes'
    candidate stresses at their own (stress-only) cost; rsqrt not counted."""
    en = st.get("enum_candidate_passes", 0.0)
    return st["pairs"] * (st["matvec_passes"] * FLOP_MV[dim] + st["stress_passes"] * FLOP_K2[dim]
                          - st.get("rhs_skipped", 0.0) * FLOP_RHS[dim]
                          + en * FLOP_ENUM_CAND[dim] + en / NENUM * FLOP_ENUM_SHARED[dim])


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


def fp32_peak_tflops(dev):
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flop x the measured maximum SM clock."""
    import torch

    peaks, src = _peaks()
    clk = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * clk * 1e6 / 1e12, sms, clk, src


TAG_NAMES = {4: "rhs0", 5: "lw_x0", 6: "lw_u0", 7: "lw_cg", 8: "candidates", 9: "vertex_phase", 10: "dense_apply",
             11: "rhs_z", 12: "cg_last"}


def pass_profile(L, X, dim, iters, opts, code_bytes_total, pairs, fp32_peak, hbm_peak):
    """Per-pass roofline of the layout kernel from its %globaltimer marks:
    one extra run of `iters` iterations from X (a copy) with the timeline on.
    A pass's duration runs from the mark before it to its own mark (grid
    barrier included).  Candidate passes (both candidates' stresses, the
    extrapolated one's L^X X) are rated against the FP32 peak; L^W passes
    against the HBM copy bandwidth (their 1-byte codes) and the FP32 peak;
    rhs_z is the right-hand-side pass of a kept first candidate, cg_last the
    pass-less last CG update."""
    import ctypes

    from paper_1711_01228_gb300 import api

    cap = 200000
    api.lib().fd_timeline_enable(L._h, cap)
    Xc = X.clone()
    L.run(Xc, max_iter=iters, **opts)
    skipped = L.stats().get("rhs_skipped", 0.0)
    buf = np.zeros(2 * cap)
    cnt = ctypes.c_int32()
    api.lib().fd_timeline_read(L._h, buf.ctypes.data, cap, ctypes.byref(cnt))
    api.lib().fd_timeline_enable(L._h, 0)
    tl = buf[:2 * cnt.value].reshape(-1, 2)
    dur = {}
    for (t0, a), (tag, b) in zip(tl[:-1], tl[1:]):
        dur.setdefault(int(tag), []).append((b - a) * 1e-9)
    out = {}
    for tag, ds in sorted(dur.items()):
        name = TAG_NAMES.get(tag, str(tag))
        mean_s = float(np.mean(ds))
        e = {"count": len(ds), "mean_us": mean_s * 1e6, "total_ms": float(np.sum(ds)) * 1e3}
        if tag in (5, 6, 7):
            e["flop_per_pair"] = FLOP_MV[dim]
            e["achieved_tflops"] = pairs * FLOP_MV[dim] / mean_s / 1e12
            e["frac_fp32"] = e["achieved_tflops"] / fp32_peak
            e["code_gbs"] = code_bytes_total / mean_s / 1e9
            e["frac_hbm"] = e["code_gbs"] / hbm_peak
        elif tag == 8:
            # both candidates' stress, the right-hand side of the second (and of the
            # first where the pass computed it)
            fpp = 2 * FLOP_K2[dim] - FLOP_RHS[dim] * min(1.0, skipped / max(len(ds), 1))
            e["flop_per_pair"] = fpp
            e["achieved_tflops"] = pairs * fpp / mean_s / 1e12
            e["frac_fp32"] = e["achieved_tflops"] / fp32_peak
            e["code_gbs"] = code_bytes_total / mean_s / 1e9
            e["frac_hbm"] = e["code_gbs"] / hbm_peak
        out[name] = e
    return out


def sampled_force_error(L_forces, X, rp, ci, rows, fill=-1.0):
    """Largest |F_ic - F_ic^oracle| / A_ic over sampled rows (A_ic: the
    magnitude of the row's terms, oracle.force_row_abs) and the Frobenius
    relative error over the sample."""
    import oracle

    F = np.asarray(L_forces, dtype=np.float64)
    Xd = np.asarray(X, dtype=np.float64)
    worst, num, den = 0.0, 0.0, 0.0
    for k, i in enumerate(rows):
        d = oracle.bfs_row(rp, ci, int(i)).astype(np.float64)
        if fill > 0:
            d[d < 0] = fill
        ref = oracle.force_row(Xd, int(i), d)
        A = oracle.force_row_abs(Xd, int(i), d)
        err = np.abs(F[k] - ref)
        worst = max(worst, float(np.max(err / np.maximum(A, 1e-300))))
        num += float(np.sum(err ** 2))
        den += float(np.sum(ref ** 2))
    return {"max_elem_err_over_row_magnitude": worst, "frobenius_rel": (num / den) ** 0.5 if den > 0 else 0.0,
            "rows": int(len(rows))}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1711_01228_gb300 import api, build

    build.build()
    api.lib()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    dims = tuple(int(d) for d in args.dims.split(","))
    rp, ci = synth.workload(args.headline)
    n = len(rp) - 1
    x0 = {d: synth.initial_layout(n, d, 0) for d in dims}
    rpd, cid = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    x0d = {d: torch.from_numpy(x0[d]).to(dev) for d in dims}
    opts = dict(omega=0.5, tol=0.0, stop=api.STOP_REL_DISP)
    ips = args.iters_per_step
    # row a0: ideal distances, once per layout (CUDA events inside fd_layout_create)
    layouts = {d: api.Layout(rpd, cid, dim=d, disconnected_policy=1, stream=stream.cuda_stream) for d in dims}
    info = {d: layouts[d].info() for d in dims}

    def zero():
        return dict(pairs=0.0, iters=0, kernel_ms=0.0, flops=0.0, cg=0, mv=0.0, st=0.0, launches=0, h2d=0, d2h=0)

    def step(acc, X, s, host=False, Ls=None):
        Ls = Ls or layouts
        for d in dims:
            r = Ls[d].run(X[d], max_iter=ips, first_iter=s * ips, **opts)
            st = r.stats
            acc["pairs"] += st["pair_passes"] * st["pairs"]
            acc["iters"] += st["iterations"]
            acc["kernel_ms"] += st["kernel_ms"]
            acc["flops"] += algorithmic_flops(st, d)
            acc["cg"] += st["cg_steps"]
            acc["mv"] += st["matvec_passes"]
            acc["st"] += st["stress_passes"]
            acc["launches"] += 1
            acc["last_stress_" + str(d)] = r.stress
            if host:
                acc["h2d"] += X[d].numel() * 4
                acc["d2h"] += X[d].numel() * 4 + 8

    Xw = {d: x0d[d].clone() for d in dims}
    for s_ in range(args.warmup):
        step(zero(), Xw, s_)
    del Xw
    torch.cuda.synchronize()
    # ----- device-resident timed region: the inputs (CSR, X0) and the 20 GB of
    # distance codes per layout are in HBM; the codes exceed L2, so no flush
    sampler = ClockSampler(local_rank)
    acc = zero()
    X = {d: x0d[d].clone() for d in dims}
    times = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for s_ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(acc, X, s_)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = sum(times)
    fp32_peak, sms, clk, src = fp32_peak_tflops(dev)
    peaks, _ = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # ----- per-pass roofline (timeline of one extra chunk, outside the timed steps)
    passes = {}
    for d in dims:
        passes[str(d)] = pass_profile(layouts[d], X[d], d, ips, opts, info[d]["distance_bytes"], 0.5 * n * (n - 1),
                                      fp32_peak, hbm)
    # ----- error against the FP64 oracle: sampled force rows at X0 and at the final layout
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 14, replace=False)]))
    runs = []
    Xf = {d: X[d].cpu().numpy() for d in dims}
    for d in dims:
        F0 = layouts[d].forces(x0[d])[rows]
        Ff = layouts[d].forces(Xf[d])[rows]
        runs.append({"graph": args.headline, "n": n, "m": int(rp[-1]) // 2, "dim": d, "omega_c": 1.5,
                     "iterations": args.steps * ips, "final_stress": acc["last_stress_" + str(d)],
                     "error_vs_oracle": {"forces_at_x0": sampled_force_error(F0, x0[d], rp, ci, rows),
                                         "forces_at_final": sampled_force_error(Ff, Xf[d], rp, ci, rows)}})
    apsp = {d: info[d]["apsp_ms"] for d in dims}
    # a pass over the edge list with W-bit source words: row_ptr (4 B), the
    # reached word (read), the next word (written) per vertex; col_idx (4 B)
    # and the neighbour's frontier word per edge
    wb = {d: max(info[d]["bfs_sources"], 64) / 8.0 for d in dims}
    apsp_bytes = {d: info[d]["bfs_sweeps"] * ((4.0 + 2.0 * wb[d]) * n + (4.0 + wb[d]) * int(rp[-1]))
                  + 0.5 * n * (n - 1) for d in dims}
    apsp_kernel = {d: "bfs_wide_kernel" if info[d]["bfs_sources"] == 256 else "bfs_batch_kernel" for d in dims}
    for L in layouts.values():
        L.close()
    del layouts
    torch.cuda.synchronize()
    # ----- end to end through the public API with host buffers: the handles are
    # made from the host CSR (distances included), and every step copies the
    # layouts in from pinned host memory and out again
    acc_e = zero()
    e2e_ms = 0.0
    if not args.no_e2e:
        Xh = {d: torch.from_numpy(x0[d]).pin_memory() for d in dims}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ls = {d: api.Layout(rp, ci, dim=d, disconnected_policy=1) for d in dims}
        acc_e["h2d"] += rp.nbytes + ci.nbytes
        for s_ in range(args.steps):
            step(acc_e, Xh, s_, host=True, Ls=Ls)
        torch.cuda.synchronize()
        e2e_ms = max((time.perf_counter() - t0) * 1e3, 1e-9)
        for L in Ls.values():
            L.close()
        del Ls
    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], dev, world)
    value = job_rate(acc["pairs"], world, total_ms)
    e2e_value = job_rate(acc_e["pairs"], world, e2e_ms) if e2e_ms > 1e-6 else None
    fp32_measured = {"fma_f32": api.fp32_peak(False), "fma_f32x2": api.fp32_peak(True)}
    achieved = acc["flops"] / (acc["kernel_ms"] / 1e3) / 1e12
    # the final stress of every layout against the oracle's Eq. (1) over all pairs
    if rank == 0 and not args.no_oracle_check:
        import oracle

        t0 = time.perf_counter()
        f_ref = oracle.stress_stream_multi([Xf[d] for d in dims], rp, ci, workers=max(1, (os.cpu_count() or 2) - 1))
        for r_, fr in zip(runs, f_ref):
            r_["error_vs_oracle"]["final_stress_rel"] = abs(r_["final_stress"] - fr) / abs(fr)
            r_["error_vs_oracle"]["oracle_final_stress"] = float(fr)
            r_["error_vs_oracle"]["oracle_s"] = time.perf_counter() - t0
    sweep = run_sweep(args, local_rank, fp32_peak) if (args.sweep_sec and rank == 0) else None
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
        "config": headline_config(args, n, int(rp[-1]) // 2, world),
        "sor_iterations_per_s": acc["iters"] * world / (total_ms / 1e3),
        "cg_steps_per_sor_iteration": acc["cg"] / max(acc["iters"], 1),
        "gpu_launches": acc["launches"],
        "roofline": {"bound": "alu", "kernel": "fd_main_kernel", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": measured_traffic(args.headline),
                     "traffic_unit": "DRAM bytes per launch (ncu, read + write)",
                     "peak_note": f"FP32 CUDA cores {sms} SMs x 128 x 2 flop at {clk:.0f} MHz ({src} max clock)",
                     "peak_measured_tflops": fp32_measured,
                     "peak_measured_note": "fd_fp32_peak: 16 independent FMA chains per thread, scalar and "
                                           "two-wide packed, best of 5 launches",
                     "algorithmic_flops_note": "per unordered pair: L^W p 8 (2-D) / 12 (3-D); stress + L^X X "
                                               "per candidate 19 (2-D) / 25 (3-D); rsqrt not counted",
                     "passes": passes},
        "apsp": {"kernel": apsp_kernel, "ms": apsp, "sources_per_search": {d: info[d]["bfs_sources"] for d in dims},
                 "algorithmic_bytes": apsp_bytes,
                 "achieved_gbs": {d: apsp_bytes[d] / (apsp[d] / 1e3) / 1e9 for d in dims},
                 "peak_gbs": hbm,
                 "frac": {d: apsp_bytes[d] / (apsp[d] / 1e3) / 1e9 / hbm for d in dims},
                 "note": "once per layout before the timed steps; bytes a pass over the edge list must move per "
                         "multi-source search (row_ptr, reached and next words, col_idx, neighbour frontier words) "
                         "times the passes run, plus 1 B per pair written; for bfs_wide_kernel (256 sources "
                         "per search, all CTAs, a grid barrier per level) the words are L2-resident and the "
                         "kernel is bound by the per-level latency, not by these bytes"},
        "layout_kernel_ms_per_step": acc["kernel_ms"] / args.steps,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": acc_e["h2d"] // max(args.steps, 1),
                "d2h_bytes_per_step": acc_e["d2h"] // max(args.steps, 1),
                "note": "fd_layout_create from the host CSR (distances included) + every step's fd_run on pinned "
                        "host layouts, wall clock"},
        "runs": runs,
    }
    for k, v in (("sweep", sweep), ("batched", batched), ("differentiable", differentiable),
                 ("direct_solver", direct), ("vertex_omega", vertex_omega)):
        if v is not None:
            line[k] = v
    return line


def run_sweep(args, local_rank, fp32_peak):
    """The benchmark-set stand-ins (ER n=10,000 mean degree 6, Delaunay
    n=20,000, random binary tree n=16,383; 2-D, X0 seed 0) run to convergence
    (relative displacement 1e-4, at most 1000 iterations) at classical omega
    1.0 ... 1.9, L2 flushed before each run.  Error against the oracle at
    omega_c 1.5: final stress (Eq. (1) streamed over all pairs) and sampled
    force rows at X0 and at the final layout.  Iteration counts against the
    oracle's: the stand-ins at n ~ 2000 (tests/golden/converged_runs.json,
    written by the oracle alone) laid out by the GPU with the same options."""
    import json as _json

    import torch

    import oracle
    from paper_1711_01228_gb300 import api

    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    oms = omegas(True) if not args.sweep_quick else [0.0, 0.5, 0.9]
    out = {"workload": "er10k + delaunay20k + tree16k, 2-D, X0 U[0,1]^2 seed 0, rel-disp tol 1e-4, max "
                       f"{args.max_iter} iterations, unreachable pairs at (largest d) + 1; L2 flushed before each run",
           "graphs": {}}
    tot_pairs, tot_ms, tot_flops = 0.0, 0.0, 0.0
    for nm in WORKLOAD:
        rp, ci = synth.workload(nm)
        n = len(rp) - 1
        x0 = synth.initial_layout(n, 2, 0)
        X0 = torch.from_numpy(x0).to(dev)
        g = {"n": n, "m": int(rp[-1]) // 2, "runs": []}
        with api.Layout(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), dim=2, disconnected_policy=1,
                        stream=stream.cuda_stream) as L:
            g["diameter"] = L.info()["diameter"]
            g["disconnected"] = bool(L.info()["disconnected"])
            fill = float(g["diameter"] + 1) if g["disconnected"] else -1.0
            for om in oms:
                flush.fill_(1.0)
                torch.cuda.synchronize()
                X = X0.clone()
                r = L.run(X, omega=om, tol=1e-4, max_iter=args.max_iter, stop=api.STOP_REL_DISP)
                st = r.stats
                tot_pairs += st["pair_passes"] * st["pairs"]
                tot_ms += st["kernel_ms"]
                tot_flops += algorithmic_flops(st, 2)
                e = {"omega_c": round(1.0 + om, 1), "iterations": r.iterations, "cg_steps": st["cg_steps"],
                     "final_stress": r.stress, "final_crit": st["final_crit"], "kernel_ms": st["kernel_ms"],
                     "pairs_per_s": st["pair_passes"] * st["pairs"] / (st["kernel_ms"] / 1e3)}
                if abs(om - 0.5) < 1e-9 and not args.no_oracle_check:
                    rng = np.random.default_rng(11)
                    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 14, replace=False)]))
                    xf = X.cpu().numpy()
                    fr = oracle.stress_stream(xf, rp, ci, fill, workers=max(1, (os.cpu_count() or 2) - 1))
                    e["error_vs_oracle"] = {
                        "final_stress_rel": abs(r.stress - fr) / abs(fr), "oracle_final_stress": fr,
                        "forces_at_x0": sampled_force_error(L.forces(x0)[rows], x0, rp, ci, rows, fill),
                        "forces_at_final": sampled_force_error(L.forces(xf)[rows], xf, rp, ci, rows, fill)}
                g["runs"].append(e)
        out["graphs"][nm] = g
    out["pairs_per_s"] = tot_pairs / (tot_ms / 1e3)
    out["fp32_frac"] = tot_flops / (tot_ms / 1e3) / 1e12 / fp32_peak
    # iteration counts against the oracle's on the n ~ 2000 stand-ins of each family
    gpath = os.path.join(ROOT, "tests", "golden", "converged_runs.json")
    if os.path.exists(gpath):
        import importlib.util

        spec = importlib.util.spec_from_file_location("make_converged",
                                                      os.path.join(ROOT, "tests", "golden", "make_converged.py"))
        mk = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mk)
        with open(gpath) as f:
            gold = _json.load(f)
        cmp_ = []
        for c in gold["cases"]:
            if c["kind"] != "family":
                continue
            rp, ci = mk.family_graph(c["key"])
            with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
                X = synth.initial_layout(c["n"], 2, 0)
                r = L.run(X, omega=c["omega"], tol=gold["tol"], max_iter=gold["max_iter"], stop=api.STOP_REL_DISP)
            cmp_.append({"graph": c["key"], "n": c["n"], "omega_c": round(1.0 + c["omega"], 1),
                         "gpu_iterations": r.iterations, "oracle_iterations": c["iterations"],
                         "gpu_stress": r.stress, "oracle_stress": c["stress"],
                         "stress_rel": abs(r.stress - c["stress"]) / c["stress"],
                         "both_capped_or_both_converged": (r.iterations < gold["max_iter"]) == c["converged"]})
        out["oracle_iterations_n2000"] = cmp_
    return out


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
    tiles = B.tiles()
    st = res.stats
    it = res.iterations
    pairs_s = st["pairs"] / (ms / 1e3)
    flops = 0.0
    for g in range(G):
        pg = 0.5 * sizes[g] * (sizes[g] - 1)
        # one two-candidate pass per iteration (omega != 0), without the first candidate's RHS
        flops += pg * (res.matvec_passes[g] * FLOP_MV[2] + res.stress_passes[g] * FLOP_K2[2]
                       - it[g] * FLOP_RHS[2])
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
        "launch": {"kernel": "fd_batch_kernel", "grid": info["grid"], "units_per_cta": groups, "stages": stages,
                   "tuned": True, "cuda_graph": bool(info["graph_captured"]),
                   "launches_per_run": "one CUDA graph: one persistent launch per tile edge (128, 64, 32)",
                   "tile_edge_by_bucket": dict(zip(["n<=32", "n<=64", "n<=128", "n<=256", "n<=512", "n<=1024",
                                                    "n<=2048"], tiles)),
                   "graphs_by_tile_edge": {"128": info["graphs_t128"], "64": info["graphs_t64"],
                                           "32": info["graphs_t32"]},
                   "tuner": "fd_batch_tune: launch shape (units x stages), then per size bucket the tile edge "
                            "in {128, 64, 32} (each bucket's graphs alone, 5 iterations, best of 2)"},
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


def run_batch_tiles(args, local_rank, peak_tflops):
    """The batched workload at every fixed tile edge (128, 64, 32 for all size
    buckets, launch shape 2 units x 2 stages) and with the autotuner's choice:
    per case the kernel's CUDA-event time (one warm-up run, L2 flushed before
    the timed run), pair interactions/s, the FP32 fraction, and per size bucket
    the device time per all-pairs pass and the share of all CTA time."""
    import torch

    from paper_1711_01228_gb300 import api

    dev = torch.device("cuda", local_rank)
    G = args.batch_graphs
    graphs = synth.batch_graphs(G, seed=0)
    sizes = np.array([len(rp) - 1 for rp, _ in graphs])
    X0 = synth.batch_initial_layout(sizes, 2, seed=0)
    stream = torch.cuda.Stream(dev)
    opts = dict(omega=0.5, tol=1e-4, max_iter=args.max_iter, stop=api.STOP_REL_DISP)
    Xd = torch.from_numpy(X0).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    buckets = [(0, 32), (32, 64), (64, 128), (128, 256), (256, 512), (512, 1024), (1024, 2048)]
    api.batch_clear_tile_cache()
    B = api.Batch.from_graphs(graphs, dim=2, disconnected_policy=1, stream=stream.cuda_stream)
    cases = []

    def measure(label):
        X = Xd.clone()
        B.run(X, **opts)
        X = Xd.clone()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        res = B.run(X, **opts)
        ms = res.stats["kernel_ms"]
        flops = float(np.sum(0.5 * sizes * (sizes - 1) * (res.matvec_passes * FLOP_MV[2]
                                                          + res.stress_passes * FLOP_K2[2]
                                                          - res.iterations * FLOP_RHS[2])))
        info = B.info()
        tot = float(res.graph_ms.sum())
        per = {}
        for lo, hi in buckets:
            m = (sizes > lo) & (sizes <= hi)
            npass = float((res.matvec_passes[m] + res.stress_passes[m]).sum())
            per[f"n<={hi}"] = {"graphs": int(m.sum()), "us_per_pass": 1e3 * float(res.graph_ms[m].sum()) / max(npass, 1.0),
                              "cta_time_share": float(res.graph_ms[m].sum()) / tot}
        cases.append({"tiles": label, "tile_edge_by_bucket": B.tiles(), "units_per_cta": info["groups"],
                      "stages": info["stages"], "kernel_ms": ms, "pairs_per_s": res.stats["pairs"] / (ms / 1e3),
                      "fp32_frac": flops / (ms / 1e3) / 1e12 / peak_tflops, "buckets": per})

    with B:
        for T in (128, 64, 32):
            B.set_shape(2, 2)
            B.set_tiles([T] * api.BATCH_BUCKETS)
            measure(f"{T} everywhere")
        B.set_tiles([128] * api.BATCH_BUCKETS)
        B.tune(Xd, probe_iter=5, repeats=2, **opts)
        measure("tuned")
    return {"batch_tiles": {"workload": f"{G} graphs of the batched workload (synth.batch_graphs, seed 0), 2-D, "
                                        f"omega_c 1.5, rel-disp tol 1e-4, max {args.max_iter} iterations",
                            "cases": cases}}


def run_differentiable(args, local_rank):
    """The differentiable form on a random geometric graph of args.grad_n
    points in the unit cube (mean degree 6, seed 0; its largest component,
    since derivatives in the edge lengths need every pair connected) in 3-D,
    every edge length a float32 parameter initialised at 1.0.  Timed: the
    weighted shortest paths at creation, the stress pass, the position
    gradient (force pass), the length gradient (shortest-path back-
    propagation), one autograd.stress_lengths forward + backward, and
    unrolled_layout with K = 32 iterations of Algorithm 2 (checkpoint every
    8) forward and forward + backward.  Then a few gradient steps fit the
    edge lengths so that X^K's distances on 4096 sampled pairs match seeded
    target distances (a random layout's), loss before and after."""
    import torch

    from paper_1711_01228_gb300 import api, autograd

    dev = torch.device("cuda", local_rank)
    rp0, ci0, pts0 = synth.random_geometric(args.grad_n, 3, 6.0, seed=0)
    rp, ci, keep = _largest_component(rp0, ci0)
    n = len(rp) - 1
    w = np.ones(len(ci), dtype=np.float32)
    X = torch.from_numpy(synth.initial_layout(n, 3, 0) * 10.0).to(dev)
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

    t0 = time.perf_counter()
    L = api.Layout(rp, ci, dim=3, edge_len=w, disconnected_policy=0)
    create_s = time.perf_counter() - t0
    info = L.info()
    F = torch.empty_like(X)
    G = torch.empty(len(ci), dtype=torch.float32, device=dev)
    ms_energy = timed(lambda: L.energy(X))
    ms_forces = timed(lambda: L.forces(X, out=F))
    ms_lgrad = timed(lambda: L.length_grad(X, out=G), reps=1)
    L.close()

    def step():
        wt.grad = None
        f = autograd.stress_lengths(X, wt, rpt, cit)
        f.backward()

    ms_step = timed(step, reps=1)

    # adjoint through K = 32 unrolled iterations (checkpoint every 8): fit lengths to target distances
    K, every = 32, 8
    rng2 = np.random.default_rng(1)
    Yt = torch.from_numpy((rng2.random((n, 3)) * 10.0).astype(np.float32)).to(dev)
    pi = torch.from_numpy(rng2.integers(0, n, 4096)).to(dev)
    pj = torch.from_numpy(rng2.integers(0, n, 4096)).to(dev)
    ok = pi != pj
    pi, pj = pi[ok], pj[ok]
    tgt = (Yt[pi] - Yt[pj]).norm(dim=1)
    X0 = X.clone()

    def loss_of(lens):
        XK = autograd.unrolled_layout(X0, lens, rpt, cit, K=K, omega=0.5, every=every)
        return ((XK[pi] - XK[pj]).norm(dim=1) - tgt).pow(2).sum()

    def unrolled_step():
        wt.grad = None
        loss_of(wt).backward()

    def unrolled_forward():
        with torch.no_grad():
            autograd.unrolled_layout(X0, wt.detach(), rpt, cit, K=K, omega=0.5, every=every)

    ms_unrolled_fwd = timed(unrolled_forward, reps=1)
    ms_unrolled = timed(unrolled_step, reps=1)
    # the fit: Adam on the lengths (kept >= 0.05)
    lens = torch.ones(len(ci), dtype=torch.float32, device=dev, requires_grad=True)
    opt = torch.optim.Adam([lens], lr=0.05)
    losses = []
    t0 = time.perf_counter()
    for _ in range(args.grad_fit_steps + 1):
        opt.zero_grad()
        loss = loss_of(lens)
        losses.append(float(loss))
        if len(losses) > args.grad_fit_steps:
            break
        loss.backward()
        opt.step()
        with torch.no_grad():
            lens.clamp_(min=0.05)
    fit_s = time.perf_counter() - t0
    pairs = 0.5 * n * (n - 1)
    return {"workload": f"largest component (n={n}) of a random geometric graph of {args.grad_n} points in the "
                        "unit cube, mean degree 6 (seed 0); edge lengths float32 parameters at 1.0; 3-D, X0 "
                        "U[0,1]^3 x 10 seed 0",
            "n": n, "edges": int(len(ci)) // 2, "distance_bytes": info["distance_bytes"],
            "weighted_apsp_ms": info["apsp_ms"], "create_s": create_s,
            "stress_pass_ms": ms_energy, "position_grad_ms": ms_forces, "length_grad_ms": ms_lgrad,
            "autograd_step_ms": ms_step,
            "unrolled": {"iterations": K, "checkpoint_every": every, "omega_c": 1.5,
                         "forward_ms": ms_unrolled_fwd, "forward_backward_ms": ms_unrolled,
                         "loss": "squared error of 4096 sampled pair distances of X^K against a seeded "
                                 "random layout's"},
            "fit": {"optimizer": "Adam lr 0.05 on the edge lengths (>= 0.05)", "steps": args.grad_fit_steps,
                    "loss_before": losses[0], "loss_after": losses[-1], "losses": losses, "seconds": fit_s},
            "stress_pairs_per_s": pairs / (ms_energy / 1e3), "position_grad_pairs_per_s": pairs / (ms_forces / 1e3),
            "gradient_check": "FP64 finite differences and the oracle on 64-vertex subgraphs "
                              "(tests/test_gpu_grad.py), and the homogeneity identity at n ~ 5000",
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


_CPU_SAMPLE = {}


def cpu_sample(budget_s: float, headline: str = HEADLINE):
    """The oracle, as it is, on a bounded sample of the headline workload:
    its row functions L^X X and the force (L^X - L^W) X (single-thread FP64,
    explicit loops) on 32 sampled rows of the 2-D layout, the rows' BFS
    distances computed beforehand (not timed), repeated to ~budget_s.  A row
    call evaluates n - 1 ordered pairs, half of an all-pairs pass's n (n - 1)
    ordered pair evaluations per row share, so it counts (n - 1) / 2
    unordered pair interactions."""
    import oracle

    if _CPU_SAMPLE.get("headline") != headline:
        rp, ci = synth.workload(headline)
        n = len(rp) - 1
        rows = np.random.default_rng(3).choice(n, 32, replace=False)
        _CPU_SAMPLE.update(headline=headline, n=n, X=synth.initial_layout(n, 2, 0).astype(np.float64), rows=rows,
                           drows=[oracle.bfs_row(rp, ci, int(i)).astype(np.float64) for i in rows])
    n, X, rows, drows = (_CPU_SAMPLE[k] for k in ("n", "X", "rows", "drows"))
    calls, t0 = 0, time.perf_counter()
    while True:
        for i, d in zip(rows, drows):
            oracle.rhs_row(X, int(i), d)
            oracle.force_row(X, int(i), d)
            calls += 2
            if time.perf_counter() - t0 >= budget_s:
                break
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return {"value": calls * 0.5 * (n - 1) / el, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle rhs_row + force_row, {calls} single-thread FP64 row calls on 32 sampled rows of "
                      f"{headline} 2-D (n={n}; BFS rows precomputed, not timed) in {el:.1f} s; a row call counts "
                      "(n-1)/2 unordered pair interactions"}


def headline_config(args, n, m, world):
    """The bench line's config: the workload both arms are quoted on."""
    return {"workload": f"{args.headline}: Barabasi-Albert n={n} m=3 ({m} edges), "
                        + "+".join(f"{d}-D" for d in args.dims.split(","))
                        + f" layouts, X0 U[0,1]^d seed 0, omega_c 1.5, {args.iters_per_step} iterations of "
                          f"each layout per step ({args.steps} steps = {args.steps * args.iters_per_step} "
                          "iterations; the configuration is 200)",
            "l2": "inputs larger than L2 (20 GB of distance codes per layout, streamed every pass); no flush",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    """The oracle, as it is, on the host cores: each step a bounded sample of
    the headline workload (see cpu_sample), on the GPU arm's config and metric."""
    if rank != 0:
        return None
    for _ in range(args.warmup):
        cpu_sample(0.5, args.headline)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_sample(3.0, args.headline))
    el = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    rp, _ = synth.workload(args.headline)
    return {"impl": "reference", "metric": "pair-interactions/s", "value": v, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(args, len(rp) - 1, int(rp[-1]) // 2, world),
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--headline", default=HEADLINE, help="graph of the timed steps (synth.workload name)")
    ap.add_argument("--dims", default=",".join(str(d) for d in HEADLINE_DIMS), help="layout dimensions, e.g. 2,3")
    ap.add_argument("--iters-per-step", type=int, default=ITERS_PER_STEP)
    ap.add_argument("--no-sweep", dest="sweep_sec", action="store_false",
                    help="skip the benchmark-set stand-ins' omega sweep")
    ap.add_argument("--sweep-quick", action="store_true", help="sweep only classical omega 1.0, 1.5, 1.9")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's full-size stress evaluations (minutes of host time)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--max-iter", type=int, default=1000, help="iteration cap per run of the sweep (1000)")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batched-form section")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-sample", type=int, default=64, help="graphs timed through the single-graph path")
    ap.add_argument("--batch-tiles", action="store_true",
                    help="the batched workload at every fixed tile edge and tuned, then exit")
    ap.add_argument("--no-grad", dest="grad", action="store_false", help="skip the differentiable-form section")
    ap.add_argument("--table1", action="store_true", help="omega strategies on stand-ins at Table 1's sizes, then exit")
    ap.add_argument("--table1-seeds", type=int, default=5)
    ap.add_argument("--grad-n", type=int, default=50000, help="points of the differentiable workload's graph")
    ap.add_argument("--grad-fit-steps", type=int, default=3, help="gradient steps of the edge-length fit")
    ap.add_argument("--no-direct", dest="direct_sec", action="store_false",
                    help="skip the direct-solver and per-vertex omega sections")
    ap.add_argument("--direct", action="store_true", help="only the direct-solver section, then exit")
    ap.add_argument("--direct-n", type=int, default=0, help="Delaunay graph size of --direct (0 = delaunay20k)")
    args = ap.parse_args()
    rank, world, local_rank = _env_rank()
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
    if args.batch_tiles:
        import torch

        from paper_1711_01228_gb300 import build

        build.build()
        torch.cuda.set_device(local_rank)
        if rank == 0:
            peaks, src = _peaks()
            sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
            fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            print(json.dumps(run_batch_tiles(args, local_rank, fp32_peak)), flush=True)
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
            line["cpu_baseline"] = cpu_sample(10.0, args.headline)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
