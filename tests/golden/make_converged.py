"""Writes tests/golden/converged_runs.json: converged runs of Algorithm 2
(Sec. 3, Eq. (10); fixed-omega strategy of Sec. 5.2.1) computed by the FP64
oracle alone, for the converged-run parity tests of the CUDA path.

Cases (2-D, X^0 = synth.initial_layout(n, 2, seed 0), i.e. uniform in the unit
square as in Sec. 5.1; relative displacement 1e-4; at most 1000 iterations;
unreachable pairs at (largest finite d) + 1):

* three families of the benchmark's graphs at a size the dense oracle
  handles: Erdos-Renyi n = 2000 mean degree 6 (disconnected: 7 vertices
  outside the giant component), random binary tree n = 2047, Delaunay mesh of
  2000 uniform points; classical omega 1.0, 1.5, 1.9 (paper omega 0, 0.5, 0.9);
* eight graphs of the 4096-graph batched workload (every 512th by size),
  classical omega 1.5.

Run: python tests/golden/make_converged.py   (a few minutes on 8 cores).
Only oracle/ and the seeded generators are called; nothing here comes from
the CUDA path.
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "converged_runs.json")

FAMILIES = {
    "er2000": ("erdos_renyi", (2000, 6.0), {"seed": 0}),
    "tree2047": ("random_binary_tree", (2047,), {"seed": 0}),
    "delaunay2000": ("delaunay", (2000,), {"seed": 0}),
}
OMEGAS = (0.0, 0.5, 0.9)
TOL, MAX_ITER, NTRACE = 1e-4, 1000, 20
BATCH_GRAPHS, BATCH_STRIDE, BATCH_PICK = 4096, 512, 8


def family_graph(name):
    from paper_1711_01228_gb300 import synth

    fn, a, kw = FAMILIES[name]
    return getattr(synth, fn)(*a, **kw)


def batch_pick():
    """Indices (into synth.batch_graphs(4096)) of every 512th graph by size."""
    import numpy as np

    from paper_1711_01228_gb300 import synth

    sizes = synth.batch_sizes(BATCH_GRAPHS, seed=0)
    order = np.argsort(-sizes, kind="stable")
    return [int(g) for g in order[::BATCH_STRIDE][:BATCH_PICK]]


def batch_graph(g):
    from paper_1711_01228_gb300 import synth

    return synth.batch_graphs(BATCH_GRAPHS, seed=0)[g]


def _case(task):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle
    from paper_1711_01228_gb300 import synth

    kind, key, omega = task
    if kind == "family":
        rp, ci = family_graph(key)
        n = len(rp) - 1
        X0 = synth.initial_layout(n, 2, 0)
    else:
        rp, ci = batch_graph(key)
        n = len(rp) - 1
        sizes = synth.batch_sizes(BATCH_GRAPHS, seed=0)
        gp = np.concatenate([[0], np.cumsum(sizes)])
        X0 = synth.batch_initial_layout(sizes, 2, seed=0)[gp[key]:gp[key + 1]]
    st, D = oracle.apsp(rp, ci, policy=1)
    r = oracle.sor_run(D, X0.astype(np.float64), omega=omega, tol=TOL, max_iter=MAX_ITER)
    return {"kind": kind, "key": key, "n": n, "omega": omega, "iterations": r.iterations,
            "converged": bool(r.converged), "stress": r.stress, "accept": [bool(a) for a in r.trace_accept[:NTRACE]],
            "trace_f": [float(f) for f in r.trace_f[:NTRACE + 1]], "crit_last": float(r.trace_crit[-1]),
            "disconnected": bool(_disconnected(rp, ci))}


def _disconnected(rp, ci):
    import numpy as np
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    n = len(rp) - 1
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    return connected_components(A, directed=False)[0] > 1


def main():
    import multiprocessing as mp

    sys.path.insert(0, ROOT)
    tasks = [("family", name, om) for name in FAMILIES for om in OMEGAS]
    tasks += [("batch", g, 0.5) for g in batch_pick()]
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 4)) as pool:
        res = pool.map(_case, tasks, chunksize=1)
    doc = {"about": "converged runs of Algorithm 2 by the FP64 oracle (tests/golden/make_converged.py); "
                    "2-D, X0 seed 0, relative displacement 1e-4, max 1000 iterations, policy 1",
           "tol": TOL, "max_iter": MAX_ITER, "cases": res}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    for c in res:
        print(c["kind"], c["key"], c["n"], c["omega"], c["iterations"], c["converged"], c["stress"])


if __name__ == "__main__":
    main()
