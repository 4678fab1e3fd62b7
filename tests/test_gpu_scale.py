"""The method at scale: Barabasi-Albert graph n = 200,000, m = 3 (about 6e5
edges), 2-D and 3-D layouts, 200 iterations of Algorithm 2 at omega = 0.5
(classical 1.5).  The distance tiles take 20 GB; the FP64 oracle checks what it
can compute row by row: sampled distance rows (bit-exact), sampled force rows
element by element at X^0 and at the final layout (|F_ic - F_ic^oracle| <=
1e-5 A_ic, A_ic = sum_j |w_ij (d_ij/r_ij - 1)(x_ic - x_jc)|), the H-step
residual of Eq. (2-5) at sampled rows for the first three iterations, and the
final stress of both layouts against the oracle's Eq. (1) streamed over all
2e10 pairs (one BFS per row for both layouts, rows split over the host cores).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()


@pytest.fixture(scope="module")
def graph():
    rp, ci = synth.workload("ba200k")
    return rp, ci


def _rows(n):
    rng = np.random.default_rng(7)
    return np.unique(np.concatenate([[0, n - 1], rng.choice(n, 14, replace=False)]))


def _residual_ok(X_prev, Z, rp, ci, rows):
    """|L^W Z - L^{X} X|_i against the bound of the full-size residual test."""
    eps32 = np.finfo(np.float32).eps
    Zd = Z.astype(np.float64)
    brs, res, floor = [], [], []
    for i in rows:
        d = oracle.bfs_row(rp, ci, int(i)).astype(np.float64)
        b = oracle.rhs_row(X_prev, int(i), d)
        lwz = oracle.rhs_row(Zd, int(i), d) - oracle.force_row(Zd, int(i), d)
        w = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0) ** 2, 0.0)
        floor.append(eps32 * float(np.sum(w * (np.abs(Zd[i]).sum() + np.abs(Zd).sum(axis=1)))))
        brs.append(b)
        res.append(np.linalg.norm(lwz - b))
    b_rms = np.sqrt(np.mean(np.sum(np.square(brs), axis=1)))
    return all(r <= 4.0 * (1e-6 * b_rms + fl) for r, fl in zip(res, floor)), res


def _force_rows_ok(F, X, rp, ci, rows):
    """Element-wise force bound at the sampled rows; returns the worst ratio."""
    worst = 0.0
    for k, i in enumerate(rows):
        d = oracle.bfs_row(rp, ci, int(i)).astype(np.float64)
        ref = oracle.force_row(X, int(i), d)
        A = oracle.force_row_abs(X, int(i), d)
        err = np.abs(np.asarray(F[k], dtype=np.float64) - ref)
        assert np.all(err <= 1e-5 * A + 1e-30), (i, err, A)
        worst = max(worst, float(np.max(err / np.maximum(A, 1e-300))))
    return worst


def test_ba200k(graph):
    rp, ci = graph
    n = len(rp) - 1
    rows = _rows(n)
    finals = []
    for dim in (2, 3):
        X0 = synth.initial_layout(n, dim, 0)
        with api.Layout(rp, ci, dim=dim) as L:
            info = L.info()
            assert info["code_bytes"] == 1 and info["disconnected"] == 0
            assert info["bfs_sources"] == 256  # n >= 65536, few levels: the level-synchronous search
            for i in rows[:6]:
                assert np.array_equal(L.distance_rows(int(i), 1)[0],
                                      oracle.bfs_row(rp, ci, int(i)).astype(np.float64))
            _force_rows_ok(L.forces(X0).astype(np.float64)[rows], X0, rp, ci, rows)
            # three H steps (omega = 0: X^{k+1} = H(X^k)), each checked against Eq. (2-5)
            X = X0.copy()
            for k in range(3):
                Xp = X.astype(np.float64)
                L.sor_step(X, k=k, omega=0.0, cg_tol=1e-6, cg_max=500)
                ok, res = _residual_ok(Xp, X, rp, ci, rows)
                assert ok, (k, res)
            # 200 iterations of Algorithm 2 at omega = 0.5
            X = X0.copy()
            r = L.run(X, trace=True, omega=0.5, tol=0.0, max_iter=200)
            assert r.iterations == 200
            assert np.all(np.diff(r.trace_f) <= 1e-6 * r.trace_f[:-1])
            _force_rows_ok(L.forces(X).astype(np.float64)[rows], X.astype(np.float64), rp, ci, rows)
            st = r.stats
            print(f"ba200k dim={dim}: 200 iterations in {st['kernel_ms']:.0f} ms, "
                  f"{st['pair_passes'] * st['pairs'] / (st['kernel_ms'] / 1e3):.3e} pair interactions/s, "
                  f"{st['cg_steps'] / 200:.2f} CG steps per iteration, stress {r.stress:.6e}")
            finals.append((X.copy(), r.stress))
    # the final stress of both layouts against the oracle over all pairs
    f_ref = oracle.stress_stream_multi([x for x, _ in finals], rp, ci, workers=max(1, (os.cpu_count() or 2) - 1))
    for (x, f), fr in zip(finals, f_ref):
        assert f == pytest.approx(fr, rel=1e-5), (f, fr)
