"""Pins of the oracle's ideal distances d_ij (shortest paths, Sec. 2 Eq. (1)).

Each check compares against something other than the oracle itself: the
closed-form lattice distance, scipy's shortest-path routine, and a brute-force
Floyd-Warshall written out here.
"""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle
from paper_1711_01228_gb300 import synth


def _scipy_apsp(rp, ci, w=None):
    n = len(rp) - 1
    data = np.ones(len(ci)) if w is None else np.asarray(w, dtype=np.float64)
    A = csr_matrix((data, ci, rp), shape=(n, n))
    return shortest_path(A, directed=False, unweighted=(w is None))


def _floyd_warshall(rp, ci, w=None):
    n = len(rp) - 1
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            D[u, ci[e]] = min(D[u, ci[e]], 1.0 if w is None else w[e])
    for k in range(n):
        for i in range(n):
            for j in range(n):
                if D[i, k] + D[k, j] < D[i, j]:
                    D[i, j] = D[i, k] + D[k, j]
    return D


def test_grid_is_manhattan():
    rows, cols = 7, 11
    rp, ci = synth.grid(rows, cols)
    st, D = oracle.apsp(rp, ci)
    assert st == 0
    r = np.arange(rows * cols) // cols
    c = np.arange(rows * cols) % cols
    expect = np.abs(r[:, None] - r[None, :]) + np.abs(c[:, None] - c[None, :])
    assert np.array_equal(D, expect.astype(np.float64))


@pytest.mark.parametrize("maker", [
    lambda: synth.erdos_renyi(120, 5.0, seed=3),
    lambda: synth.random_binary_tree(150, seed=1),
    lambda: synth.barabasi_albert(200, 2, seed=2),
    lambda: synth.delaunay(90, seed=4),
    lambda: synth.random_geometric(100, 2, 6.0, seed=5)[:2],
])
def test_unweighted_matches_scipy(maker):
    rp, ci = maker()
    ref = _scipy_apsp(rp, ci)
    st, D = oracle.apsp(rp, ci, policy=1)
    fin = np.isfinite(ref)
    assert np.array_equal(D[fin], ref[fin])
    if not fin.all():
        assert np.all(D[~fin] == ref[fin].max() + 1)
        st0, _ = oracle.apsp(rp, ci, policy=0)
        assert st0 == oracle.ERR_DISCONNECTED
    else:
        assert st == 0


def test_weighted_matches_scipy_and_brute_force():
    rp, ci = synth.erdos_renyi(40, 4.0, seed=7)
    rng = np.random.default_rng(0)
    # symmetric lengths: one per undirected edge
    n = len(rp) - 1
    lens = {}
    w = np.empty(len(ci))
    for u in range(n):
        for e in range(rp[u], rp[u + 1]):
            key = (min(u, ci[e]), max(u, ci[e]))
            if key not in lens:
                lens[key] = rng.uniform(0.5, 2.0)
            w[e] = lens[key]
    st, D = oracle.apsp(rp, ci, edge_len=w, policy=1)
    ref = _scipy_apsp(rp, ci, w)
    fw = _floyd_warshall(rp, ci, w)
    fin = np.isfinite(ref)
    assert np.allclose(D[fin], ref[fin], rtol=1e-14, atol=0)
    assert np.allclose(D[fin], fw[fin], rtol=1e-14, atol=0)


def test_unweighted_brute_force_tiny():
    for seed in range(5):
        rp, ci = synth.erdos_renyi(25, 3.0, seed=seed)
        fw = _floyd_warshall(rp, ci)
        st, D = oracle.apsp(rp, ci, policy=1)
        fin = np.isfinite(fw)
        assert np.array_equal(D[fin], fw[fin])


def test_bfs_row_and_stream():
    rp, ci = synth.delaunay(150, seed=9)
    st, D = oracle.apsp(rp, ci)
    for s in (0, 17, 149):
        assert np.array_equal(oracle.bfs_row(rp, ci, s), D[s].astype(np.int32))
    X = synth.initial_layout(150, 2, seed=1)
    assert oracle.stress_stream(X, rp, ci) == pytest.approx(oracle.stress(X, D), rel=1e-12)


def test_stream_split_over_processes():
    # the rows of Eq. (1) split between spawned processes sum to the serial stress
    rp, ci = synth.erdos_renyi(4500, 6.0, seed=3)
    X = synth.initial_layout(4500, 2, seed=2)
    st, D = oracle.apsp(rp, ci, policy=1)
    fill = float(D.max())
    f1 = oracle.stress_stream(X, rp, ci, fill)
    f2 = oracle.stress_stream(X, rp, ci, fill, workers=2)
    assert f2 == pytest.approx(f1, rel=1e-12)
    assert f1 == pytest.approx(oracle.stress(X, D), rel=1e-12)


def test_stream_several_layouts_share_rows():
    # one BFS per row for a 2-D and a 3-D layout: each equals its own stress
    rp, ci = synth.delaunay(300, seed=4)
    st, D = oracle.apsp(rp, ci)
    X2, X3 = synth.initial_layout(300, 2, seed=1), synth.initial_layout(300, 3, seed=2)
    f = oracle.stress_stream_multi([X2, X3], rp, ci)
    assert f[0] == pytest.approx(oracle.stress(X2, D), rel=1e-12)
    assert f[1] == pytest.approx(oracle.stress(X3, D), rel=1e-12)
