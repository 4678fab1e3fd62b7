"""Parity of the batched form (many graphs in one persistent launch) with the
FP64 oracle, graph by graph.

Tolerances are those of the single-graph parity tests: distances bit-exact,
converged runs within 1e-4 relative on final stress and 2 % (at least 1) on
the iteration count.  Every graph of a batch runs Algorithm 2 on its own; the
oracle runs it on each graph separately.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.lib()


def _mixed_graphs():
    """Sizes across the tile boundaries (1 vertex, 2, 127, 128, 129, 300,
    600), lattices, sparse random graphs (disconnected), geometric graphs."""
    gs = [synth.path(1), synth.path(2), synth.complete(3), synth.grid(20, 20),
          synth.erdos_renyi(127, 4.0, seed=1), synth.erdos_renyi(128, 4.0, seed=2),
          synth.random_geometric(129, 2, 6.0, seed=3)[:2], synth.erdos_renyi(300, 4.0, seed=4),
          synth.random_geometric(600, 2, 6.0, seed=5)[:2], synth.random_binary_tree(255, seed=6)]
    return gs


def _layouts(sizes, dim, seed=0):
    return synth.batch_initial_layout(sizes, dim, seed)


def _close_iters(a, b):
    return abs(a - b) <= max(1, math.ceil(0.02 * b))


def test_batch_distances_bit_exact():
    gs = _mixed_graphs()
    with api.Batch.from_graphs(gs, dim=2, disconnected_policy=1) as B:
        info = B.info()
        assert info["num_graphs"] == len(gs)
        for g, (rp, ci) in enumerate(gs):
            _, D = oracle.apsp(rp, ci, policy=1)
            assert np.array_equal(B.distances(g), D), g


# In 1-D the stress has many local minima (orderings of the vertices on the
# line): FP32 and FP64 runs may settle in different ones, so 1-D compares the
# first iterations of the trajectory; 2-D and 3-D compare converged runs.
@pytest.mark.parametrize("dim,max_iter", [(1, 5), (2, 1000), (3, 1000)])
def test_batch_runs_match_oracle(dim, max_iter):
    gs = _mixed_graphs()
    sizes = [len(rp) - 1 for rp, _ in gs]
    X0 = _layouts(sizes, dim, seed=1)
    X = X0.copy()
    with api.Batch.from_graphs(gs, dim=dim, disconnected_policy=1) as B:
        r = B.run(X, omega=0.5, tol=1e-4, max_iter=max_iter)
        gp = B.graph_ptr
    assert np.all(r.status == 0)
    for g, (rp, ci) in enumerate(gs):
        _, D = oracle.apsp(rp, ci, policy=1)
        x0 = X0[gp[g]:gp[g + 1]].astype(np.float64)
        ref = oracle.sor_run(D, x0, omega=0.5, tol=1e-4, max_iter=max_iter)
        assert r.stress[g] == pytest.approx(ref.stress, rel=1e-4, abs=1e-9), g
        assert _close_iters(int(r.iterations[g]), ref.iterations), (g, r.iterations[g], ref.iterations)
        # the returned layout has the reported stress
        assert oracle.stress(X[gp[g]:gp[g + 1]], D) == pytest.approx(r.stress[g], rel=1e-5, abs=1e-9)


def test_batch_matches_single_graph_path():
    gs = [synth.grid(20, 20), synth.delaunay(900, seed=9), synth.random_geometric(1500, 2, 6.0, seed=10)[:2]]
    sizes = [len(rp) - 1 for rp, _ in gs]
    X0 = _layouts(sizes, 2, seed=2)
    Xb = X0.copy()
    with api.Batch.from_graphs(gs, dim=2, disconnected_policy=1) as B:
        rb = B.run(Xb, omega=0.5, tol=1e-4, max_iter=1000)
        gp = B.graph_ptr
    for g, (rp, ci) in enumerate(gs):
        x = X0[gp[g]:gp[g + 1]].copy()
        with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
            r = L.run(x, omega=0.5, tol=1e-4, max_iter=1000)
        assert rb.stress[g] == pytest.approx(r.stress, rel=1e-4)
        assert _close_iters(int(rb.iterations[g]), r.iterations)


def test_per_graph_omega_and_algorithm1():
    # omega = 0 for one graph is Algorithm 1; the others use their own omega
    gs = [synth.grid(12, 12), synth.grid(12, 12), synth.grid(12, 12)]
    oms = np.array([0.0, 0.5, 1.0])
    X0 = _layouts([144] * 3, 2, seed=3)
    X = X0.copy()
    with api.Batch.from_graphs(gs, dim=2) as B:
        r = B.run(X, omega=oms, tol=1e-4, max_iter=1000)
    _, D = oracle.apsp(*gs[0])
    for g in range(3):
        ref = oracle.sor_run(D, X0[144 * g:144 * (g + 1)].astype(np.float64), omega=float(oms[g]), tol=1e-4,
                             max_iter=1000)
        assert r.stress[g] == pytest.approx(ref.stress, rel=1e-4)
        assert _close_iters(int(r.iterations[g]), ref.iterations)
    assert r.accepted[0] == r.iterations[0]  # omega = 0: X^{k+1} = H(X^k) every time


def test_probabilistic_strategy():
    gs = [synth.grid(10, 10), synth.erdos_renyi(200, 4.0, seed=8)]
    sizes = [100, 200]
    X0 = _layouts(sizes, 2, seed=4)
    X = X0.copy()
    with api.Batch.from_graphs(gs, dim=2, disconnected_policy=1) as B:
        r = B.run(X, strategy=api.OMEGA_PROB, seed=42, tol=1e-4, max_iter=300)
        gp = B.graph_ptr
    for g, (rp, ci) in enumerate(gs):
        _, D = oracle.apsp(rp, ci, policy=1)
        ref = oracle.sor_run(D, X0[gp[g]:gp[g + 1]].astype(np.float64), strategy=oracle.OMEGA_PROB, seed=42,
                             tol=1e-4, max_iter=300)
        assert r.stress[g] == pytest.approx(ref.stress, rel=1e-4)
        assert _close_iters(int(r.iterations[g]), ref.iterations)


@pytest.mark.parametrize("groups,stages", [(1, 2), (1, 3), (2, 2), (2, 3)])
def test_every_launch_shape_agrees(groups, stages):
    gs = [synth.delaunay(1100, seed=12), synth.erdos_renyi(400, 4.0, seed=13), synth.grid(9, 9)]
    sizes = [len(rp) - 1 for rp, _ in gs]
    X0 = _layouts(sizes, 2, seed=5)
    with api.Batch.from_graphs(gs, dim=2, disconnected_policy=1) as B:
        B.set_shape(groups, stages)
        info = B.info()
        assert (info["groups"], info["stages"]) == (groups, stages)
        X = X0.copy()
        r = B.run(X, omega=0.5, tol=1e-4, max_iter=1000)
        gp = B.graph_ptr
    for g, (rp, ci) in enumerate(gs):
        _, D = oracle.apsp(rp, ci, policy=1)
        ref = oracle.sor_run(D, X0[gp[g]:gp[g + 1]].astype(np.float64), omega=0.5, tol=1e-4, max_iter=1000)
        assert r.stress[g] == pytest.approx(ref.stress, rel=1e-4)
        assert _close_iters(int(r.iterations[g]), ref.iterations)


def test_tuner_and_graph_capture():
    import torch

    gs = synth.batch_graphs(64, n_max=512, seed=3)
    sizes = [len(rp) - 1 for rp, _ in gs]
    X0 = _layouts(sizes, 2, seed=6)
    stream = torch.cuda.Stream()  # a stream that can be captured (not the legacy default stream)
    torch.cuda.synchronize()
    with api.Batch.from_graphs(gs, dim=2, disconnected_policy=1, stream=stream.cuda_stream) as B:
        g, s = B.tune(torch.from_numpy(X0).cuda(), probe_iter=3, repeats=1)
        assert (g, s) in ((1, 2), (1, 3), (2, 2), (2, 3))
        assert (B.info()["groups"], B.info()["stages"]) == (g, s)
        tiles = B.tiles()
        assert all(t in api.BATCH_TILES for t in tiles)
        assert api.batch_cached_tiles(2) == tiles  # kept for later batches of this dimension
        # one tile group (one 128-thread unit at edge 128) adds every sum in a
        # fixed order: replays are bit-identical
        B.set_shape(1, 2)
        B.set_tiles([128] * api.BATCH_BUCKETS)
        Xa = torch.from_numpy(X0).cuda()
        ra = B.run(Xa, omega=0.5, tol=1e-4, max_iter=1000)
        Xb = torch.from_numpy(X0).cuda()
        rb = B.run(Xb, omega=0.5, tol=1e-4, max_iter=1000)  # replayed from the captured graph
        assert B.info()["graph_captured"] == 1
    assert np.array_equal(ra.iterations, rb.iterations)
    assert np.array_equal(ra.stress, rb.stress)
    assert torch.equal(Xa, Xb)


def _edge_graphs():
    """Sizes across the 32- and 64-vertex block boundaries and into buckets 0-4."""
    return [synth.path(1), synth.path(2), synth.complete(3), synth.erdos_renyi(31, 4.0, seed=21),
            synth.grid(4, 8), synth.random_geometric(33, 2, 6.0, seed=22)[:2], synth.erdos_renyi(63, 4.0, seed=23),
            synth.grid(8, 8), synth.random_binary_tree(65, seed=24), synth.erdos_renyi(100, 4.0, seed=25),
            synth.random_geometric(129, 2, 6.0, seed=26)[:2], synth.erdos_renyi(300, 4.0, seed=27)]


def _connected(rp, ci):
    return oracle.apsp(rp, ci, policy=0)[0] == 0


# Every tile edge against the oracle: the stress after one iteration (every
# code of every tile enters it) within 1e-5, converged stress within 1e-4, and
# the iteration count within 2 % on the connected graphs.  On the
# disconnected ones (unreachable pairs at (largest d) + 1) the criterion
# decays by under 2 % per iteration near the tolerance, the FP32 runs of every
# path (both kernels, every tile edge) stop 1-10 % before the FP64 oracle
# (e.g. ER n = 31: 248-254 vs 265 in 2-D), and only the stress is compared.
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("tile", [32, 64, 128])
def test_every_tile_edge_agrees(tile, dim):
    gs = _edge_graphs()
    sizes = [len(rp) - 1 for rp, _ in gs]
    X0 = _layouts(sizes, dim, seed=7)
    with api.Batch.from_graphs(gs, dim=dim, disconnected_policy=1) as B:
        B.set_tiles([tile] * api.BATCH_BUCKETS)
        info = B.info()
        assert info[f"graphs_t{tile}"] == len(gs)
        X1 = X0.copy()
        r1 = B.run(X1, omega=0.5, tol=0.0, max_iter=1)
        X = X0.copy()
        r = B.run(X, omega=0.5, tol=1e-4, max_iter=1000)
        gp = B.graph_ptr
    for g, (rp, ci) in enumerate(gs):
        _, D = oracle.apsp(rp, ci, policy=1)
        x0 = X0[gp[g]:gp[g + 1]].astype(np.float64)
        one = oracle.sor_run(D, x0, omega=0.5, tol=0.0, max_iter=1)
        assert r1.stress[g] == pytest.approx(one.stress, rel=1e-5, abs=1e-9), (g, tile)
        ref = oracle.sor_run(D, x0, omega=0.5, tol=1e-4, max_iter=1000)
        assert r.stress[g] == pytest.approx(ref.stress, rel=1e-4, abs=1e-9), (g, tile)
        if _connected(rp, ci):
            assert _close_iters(int(r.iterations[g]), ref.iterations), (g, tile, r.iterations[g], ref.iterations)


def test_mixed_tile_edges_and_cache():
    gs = _edge_graphs() + [synth.delaunay(700, seed=28)]
    sizes = [len(rp) - 1 for rp, _ in gs]
    X0 = _layouts(sizes, 2, seed=8)
    tiles = [32, 64, 32, 64, 128, 64, 128]
    api.batch_clear_tile_cache()
    with api.Batch.from_graphs(gs, dim=2, disconnected_policy=1) as B:
        assert B.tiles() == [128] * api.BATCH_BUCKETS  # nothing cached: edge 128
        B.set_tiles(tiles)
        assert B.tiles() == tiles
        info = B.info()
        edge = [tiles[min(6, max(0, int(np.ceil(np.log2(max(n, 1) / 32)))))] for n in sizes]
        assert (info["graphs_t32"], info["graphs_t64"], info["graphs_t128"]) == (
            edge.count(32), edge.count(64), edge.count(128))
        assert info["small_tile_bytes"] > 0
        X = X0.copy()
        r = B.run(X, omega=0.5, tol=1e-4, max_iter=1000)
        gp = B.graph_ptr
        with pytest.raises(api.FdError) as e:
            B.set_tiles([16] * api.BATCH_BUCKETS)
        assert e.value.status == 1
    for g, (rp, ci) in enumerate(gs):
        _, D = oracle.apsp(rp, ci, policy=1)
        ref = oracle.sor_run(D, X0[gp[g]:gp[g + 1]].astype(np.float64), omega=0.5, tol=1e-4, max_iter=1000)
        assert r.stress[g] == pytest.approx(ref.stress, rel=1e-4, abs=1e-9), g
        if _connected(rp, ci):
            assert _close_iters(int(r.iterations[g]), ref.iterations), g
    assert api.batch_cached_tiles(2) == [0] * api.BATCH_BUCKETS  # set_tiles does not touch the cache


def test_batch_errors():
    rp, ci = synth.grid(4, 4)
    gp, rpa, cia = api.concat_graphs([(rp, ci), (rp, ci)])
    bad = cia.copy()
    # move one edge of graph 0 to a vertex of graph 1 (and its reverse entry)
    u = 0
    v = int(bad[rpa[u]])
    bad[rpa[u]] = 16 + v
    with pytest.raises(api.FdError) as e:
        api.Batch(gp, rpa, bad, dim=2)
    assert e.value.status in (1, 2)
    big = synth.path(2049)
    with pytest.raises(api.FdError) as e:
        api.Batch.from_graphs([big], dim=2)
    assert e.value.status == 1
    dis = synth.erdos_renyi(100, 1.0, seed=1)
    with pytest.raises(api.FdError) as e:
        api.Batch.from_graphs([dis], dim=2, disconnected_policy=0)
    assert e.value.status == 3
    with api.Batch.from_graphs([(rp, ci), (rp, ci)], dim=2) as B:
        X = _layouts([16, 16], 2)
        with pytest.raises(api.FdError) as e:
            B.run(X.copy(), strategy=api.OMEGA_ENUM)
        assert e.value.status == 10
        with pytest.raises(api.FdError) as e:
            B.run(X.copy(), solver=api.SOLVER_DIRECT)
        assert e.value.status == 10
        Xn = X.copy()
        Xn[3, 0] = np.nan  # graph 0 only
        r = B.run(Xn, check=False, omega=0.5)
        assert r.status[0] == 4 and r.status[1] == 0
        assert r.iterations[1] > 0
