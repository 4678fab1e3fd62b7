"""Seeded synthetic inputs: graphs as int32 CSR and initial layouts.

These generators hold none of the layout method's arithmetic; the CUDA path,
the oracle, the tests and the benchmark all take their inputs from here so
that both sides see the same arrays.

The paper evaluates on graph-drawing benchmark sets (band-*, grid-*, net-*;
Table 1 of Sec. 5) that are not distributed with it.  Stand-ins here have the
same kinds of structure: lattices, sparse random graphs, planar meshes, trees,
power-law graphs and random geometric graphs.  The initial layout is uniform
on the unit square (Sec. 5.1), generalised to the unit cube for dim = 3.

Every graph is undirected, simple (no self loops, no multi-edges) and returned
as ``(row_ptr[n+1], col_idx[2m])`` with both directions of each edge and
neighbours sorted within each row.
"""
from __future__ import annotations

import math

import numpy as np


def csr_from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR of an undirected simple graph from an (m, 2) edge array.

    Self loops and duplicate edges are dropped.
    """
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    key = np.unique(lo * n + hi)
    lo, hi = key // n, key % n
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr.astype(np.int32), dst.astype(np.int32)


def num_edges(row_ptr) -> int:
    return int(row_ptr[-1]) // 2


def grid(rows: int, cols: int):
    """rows x cols 4-neighbour lattice (20 x 20: n = 400, m = 760)."""
    idx = np.arange(rows * cols).reshape(rows, cols)
    h = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    v = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    return csr_from_edges(rows * cols, np.concatenate([h, v]))


def path(n: int):
    e = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1)
    return csr_from_edges(n, e)


def cycle(n: int):
    e = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1)
    return csr_from_edges(n, e)


def complete(n: int):
    i, j = np.triu_indices(n, 1)
    return csr_from_edges(n, np.stack([i, j], axis=1))


def star(leaves: int):
    e = np.stack([np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1)], axis=1)
    return csr_from_edges(leaves + 1, e)


def erdos_renyi(n: int, mean_degree: float, seed: int = 0):
    """G(n, p) with p = mean_degree / (n - 1): the edge count is drawn from
    Binomial(n(n-1)/2, p) and that many distinct pairs are drawn uniformly."""
    rng = np.random.default_rng(seed)
    npairs = n * (n - 1) // 2
    p = mean_degree / max(n - 1, 1)
    m = int(rng.binomial(npairs, min(p, 1.0)))
    chosen = set()
    out = []
    while len(out) < m:
        k = m - len(out)
        a = rng.integers(0, n, size=2 * k + 16)
        b = rng.integers(0, n, size=2 * k + 16)
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            key = (x, y) if x < y else (y, x)
            if key in chosen:
                continue
            chosen.add(key)
            out.append(key)
            if len(out) == m:
                break
    return csr_from_edges(n, np.array(out, dtype=np.int64).reshape(-1, 2))


def delaunay(n: int, seed: int = 0):
    """Delaunay triangulation of n uniform points in [0,1]^2; edges are the
    unique triangle sides (about 3n)."""
    from scipy.spatial import Delaunay

    pts = np.random.default_rng(seed).random((n, 2))
    tri = Delaunay(pts)
    s = tri.simplices.astype(np.int64)
    e = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]])
    return csr_from_edges(n, e)


def random_binary_tree(n: int, seed: int = 0):
    """Random binary tree: vertex t >= 1 attaches to a uniformly chosen
    earlier vertex that has fewer than two children."""
    rng = np.random.default_rng(seed)
    open_nodes = [0]
    children = np.zeros(n, dtype=np.int8)
    e = np.empty((max(n - 1, 0), 2), dtype=np.int64)
    draws = rng.random(max(n - 1, 0))
    for t in range(1, n):
        k = int(draws[t - 1] * len(open_nodes))
        par = open_nodes[k]
        e[t - 1] = (par, t)
        children[par] += 1
        if children[par] == 2:
            open_nodes[k] = open_nodes[-1]
            open_nodes.pop()
        open_nodes.append(t)
    return csr_from_edges(n, e)


def barabasi_albert(n: int, m: int, seed: int = 0):
    """Preferential attachment: vertex m links to 0..m-1; each later vertex
    links to m distinct earlier vertices drawn with probability proportional
    to degree (drawn from the list of edge endpoints)."""
    rng = np.random.default_rng(seed)
    edges = np.empty(((n - m) * m, 2), dtype=np.int64)
    ends = np.empty(2 * (n - m) * m, dtype=np.int64)
    ne = 0
    targets = list(range(m))
    for v in range(m, n):
        for t in targets:
            edges[ne] = (v, t)
            ends[2 * ne] = v
            ends[2 * ne + 1] = t
            ne += 1
        chosen = set()
        while len(chosen) < m:
            chosen.add(int(ends[rng.integers(0, 2 * ne)]))
        targets = sorted(chosen)
    return csr_from_edges(n, edges[:ne])


def random_geometric(n: int, dim: int = 2, mean_degree: float = 6.0, seed: int = 0,
                     rescale: bool = True):
    """Random geometric graph of n uniform points in [0,1]^dim.

    The radius starts from the mean-degree estimate without boundary effects
    and, if ``rescale``, is bisected until the realised mean degree is within
    0.5 of the target.  Returns (row_ptr, col_idx, points).
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.random((n, dim))
    tree = cKDTree(pts)
    unit_ball = math.pi ** (dim / 2) / math.gamma(dim / 2 + 1)
    r = (mean_degree / (max(n - 1, 1) * unit_ball)) ** (1.0 / dim)

    def pairs(rad):
        return tree.query_pairs(rad, output_type="ndarray")

    p = pairs(r)
    if rescale and n > 1:
        lo, hi = r, r
        deg = 2.0 * len(p) / n
        if deg < mean_degree:
            while 2.0 * len(pairs(hi)) / n < mean_degree:
                hi *= 1.25
        else:
            while 2.0 * len(pairs(lo)) / n > mean_degree:
                lo /= 1.25
        for _ in range(60):
            if abs(deg - mean_degree) <= 0.5:
                break
            r = 0.5 * (lo + hi)
            p = pairs(r)
            deg = 2.0 * len(p) / n
            if deg < mean_degree:
                lo = r
            else:
                hi = r
    rp, ci = csr_from_edges(n, p)
    return rp, ci, pts


def initial_layout(n: int, dim: int = 2, seed: int = 0) -> np.ndarray:
    """X^0 uniform on [0,1)^dim (Sec. 5.1), drawn in FP64 and stored as FP32."""
    return np.random.default_rng(seed).random((n, dim)).astype(np.float32)


def batch_sizes(num_graphs: int, n_min: int = 16, n_max: int = 2048, seed: int = 0) -> np.ndarray:
    """Graph sizes log-uniform in [n_min, n_max]: floor(exp(U[ln n_min, ln n_max]))."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(n_min), math.log(n_max), size=num_graphs)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), n_min, n_max)


def batch_graphs(num_graphs: int = 4096, n_min: int = 16, n_max: int = 2048, seed: int = 0):
    """The batched workload: sizes log-uniform in [n_min, n_max]; graphs with
    an even index are Erdos-Renyi with mean degree 4, odd ones random geometric
    graphs in the unit square with the radius bisected to mean degree 6 (+-0.5).
    Graph g draws from seed 1000003 * seed + g.  Returns a list of CSR pairs."""
    sizes = batch_sizes(num_graphs, n_min, n_max, seed)
    out = []
    for g, n in enumerate(sizes.tolist()):
        sg = 1000003 * seed + g
        if g % 2 == 0:
            out.append(erdos_renyi(n, 4.0, sg))
        else:
            rp, ci, _ = random_geometric(n, 2, 6.0, sg)
            out.append((rp, ci))
    return out


def batch_initial_layout(sizes, dim: int = 2, seed: int = 0) -> np.ndarray:
    """X^0 of every graph of a batch, concatenated: graph g's rows are
    initial_layout(n_g, dim, 1000003 * seed + g)."""
    return np.concatenate([initial_layout(int(n), dim, 1000003 * seed + g) for g, n in enumerate(sizes)])


# Named workloads (sizes of the graph-drawing benchmark stand-ins).
def workload(name: str, seed: int = 0):
    """CSR of a named synthetic workload."""
    if name == "grid20":
        return grid(20, 20)
    if name == "er10k":
        return erdos_renyi(10_000, 6.0, seed)
    if name == "delaunay20k":
        return delaunay(20_000, seed)
    if name == "tree16k":
        return random_binary_tree(16_383, seed)
    if name == "ba200k":
        return barabasi_albert(200_000, 3, seed)
    if name == "ba50k":
        return barabasi_albert(50_000, 3, seed)
    raise KeyError(name)
