"""The graph of the paper's Fig. 4 (left): a protein-protein interaction
module (179 vertices, 208 edges), printed with the coordinates of the
paper's SOR layout (tests/golden/fig4_ppi_module.txt).  A weak pin on real
data: the printed layout, scaled optimally, has a stress the method reaches
from random starts (stress majorization has many local minima, so the best
of a few seeded starts is compared)."""
import os

import numpy as np

import oracle
from paper_1711_01228_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def load_fig4():
    rows = [l for l in open(os.path.join(HERE, "golden", "fig4_ppi_module.txt")) if not l.startswith("#")]
    n, m = (int(t) for t in rows[0].split())
    X = np.array([[float(t) for t in r.split()[1:]] for r in rows[1:1 + n]])
    E = np.array([[int(t) - 1 for t in r.split()] for r in rows[1 + n:1 + n + m]])
    rp, ci = synth.csr_from_edges(n, E)
    return rp, ci, X


def test_fig4_graph_shape():
    rp, ci, X = load_fig4()
    st, D = oracle.apsp(rp, ci)
    assert st == 0 and len(rp) - 1 == 179 and rp[-1] // 2 == 208 and D.max() == 20


def test_printed_layout_stress_is_reached():
    rp, ci, X = load_fig4()
    _, D = oracle.apsp(rp, ci)
    # optimal scale of the printed coordinates: argmin_s f(s X) = sum w d r / sum w r^2
    iu = np.triu_indices(len(X), 1)
    d = D[iu]
    r = np.linalg.norm(X[iu[0]] - X[iu[1]], axis=1)
    s = np.sum(r / d) / np.sum(r * r / d ** 2)
    f_printed = oracle.stress(s * X, D)
    best = min(oracle.sor_run(D, synth.initial_layout(179, 2, seed).astype(np.float64), omega=0.5, tol=1e-6,
                              stop=oracle.STOP_REL_STRESS, max_iter=5000).stress for seed in range(5))
    assert best <= f_printed
    assert best >= 0.95 * f_printed  # the printed layout is near the best local minimum found
