"""Host-side pieces of the batched form (no GPU): the concatenation of
graphs into one CSR and the batched workload's generators."""
import math
import os
import shutil

import numpy as np
import pytest

from paper_1711_01228_gb300 import api, build, synth


def test_concat_graphs_is_the_disjoint_union():
    gs = [synth.path(3), synth.grid(2, 2), synth.complete(1)]
    gp, rp, ci = api.concat_graphs(gs)
    assert gp.tolist() == [0, 3, 7, 8]
    assert rp[0] == 0 and rp[-1] == sum(int(r[-1]) for r, _ in gs)
    for g, (rpg, cig) in enumerate(gs):
        v0, v1 = gp[g], gp[g + 1]
        for v in range(v0, v1):
            nb = ci[rp[v]:rp[v + 1]]
            assert np.all((nb >= v0) & (nb < v1))
            assert np.array_equal(nb - v0, cig[rpg[v - v0]:rpg[v - v0 + 1]])


def test_batch_sizes_log_uniform():
    s = synth.batch_sizes(20000, 16, 2048, seed=1)
    assert s.min() >= 16 and s.max() <= 2048
    # log-uniform: the median of log n is the midpoint of [ln 16, ln 2048]
    mid = 0.5 * (math.log(16) + math.log(2048))
    assert abs(np.median(np.log(s + 0.5)) - mid) < 0.05


def test_batch_graph_mix():
    gs = synth.batch_graphs(40, n_max=300, seed=2)
    for g, (rp, ci) in enumerate(gs):
        n = len(rp) - 1
        deg = rp[-1] / n
        if g % 2 == 1 and n >= 64:  # random geometric: mean degree bisected to 6 +- 0.5
            assert abs(deg - 6.0) <= 0.5
        # simple and symmetric
        for v in range(n):
            nb = ci[rp[v]:rp[v + 1]]
            assert v not in nb and len(set(nb.tolist())) == len(nb)
    X = synth.batch_initial_layout([len(rp) - 1 for rp, _ in gs], 2, seed=0)
    assert X.dtype == np.float32 and X.shape[1] == 2 and np.all((X >= 0) & (X < 1))


def test_tile_cache_is_host_state():
    # the tuned tile edges live in a process-wide table on the host
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    build.build()
    api.batch_clear_tile_cache()
    for dim in (1, 2, 3):
        assert api.batch_cached_tiles(dim) == [0] * api.BATCH_BUCKETS
    with pytest.raises(api.FdError):
        api.batch_cached_tiles(4)


def test_trace_jsonl(tmp_path):
    import json

    r = api.RunResult(iterations=2, stress=1.5, trace_f=np.array([3.0, 2.0, 1.5]),
                      accepted=np.array([1, 0], dtype=np.int32), omega=np.array([0.5, 0.5]),
                      cg_steps=np.array([4, 3], dtype=np.int32), crit=np.array([0.1, 0.01]),
                      f_h=np.array([2.2, 1.5]), f_extrapolated=np.array([2.0, 1.7]), t_ms=np.array([0.25, 0.5]))
    p = tmp_path / "t.jsonl"
    api.write_trace_jsonl(r, str(p), graph="g")
    recs = [json.loads(line) for line in p.read_text().splitlines()]
    assert recs == [{"k": 1, "stress": 2.0, "stress_h": 2.2, "stress_extrapolated": 2.0, "accepted": True,
                     "omega": 0.5, "cg_steps": 4, "crit": 0.1, "t_ms": 0.25, "graph": "g"},
                    {"k": 2, "stress": 1.5, "stress_h": 1.5, "stress_extrapolated": 1.7, "accepted": False,
                     "omega": 0.5, "cg_steps": 3, "crit": 0.01, "t_ms": 0.5, "graph": "g"}]
