"""The allocation-free stress entry point agrees with fd_energy and the oracle.

fd_energy_noalloc serves callers that cannot allocate GPU memory (a process
whose device memory belongs to another allocator, or a loop that cannot
afford an allocation's synchronisation): it takes a dense distance matrix and
uses only a fixed scratch array inside the library.  This file is collected
last so that a failure here comes after every other test has run; it must
pass alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_fd_energy_and_oracle_twice():
    import torch

    build.build()
    rp, ci = synth.delaunay(900, seed=13)
    n = len(rp) - 1
    with api.Layout(rp, ci, dim=2, disconnected_policy=1) as L:
        Dd = L.distance_rows(0, n)
        D = torch.from_numpy(Dd.astype(np.float32)).cuda()
        for seed in (1, 2):  # two calls in a row share the scratch array
            X = synth.initial_layout(n, 2, seed=seed) * 2.0
            f_ref = L.energy(X)
            f = api.energy_noalloc(torch.from_numpy(X).cuda(), D)
            # stress tolerance of the parity tests: 1e-5 relative
            assert f == pytest.approx(f_ref, rel=1e-5)
            assert f == pytest.approx(oracle.stress(X, Dd), rel=1e-5)


def test_noalloc_device_output_and_no_pairs():
    import torch

    build.build()
    rp, ci = synth.erdos_renyi(700, 5.0, seed=4)
    n = len(rp) - 1
    st, Dd = oracle.apsp(rp, ci, policy=1)
    X = synth.initial_layout(n, 3, seed=3)
    Xd, D = torch.from_numpy(X).cuda(), torch.from_numpy(Dd.astype(np.float32)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stt = api.lib().fd_energy_noalloc(Xd.data_ptr(), D.data_ptr(), n, 3, out.data_ptr(), None)
    assert stt == 0
    with api.Layout(rp, ci, dim=3, disconnected_policy=1) as L:
        assert float(out.item()) == pytest.approx(L.energy(X), rel=1e-5)
    # a pair whose stored d_ij is 0 is no pair: it adds nothing
    X3 = np.array([[0.0, 0.0], [0.5, 0.0], [0.0, 2.0]], dtype=np.float32)
    D3 = np.array([[0, 0, 0], [0.0, 0, 0], [1.0, 1.0, 0]], dtype=np.float32)  # d_01 = 0, d_02 = d_12 = 1
    f = api.energy_noalloc(torch.from_numpy(X3).cuda(), torch.from_numpy(D3).cuda())
    want = (2.0 - 1.0) ** 2 + (np.hypot(0.5, 2.0) - 1.0) ** 2
    assert f == pytest.approx(want, rel=1e-6)


def test_noalloc_rejects_oversize_and_host_inputs():
    import torch

    build.build()
    X = torch.zeros((4, 2), dtype=torch.float32)
    D = torch.ones((4, 4), dtype=torch.float32)
    with pytest.raises(api.FdError) as e:
        api.energy_noalloc(X, D)  # host tensors: the call cannot stage them without allocating
    assert e.value.status == 1
    Xd, Dd = X.cuda(), D.cuda()
    f = ctypes.c_double()
    # n above the limit is rejected before any memory is touched
    st = api.lib().fd_energy_noalloc(Xd.data_ptr(), Dd.data_ptr(), api.NOALLOC_MAX_N + 1, 2, ctypes.addressof(f),
                                     None)
    assert st == 1
