"""The allocation-free stress entry point agrees with fd_energy.

fd_energy_noalloc serves callers that cannot allocate GPU memory (a process
whose device memory belongs to another allocator, or a loop that cannot
afford an allocation's synchronisation): it takes a dense distance matrix and
uses only a fixed scratch array inside the library.  This file is collected
last so that a failure here comes after every other test has run; it must
pass alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_1711_01228_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_fd_energy_twice():
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
            assert f == pytest.approx(f_ref, rel=1e-5)


def test_noalloc_rejects_oversize_and_host_inputs():
    import torch

    build.build()
    X = torch.zeros((4, 2), dtype=torch.float32)
    D = torch.ones((4, 4), dtype=torch.float32)
    with pytest.raises(api.FdError) as e:
        api.energy_noalloc(X, D)  # host tensors: the call cannot stage them without allocating
    assert e.value.status == 1
    import ctypes

    Xd, Dd = X.cuda(), D.cuda()
    f = ctypes.c_double()
    # n above the limit is rejected before any memory is touched
    st = api.lib().fd_energy_noalloc(Xd.data_ptr(), Dd.data_ptr(), api.NOALLOC_MAX_N + 1, 2, ctypes.addressof(f),
                                     None)
    assert st == 1
