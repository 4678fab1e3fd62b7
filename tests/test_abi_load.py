"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/fd_layout.h declares.  No GPU work."""
import ctypes
import os
import re
import shutil

import pytest

from paper_1711_01228_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fd_layout.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("fd_layout_create", "fd_forces", "fd_sor_step", "fd_energy", "fd_run"):
        assert want in names
    assert sorted(api.EXPORTED) == names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings_and_defaults(libpath):
    L = api.lib()
    for code, name in api.STATUS_NAMES.items():
        assert L.fd_status_string(code).decode() == name
    o = api.options()
    assert (o.omega, o.strategy, o.stop, o.tol, o.max_iter, o.cg_max, o.cg_tol) == (
        0.5, 0, 0, 1e-4, 1000, 200, 1e-6)


def test_option_defaults_match_the_header(libpath):
    # fd_options_default is host code: the documented defaults, no GPU needed
    from paper_1711_01228_gb300 import api

    o = api.options()
    assert (o.omega, o.strategy, o.stop, o.seed) == (0.5, api.OMEGA_FIXED, api.STOP_REL_DISP, 0)
    assert (o.tol, o.max_iter, o.cg_max, o.cg_tol) == (1e-4, 1000, 200, 1e-6)
    assert (o.solver, o.first_iter) == (api.SOLVER_CG, 0)
    o2 = api.options(solver=api.SOLVER_DIRECT, first_iter=7)
    assert (o2.solver, o2.first_iter) == (1, 7)
    with pytest.raises(TypeError):
        api.options(no_such_option=1)
