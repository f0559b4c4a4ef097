"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function declared in include/xrl.h; creating a context
without a GPU fails with an error code instead of crashing."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "xrl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xrl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


def test_header_declares_the_boundary():
    fns = _header_functions()
    for f in ["xrl_create", "xrl_set_mesh", "xrl_set_conductors", "xrl_add_port", "xrl_setup",
              "xrl_fmm_mvm", "xrl_fmm_mvm_device", "xrl_solve", "xrl_last_error", "xrl_destroy"]:
        assert f in fns


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built.library_path())
    for f in _header_functions():
        assert hasattr(L, f), f


def test_binding_covers_the_header(built):
    from paper_2409_12375_gb300 import xrl
    assert sorted(xrl.SIGNATURES) == _header_functions()


def test_create_without_gpu_returns_error(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2409_12375_gb300 import xrl
    with pytest.raises(xrl.XRLError) as e:
        xrl.XRL()
    assert e.value.code == 4   # XRL_ECUDA


def test_default_options(built):
    from paper_2409_12375_gb300 import xrl
    o = xrl.Options()
    xrl.lib().xrl_default_options(ctypes.byref(o))
    assert o.fmm_order == 8 and o.restart == 50 and o.tol == 1e-8
