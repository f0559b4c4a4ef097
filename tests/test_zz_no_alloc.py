"""The allocation-free FMM product (xrl_fmm_mvm_device_noalloc).

It exists for callers that cannot allocate GPU memory when they need a
product: a latency-critical loop where a cudaMalloc could stall or fail, or a
host framework whose own allocator owns the device memory budget.  These
tests call it through the C ABI (ctypes, raw device pointers) and compare it
with the ordinary entry point, xrl_fmm_mvm_device, on two calls in a row, in
an FP64 context and in a mixed-precision context after a solve; the file is
named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    x = pkg.XRL.from_mesh(meshgen.bar(), fmm_order=8)
    yield x
    x.close()


def _call(fn, ctx, x, y):
    import torch
    code = fn(ctx.h, x.shape[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), None)
    torch.cuda.synchronize()
    return code


def test_noalloc_matches_allocating_entry_twice(ctx):
    import torch

    from paper_2409_12375_gb300 import xrl
    L = xrl.lib()
    rng = np.random.default_rng(21)
    for call in range(2):
        x = torch.tensor(rng.standard_normal((3, ctx.n_tri)), device="cuda:0")
        y_ref = torch.empty_like(x)
        y_na = torch.full_like(x, float("nan"))
        assert _call(L.xrl_fmm_mvm_device, ctx, x, y_ref) == 0
        assert _call(L.xrl_fmm_mvm_device_noalloc, ctx, x, y_na) == 0, L.xrl_last_error(ctx.h)
        a = y_na.cpu().numpy()
        b = y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12, call


def test_noalloc_rejects_sizes_beyond_the_fixed_array(ctx):
    import torch

    from paper_2409_12375_gb300 import xrl
    L = xrl.lib()
    x = torch.zeros((2048, ctx.n_tri), device="cuda:0", dtype=torch.float64)
    y = torch.zeros_like(x)
    assert _call(L.xrl_fmm_mvm_device_noalloc, ctx, x, y) == 1      # XRL_EINVAL
    assert b"scratch" in L.xrl_last_error(ctx.h)


def test_noalloc_in_mixed_context_allocates_nothing():
    """A mixed-precision context after a solve (whose residuals built the
    FP64-accurate images): the call still runs the plain FP64 product at 64
    columns, equals xrl_fmm_mvm_device, and neither the library's allocator
    high-water mark nor the device's free memory moves across the call."""
    import torch

    import paper_2409_12375_gb300 as pkg
    from paper_2409_12375_gb300 import xrl
    L = xrl.lib()
    m = meshgen.bar()
    cx = pkg.XRL.from_mesh(m, fmm_order=7, precision=1)
    try:
        cx.solve(np.geomspace(1e3, 1e9, 12))
        rng = np.random.default_rng(5)
        for call in range(2):
            x = torch.tensor(rng.standard_normal((64, cx.n_tri)), device="cuda:0")
            y_ref = torch.empty_like(x)
            y_na = torch.full_like(x, float("nan"))
            assert _call(L.xrl_fmm_mvm_device, cx, x, y_ref) == 0
            peak0 = cx.stats()["peak_device_bytes"]
            free0 = torch.cuda.mem_get_info()[0]
            assert _call(L.xrl_fmm_mvm_device_noalloc, cx, x, y_na) == 0, L.xrl_last_error(cx.h)
            free1 = torch.cuda.mem_get_info()[0]
            assert cx.stats()["peak_device_bytes"] == peak0, call
            if call == 1:                  # the first call may still load kernel code
                assert free1 == free0
            a = y_na.cpu().numpy()
            b = y_ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12, call
    finally:
        cx.close()

