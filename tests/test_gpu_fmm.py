"""GPU parity of the tree, the direct sum and the FMM product y = P x
(Sec. II-C) against the CPU oracle, through the C-ABI."""
import numpy as np
import pytest

import meshgen
from oracle import panels, tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


@pytest.fixture(scope="module")
def bar_ctx(lib, bar_mesh):
    x = lib.XRL.from_mesh(bar_mesh, fmm_order=8)
    yield x
    x.close()


@pytest.fixture(scope="module")
def coils_mesh():
    return meshgen.coils()


@pytest.fixture(scope="module")
def coils_ctx(lib, coils_mesh):
    x = lib.XRL.from_mesh(coils_mesh, fmm_order=8)
    yield x
    x.close()


def _check_tree(ctx, mesh):
    if ctx.opts.mac_theta > 0:
        ref = tree.build_mac(mesh.xyz, mesh.tri, leaf_target=ctx.opts.leaf_target, theta=ctx.opts.mac_theta,
                             cap=0.0)
    else:
        ref = tree.build(mesh.xyz, mesh.tri, leaf_target=ctx.opts.leaf_target, ws=ctx.opts.separation)
    keys, perm, leaf = ctx.export_tree()
    assert np.array_equal(keys, ref["keys"])
    assert np.array_equal(perm, ref["perm"])
    assert np.array_equal(leaf, ref["leaf_of"])
    st = ctx.stats()
    assert st["n_levels"] == ref["L"] + 1
    for lev in range(2, ref["L"] + 1):
        bk, vptr, vsrc, uptr, usrc = ctx.export_lists(lev)
        assert np.array_equal(bk, ref["levels"][lev])
        for b, lst in enumerate(ref["V"][lev]):
            assert list(vsrc[vptr[b]:vptr[b + 1]]) == lst
        if lev == ref["L"]:
            for b, lst in enumerate(ref["U"]):
                assert list(usrc[uptr[b]:uptr[b + 1]]) == lst


def test_tree_bit_exact_bar(bar_ctx, bar_mesh):
    _check_tree(bar_ctx, bar_mesh)


def test_tree_bit_exact_coils(coils_ctx, coils_mesh):
    _check_tree(coils_ctx, coils_mesh)


@pytest.mark.parametrize("opts", [dict(mac_theta=0.0, separation=1), dict(mac_theta=0.66, leaf_target=32),
                                  dict(mac_theta=0.5, leaf_target=16)])
def test_tree_bit_exact_other_rules(lib, coils_mesh, opts):
    """The cell-distance rule at ws = 1 and the bounding-sphere rule."""
    x = lib.XRL.from_mesh(coils_mesh, **opts)
    try:
        _check_tree(x, coils_mesh)
    finally:
        x.close()


def test_bounding_sphere_lists_cut_the_near_field(lib, coils_mesh):
    """Bounding-sphere rule at theta = 0.6 without the leaf-size cap (leaf
    target 32): the near field drops below 450 entries per panel (the
    cell-distance rule with its cap holds ~2,060) and the FP64 product at
    order 8 stays within 1e-6 of the direct sum."""
    import torch
    x = lib.XRL.from_mesh(coils_mesh, mac_theta=0.6, leaf_target=32, fmm_order=8)
    try:
        st = x.stats()
        assert st["near_nnz"] / st["n_panels"] < 450, st["near_nnz"] / st["n_panels"]
        rng = np.random.default_rng(8)
        xv = _dev(rng.standard_normal((2, coils_mesh.n_tri)))
        yd = torch.empty_like(xv)
        yf = torch.empty_like(xv)
        x.direct_mvm_device(xv, yd)
        x.fmm_mvm_device(xv, yf)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(yf - yd) / torch.linalg.norm(yd))
    finally:
        x.close()
    assert err < 1e-6, err


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


def test_direct_sum_matches_dense_oracle(bar_ctx, bar_dense_P):
    import torch
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, bar_dense_P.shape[0]))
    xd = _dev(x)
    yd = torch.empty_like(xd)
    bar_ctx.direct_mvm_device(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = x @ bar_dense_P.T
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12
    assert np.max(np.abs(y - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("nc", [1, 6, 13])
def test_fmm_matches_dense_oracle(bar_ctx, bar_dense_P, nc):
    import torch
    rng = np.random.default_rng(nc)
    x = rng.standard_normal((nc, bar_dense_P.shape[0]))
    xd = _dev(x)
    yd = torch.empty_like(xd)
    bar_ctx.fmm_mvm_device(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = x @ bar_dense_P.T
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err


def test_fmm_host_entry_equals_device_entry(bar_ctx):
    import torch
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, bar_ctx.n_tri))
    yh = bar_ctx.fmm_mvm(x)
    xd = _dev(x)
    yd = torch.empty_like(xd)
    bar_ctx.fmm_mvm_device(xd, yd)
    torch.cuda.synchronize()
    # at <= 8 columns the M2L accumulates with atomics: equal up to rounding order
    yv = yd.cpu().numpy()
    assert np.max(np.abs(yh - yv)) <= 1e-13 * np.max(np.abs(yh))


def test_fmm_zero_and_linearity(bar_ctx):
    z = bar_ctx.fmm_mvm(np.zeros(bar_ctx.n_tri))
    assert np.all(z == 0.0)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal((2, bar_ctx.n_tri))
    y = bar_ctx.fmm_mvm(np.stack([a, b, 2.0 * a - 3.0 * b]))
    lin = 2.0 * y[0] - 3.0 * y[1]
    assert np.max(np.abs(y[2] - lin)) < 1e-12 * np.max(np.abs(y[2]))


def test_fmm_full_size_coils_sampled_rows(coils_ctx, coils_mesh):
    """~25k-panel coils at 6 columns (one complex system): sampled rows of
    the oracle's P times x."""
    rng = np.random.default_rng(5)
    N = coils_mesh.n_tri
    x = rng.standard_normal((6, N))
    y = coils_ctx.fmm_mvm(x)
    rows = rng.choice(N, 12, replace=False)
    G = panels.Geometry(coils_mesh.xyz, coils_mesh.tri)
    Pr = panels.rows_P(G, rows)
    ref = x @ Pr.T                       # [6, rows]
    got = y[:, rows]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err


# ---- FP32 product of the inner iterations (tensor-core M2L and CUDA-core M2L) ----------
# Tolerance: FP32 unit roundoff 6e-8 grown over sums of ~1e3-1e4 terms (near-field
# rows, 81-term translations over ~100 V-list entries) gives a few 1e-7; the order-8
# truncation adds ~1e-7.  2e-6 leaves an order of magnitude over what a correct
# kernel reaches while a wrong operand layout or split gives O(1e-3) or worse.
FP32_TOL = 2e-6


def _fp32_product(ctx, x):
    import torch
    xd = torch.tensor(np.ascontiguousarray(x, np.float32), device="cuda:0")
    yd = torch.empty_like(xd)
    ctx.fmm_mvm32_device(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def bar_ctx_scalar(lib, bar_mesh):
    x = lib.XRL.from_mesh(bar_mesh, fmm_order=8, tensor_cores=0)
    yield x
    x.close()


@pytest.mark.parametrize("nc", [1, 40, 64, 200, 384])
def test_fp32_product_matches_dense_oracle(bar_ctx, bar_ctx_scalar, bar_dense_P, nc):
    """nc >= 64 takes the tcgen05 M2L on the default context (ragged last
    128-column tile at 200); the scalar context runs the CUDA-core kernels."""
    rng = np.random.default_rng(100 + nc)
    x = rng.standard_normal((nc, bar_dense_P.shape[0])).astype(np.float32).astype(np.float64)
    ref = x @ bar_dense_P.T
    for ctx in (bar_ctx, bar_ctx_scalar):
        y = _fp32_product(ctx, x)
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err < FP32_TOL, (ctx.opts.tensor_cores, err)


@pytest.mark.parametrize("p", [8, 7])
def test_fp32_tensor_core_m2l_full_size_coils(coils_ctx, coils_mesh, lib, p):
    """Coils (24,792 panels) at 384 columns, the launch configuration of the
    solver's 64-system block: the tensor-core FP32 product against the FP64
    product (itself checked on sampled oracle rows above), column by column.
    With random-sign x the FP32 error of a row sum is ~u sqrt(n) |y|-relative
    (n ~ 5e3 near-field terms: ~4e-6), so the bound here is 2e-5 and the
    tensor-core path must be no worse than 1.5x the CUDA-core FP32 path.
    At order 7 (64 coefficients) the M2L runs two sibling targets per CTA."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal((384, coils_mesh.n_tri)).astype(np.float32).astype(np.float64)
    ctx = coils_ctx if p == 8 else lib.XRL.from_mesh(coils_mesh, fmm_order=p)
    sc = lib.XRL.from_mesh(coils_mesh, fmm_order=p, tensor_cores=0)
    try:
        y64 = ctx.fmm_mvm(x)
        y32 = _fp32_product(ctx, x)
        ys = _fp32_product(sc, x)
    finally:
        sc.close()
        if ctx is not coils_ctx:
            ctx.close()
    nrm = np.linalg.norm(y64, axis=1)
    e_tc = (np.linalg.norm(y32 - y64, axis=1) / nrm).max()
    e_sc = (np.linalg.norm(ys - y64, axis=1) / nrm).max()
    assert e_tc < 2e-5 and e_sc < 2e-5, (e_tc, e_sc)
    assert e_tc < 1.5 * e_sc, (e_tc, e_sc)


@pytest.mark.parametrize("p", [6, 7])
def test_fp32_product_lower_orders(lib, bar_mesh, bar_dense_P, p):
    """Orders 6 and 7 (49 and 64 coefficients: the 64-wide tensor-core tiles)
    at 200 columns: the FP32 product's error against the dense oracle exceeds
    the same order's FP64 product error by at most the FP32 bound above."""
    ctx = lib.XRL.from_mesh(bar_mesh, fmm_order=p)
    try:
        rng = np.random.default_rng(200 + p)
        x = rng.standard_normal((200, bar_dense_P.shape[0])).astype(np.float32).astype(np.float64)
        ref = x @ bar_dense_P.T
        e64 = np.linalg.norm(ctx.fmm_mvm(x) - ref) / np.linalg.norm(ref)
        e32 = np.linalg.norm(_fp32_product(ctx, x) - ref) / np.linalg.norm(ref)
    finally:
        ctx.close()
    assert e64 < 1e-4 and e32 < e64 + FP32_TOL, (e64, e32)
