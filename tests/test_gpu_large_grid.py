"""Products on a tree with more than 65,535 leaves (Sec. II-C).

The tensor-core translations put their targets (leaves, boxes or sibling
groups) on the second grid dimension, which holds at most 65,535 blocks; past
that they launch in slices.  A 264k-panel plate under the bounding-sphere rule
(no leaf-size cap) at leaf target 4 has a uniform depth of 8 and about 132k
leaves, so the tensor-core launches of the FP32 product and of the solver's
FP64-accurate residual operator are sliced.  The FP64 product is checked on
oracle rows (half of them past the first slice), the FP32 product against it
on every row, and the FP64-accurate operator against the plain FP64 one."""
import numpy as np
import pytest

import meshgen
from oracle import panels

pytestmark = pytest.mark.gpu

LIMIT = 65535


@pytest.fixture(scope="module")
def lib():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


@pytest.fixture(scope="module")
def plate():
    return meshgen.bar(length=10e-3, width=10e-3, height=0.1e-3, n_w=256, n_h=1, n_l=256, jitter=0.0)


@pytest.fixture(scope="module")
def plate_ctx(lib, plate):
    x = lib.XRL.from_mesh(plate, fmm_order=7, leaf_target=4, mac_theta=0.5, precision=1, precond=0)
    yield x
    x.close()


def _fp32_product(ctx, x):
    import torch
    xd = torch.tensor(np.ascontiguousarray(x, np.float32), device="cuda:0")
    yd = torch.empty_like(xd)
    ctx.fmm_mvm32_device(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.float64)


def test_plate_tree_exceeds_grid_limit(plate_ctx):
    st = plate_ctx.stats()
    assert st["n_leaves"] > LIMIT + 30000, st["n_leaves"]
    assert st["n_boxes"] > 2 * LIMIT, st["n_boxes"]


def test_sliced_products_match_oracle_rows(plate_ctx, plate):
    """64 columns: the FP64 product on sampled oracle rows, half of them in
    leaves past index 65,535; then the FP32 tensor-core product (sliced M2L,
    M2M, P2M and near field) against it on every row, with the bound of the
    coil test (FP32 rounding over ~1e3-term row sums)."""
    rng = np.random.default_rng(11)
    N = plate.n_tri
    x = rng.standard_normal((64, N)).astype(np.float32).astype(np.float64)
    y64 = plate_ctx.fmm_mvm(x)
    _, perm, leaf_of = plate_ctx.export_tree()
    late = np.flatnonzero(leaf_of > LIMIT + 1000)
    early = np.flatnonzero(leaf_of < LIMIT)
    assert late.size > 1000
    rows = np.concatenate([rng.choice(late, 6, replace=False), rng.choice(early, 6, replace=False)])
    G = panels.Geometry(plate.xyz, plate.tri)
    Pr = panels.rows_P(G, rows)
    ref = x @ Pr.T
    err = np.linalg.norm(y64[:, rows] - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err
    y32 = _fp32_product(plate_ctx, x)
    nrm = np.linalg.norm(y64, axis=1)
    e32 = (np.linalg.norm(y32 - y64, axis=1) / nrm).max()
    assert e32 < 2e-5, e32
    # per-row check on the late leaves: a slice that skipped or repeated targets
    # leaves whole rows wrong while the global norm could still look small
    r32 = np.abs(y32[:, late] - y64[:, late]).max(axis=0) / np.abs(y64[:, late]).max()
    assert r32.max() < 1e-3, r32.max()


def test_sliced_fp64_accurate_operator(lib, plate, plate_ctx):
    """The solver's FP64 residual operator Z(f) v (eq. 8) at 16 systems (96
    columns: integer-slice tensor-core M2L, M2M and near field, all sliced)
    against the plain FP64 kernels, which launch with the targets on the
    first grid dimension.  Same FMM on both sides: they agree far below the
    order-7 truncation, as on the coils."""
    rng = np.random.default_rng(17)
    a = lib.XRL.from_mesh(plate, fmm_order=7, leaf_target=4, mac_theta=0.5, precision=0, precond=0)
    try:
        n = a.stats()["n_loops"]
        v = rng.standard_normal((16, n)) + 1j * rng.standard_normal((16, n))
        f = np.geomspace(1e3, 1e9, 16)
        w0 = a.apply_operator(f, v)
        w1 = plate_ctx.apply_operator(f, v)
    finally:
        a.close()
    err = np.linalg.norm(w1 - w0, axis=1) / np.linalg.norm(w0, axis=1)
    assert err.max() < 1e-10, err.max()
