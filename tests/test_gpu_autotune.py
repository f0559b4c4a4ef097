"""GPU tests of the FMM autotuner (xrl_autotune): the chosen leaf size and
expansion order meet the accuracy bound against the oracle's dense P
(Sec. II-C), the tree it leaves matches the oracle's tree for those options,
the solver still reproduces R and L, and an unreachable bound is reported."""
import numpy as np
import pytest

from oracle import tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


def test_autotune_meets_bound_and_keeps_parity(lib, bar_mesh, bar_dense_P):
    x = lib.XRL.from_mesh(bar_mesh, precision=1)
    try:
        leaf, order, ms, err = x.autotune(n_cols=6, mvm_tol=1e-6, precision=1)
        assert leaf in (16, 32, 64) and order in (6, 7, 8)
        assert 0.0 <= err <= 1e-6 and ms > 0.0
        assert x.stats()["tc_targets_per_cta"] in (1, 2)
        # the context is left set up with the choice: tree and product parity
        ref = tree.build(bar_mesh.xyz, bar_mesh.tri, leaf_target=leaf, ws=2)
        keys, perm, _ = x.export_tree()
        assert np.array_equal(keys, ref["keys"]) and np.array_equal(perm, ref["perm"])
        rng = np.random.default_rng(5)
        v = rng.standard_normal((3, bar_dense_P.shape[0]))
        y = x.fmm_mvm(v)
        yr = v @ bar_dense_P.T
        assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-6
        # the solver on the tuned context agrees with an untuned one
        f = np.array([1e3, 1e8])
        R, L = x.solve(f)
        y0 = lib.XRL.from_mesh(bar_mesh, precision=1)
        try:
            R0, L0 = y0.solve(f)
        finally:
            y0.close()
        assert np.max(np.abs(R - R0) / np.abs(R0)) < 1e-4
        assert np.max(np.abs(L - L0) / np.abs(L0)) < 1e-4
    finally:
        x.close()


def test_autotune_unreachable_bound(lib, bar_mesh, bar_dense_P):
    x = lib.XRL.from_mesh(bar_mesh)
    try:
        with pytest.raises(lib.XRLError) as e:
            x.autotune(n_cols=2, mvm_tol=1e-15)
        assert e.value.code == 5
        # left set up with the most accurate candidate: still a valid product
        rng = np.random.default_rng(6)
        v = rng.standard_normal(bar_dense_P.shape[0])
        y = x.fmm_mvm(v)
        yr = bar_dense_P @ v
        assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-6
    finally:
        x.close()


def test_autotune_targets_per_cta_keeps_parity(lib, bar_mesh, bar_dense_P):
    """At 64 columns (the tensor-core paths) the autotuner also chooses one or
    two sibling targets per CTA; the FP32 product of the chosen configuration
    matches the oracle within the FP32 bound either way."""
    import torch
    x = lib.XRL.from_mesh(bar_mesh, precision=1)
    try:
        leaf, order, ms, err = x.autotune(n_cols=64, mvm_tol=1e-6, precision=1)
        t = x.stats()["tc_targets_per_cta"]
        assert t in (1, 2)
        rng = np.random.default_rng(8)
        v = rng.standard_normal((64, bar_dense_P.shape[0])).astype(np.float32)
        xd = torch.tensor(v, device="cuda:0")
        yd = torch.empty_like(xd)
        x.fmm_mvm32_device(xd, yd)
        torch.cuda.synchronize()
        ref = v.astype(np.float64) @ bar_dense_P.T
        e32 = np.linalg.norm(yd.cpu().numpy().astype(np.float64) - ref) / np.linalg.norm(ref)
        e64 = np.linalg.norm(x.fmm_mvm(v.astype(np.float64)) - ref) / np.linalg.norm(ref)
        assert e32 < e64 + 2e-6, (t, e32, e64)
    finally:
        x.close()
