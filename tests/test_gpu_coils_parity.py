"""Parity at the benchmark's workload, the two-coil sweep of Sec. III.

The chosen configuration -- mixed precision (FP32 tensor-core FMM inside FP64
FGMRES-IR), the autotuned FMM, all 2 ports x 32 frequencies in one 64-system
block (384 real product columns: the two-target tcgen05 M2L and the near field
on the context's second stream) -- is compared element by element with the
dense FP64 oracle's port R and L (tests/golden/coils_rl_*.json, written by
tests/golden/make_coils_rl.py from oracle/ only), and the full-size FP32
tensor-core product is compared with rows of the oracle's P.
"""
import json
import os

import numpy as np
import pytest

import meshgen
from oracle import panels

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = {"c2": {}, "coarse": {"step": 0.3e-3}}   # meshgen.coils arguments of each golden case
RL_TOL = 1e-4                                    # R and L within 1e-4 of the FP64 oracle


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


def _golden(case):
    with open(os.path.join(GOLDEN, "coils_rl_%s.json" % case)) as f:
        return json.load(f)


@pytest.mark.parametrize("case", ["coarse", "c2"])
def test_chosen_sweep_matches_oracle(lib, case):
    g = _golden(case)
    m = meshgen.coils(**CASES[case])
    assert m.n_tri == g["n_panels"]
    freqs = np.asarray(g["freqs_hz"])             # the oracle's own frequencies (last-ulp safe)
    assert np.allclose(m.freqs, freqs, rtol=1e-12, atol=0)
    nsys = len(freqs) * len(m.ports)
    assert nsys == 64
    x = lib.XRL.from_mesh(m, precision=1)
    try:
        leaf, order, _, perr = x.autotune(6 * nsys, 1e-6, 1)
        R, L = x.solve(freqs)
        st = x.stats()
    finally:
        x.close()
    assert perr <= 1e-6 and st["tc_targets_per_cta"] in (1, 2)
    assert st["max_rel_res"] <= 1e-8
    Ro = np.asarray(g["R"])
    Lo = np.asarray(g["L"])
    # element by element at every frequency: self terms and the mutual inductance
    for name, a, b in (("R11", R[:, 0, 0], Ro[:, 0, 0]), ("R22", R[:, 1, 1], Ro[:, 1, 1]),
                       ("L11", L[:, 0, 0], Lo[:, 0, 0]), ("L22", L[:, 1, 1], Lo[:, 1, 1]),
                       ("L12", L[:, 0, 1], Lo[:, 0, 1]), ("L21", L[:, 1, 0], Lo[:, 1, 0])):
        rel = np.abs(a - b) / np.abs(b)
        assert rel.max() <= RL_TOL, (case, name, leaf, order, rel.max(), int(np.argmax(rel)))
    # the mutual resistance is small against the self terms: bounded on their scale
    scale = np.maximum(Ro[:, 0, 0], Ro[:, 1, 1])
    assert np.max(np.abs(R[:, 0, 1] - Ro[:, 0, 1]) / scale) <= RL_TOL
    # eq. 12's diff over the sweep
    for a, b in ((R, Ro), (L, Lo)):
        diff = np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2))
        assert diff <= RL_TOL


def test_fp32_tensor_core_product_full_size_vs_oracle_rows(lib):
    """The benchmark's coils (24,792 panels) at 384 columns in the solver's
    FP32 inner product (tensor-core near field, P2M, M2M and two-target M2L at
    order 7, leaf target 32) against 16 rows of the oracle's P.  Bound 2e-5:
    FP32 rounding of row sums over ~5e3 near-field terms (~u sqrt(n) = 4e-6)
    plus the order-7 truncation (~7e-7); a wrong operand piece or layout gives
    1e-3 or worse."""
    import torch
    m = meshgen.coils()
    N = m.n_tri
    rng = np.random.default_rng(11)
    x = rng.standard_normal((384, N)).astype(np.float32)
    ctx = lib.XRL.from_mesh(m, precision=1, fmm_order=7, leaf_target=32)
    try:
        xd = torch.tensor(x, device="cuda:0")
        yd = torch.empty_like(xd)
        ctx.fmm_mvm32_device(xd, yd)
        torch.cuda.synchronize()
        y32 = yd.cpu().numpy().astype(np.float64)
        y64 = ctx.fmm_mvm(x.astype(np.float64))
    finally:
        ctx.close()
    rows = rng.choice(N, 16, replace=False)
    Pr = panels.rows_P(panels.Geometry(m.xyz, m.tri), rows)
    ref = x.astype(np.float64) @ Pr.T                      # [384, 16]
    e32 = np.linalg.norm(y32[:, rows] - ref) / np.linalg.norm(ref)
    e64 = np.linalg.norm(y64[:, rows] - ref) / np.linalg.norm(ref)
    assert e64 < 2e-6, e64                # order-7 truncation on 16 rows
    assert e32 < 2e-5, (e32, e64)
