"""Parity on the package family (Sec. III-B stand-in): the 2.8 mm crop of the
BGA-like package (perforated floating ground plane with 31 via holes, 3 x 3
solder balls, 4 traces, 2 ports; 20,700 triangles, 64 global loops) solved in
the chosen configuration -- mixed precision, autotuned FMM, the diagonal-of-P
preconditioner applied by the multigrid V-cycle (its loop matrix has no
narrow band) -- against the dense FP64 oracle (tests/golden/package_crop_rl.json)."""
import json
import os

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


def test_package_crop_sweep_matches_oracle(lib):
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "package_crop_rl.json")) as f:
        g = json.load(f)
    m = meshgen.package_crop()
    assert m.n_tri == g["n_panels"]
    freqs = np.asarray(g["freqs_hz"])
    x = lib.XRL.from_mesh(m, precision=1, precond=1, restart=150, tol=1e-7, max_iters=2000)
    try:
        x.autotune(6 * len(freqs) * len(m.ports), 1e-6, 1)
        st0 = x.stats()
        R, L = x.solve(freqs)
        st = x.stats()
    finally:
        x.close()
    assert st0["mg_levels"] >= 2 and st0["n_global_loops"] == 64   # the multigrid path, not the band
    assert st["max_rel_res"] <= 1e-7
    Ro, Lo = np.asarray(g["R"]), np.asarray(g["L"])
    for i in range(2):
        assert np.max(np.abs(R[:, i, i] - Ro[:, i, i]) / Ro[:, i, i]) <= 1e-4, i
        assert np.max(np.abs(L[:, i, i] - Lo[:, i, i]) / Lo[:, i, i]) <= 1e-4, i
    # the mutual terms are ~1% of the self terms: bounded on the self terms' scale
    sR = np.maximum(Ro[:, 0, 0], Ro[:, 1, 1])
    sL = np.maximum(Lo[:, 0, 0], Lo[:, 1, 1])
    assert np.max(np.abs(R[:, 0, 1] - Ro[:, 0, 1]) / sR) <= 1e-4
    assert np.max(np.abs(L[:, 0, 1] - Lo[:, 0, 1]) / sL) <= 1e-4
