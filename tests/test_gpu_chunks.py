"""Frequency-chunked sweeps (xrl_options.rhs_chunk) and the previous-frequency
start (warm_start = 1): the chunks of the coarse two-coil sweep reproduce the
dense oracle's R and L (tests/golden/coils_rl_coarse.json) to 1e-4, and
starting each chunk from the previous chunk's last frequency does not cost
iterations."""
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


def test_chunked_sweep_matches_oracle_and_warm_start_helps(lib):
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "coils_rl_coarse.json")) as f:
        g = json.load(f)
    m = meshgen.coils(step=0.3e-3)
    freqs = np.asarray(g["freqs_hz"])
    Ro, Lo = np.asarray(g["R"]), np.asarray(g["L"])
    iters = {}
    for ws in (0, 1):
        x = lib.XRL.from_mesh(m, precision=1, fmm_order=7, rhs_chunk=16, warm_start=ws)
        try:
            R, L = x.solve(freqs)
            st = x.stats()
        finally:
            x.close()
        iters[ws] = st["total_iters"]
        assert st["max_rel_res"] <= 1e-8
        for a, b in ((R[:, 0, 0], Ro[:, 0, 0]), (R[:, 1, 1], Ro[:, 1, 1]), (L[:, 0, 0], Lo[:, 0, 0]),
                     (L[:, 1, 1], Lo[:, 1, 1]), (L[:, 0, 1], Lo[:, 0, 1])):
            assert np.max(np.abs(a - b) / np.abs(b)) <= 1e-4, ws
    assert iters[1] <= iters[0], iters
