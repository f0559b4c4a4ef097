"""Write the oracle's port R and L of the two-coil sweeps (and of the package
crop) to tests/golden/.

The coil experiment of Sec. III (two parallel square coils, self and mutual
R and L over a broadband sweep, compared by the diff of eq. 12) on the seeded
synthetic coils of `meshgen.coils`: the dense FP64 oracle (`oracle.panels`
for P by the rule table, `oracle.circuit` for the loop system of eq. 7-8 and
the port reduction) solves every frequency of the sweep directly.  Only
`oracle/` and `meshgen/` are used; nothing here touches the CUDA library.

Cases:
  c2      the benchmark's coils (two 4-turn spirals, 75 um stations,
          24,792 triangles, 2 ports, 32 frequencies 100 Hz - 10 GHz);
          about 45 minutes and 35 GB of host memory on 8 cores
  coarse  the same coils at 300 um stations (6,488 triangles), minutes
  package_crop  a 2.8 x 2.8 mm window of the BGA-like package family
          (meshgen.package_crop: 20,700 triangles, 14 conductors, 31 via
          holes, 2 ports, 16 frequencies 1 MHz - 5 GHz); written to
          package_crop_rl.json

  python tests/golden/make_coils_rl.py c2 coarse package_crop [--workers 8]

P is filled by oracle.panels.dense_P_parallel (the rows of its upper
triangle spread over a process pool, each entry by pair_values as in
dense_P).
"""
import argparse
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CASES = {"c2": {}, "coarse": {"step": 0.3e-3}, "package_crop": None}


def run(case, workers):
    import meshgen
    from oracle import circuit, panels
    params = CASES[case]
    m = meshgen.package_crop() if params is None else meshgen.coils(**params)
    t0 = time.perf_counter()
    P = panels.dense_P_parallel(m.xyz, m.tri, workers)
    t1 = time.perf_counter()
    c = circuit.Circuit(m, sparse=True)
    R, L, _ = c.solve(m.freqs, P)
    t2 = time.perf_counter()
    out = {
        "what": "oracle port R (ohm) and L (H) of the seeded sweep, R[f][q][p], L[f][q][p]",
        "case": case, "meshgen_call": ("meshgen.package_crop()" if params is None else
                                       "meshgen.coils(%s)" % ", ".join("%s=%r" % kv for kv in params.items())),
        "n_panels": int(m.n_tri), "n_loops": int(c.M.shape[0]), "n_ports": len(m.ports),
        "freqs_hz": [float(f) for f in m.freqs],
        "R": np.asarray(R).tolist(), "L": np.asarray(L).tolist(),
        "oracle_seconds": {"P": t1 - t0, "loop_solve": t2 - t1, "total": t2 - t0},
        "host": {"cores_used": workers, "machine": platform.machine(), "cpu_count": os.cpu_count()},
        "command": "python tests/golden/make_coils_rl.py %s --workers %d" % (case, workers),
    }
    name = "package_crop_rl.json" if params is None else "coils_rl_%s.json" % case
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote %s: N=%d loops=%d, %.0f s (P %.0f s, solve %.0f s)"
          % (path, m.n_tri, c.M.shape[0], t2 - t0, t1 - t0, t2 - t1), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="+", choices=sorted(CASES))
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    for case in a.cases:
        run(case, a.workers)


if __name__ == "__main__":
    main()
