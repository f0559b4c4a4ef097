#!/usr/bin/env python3
"""Benchmark of the broadband R/L sweep on GB300.

Workload (default): two stacked 4-turn square planar copper coils, 24,792
triangles, 2 ports x 32 log-spaced frequencies from 100 Hz to 10 GHz, all 64
(frequency, port) systems solved as one multi-RHS block to a relative residual
of 1e-8.  The FMM's leaf size and order come from the library's autotuner
(untimed, before the warm-up): the fastest product at the sweep's column
count whose FP64 product stays within 1e-6 of the direct sum.  One STEP = one
full sweep (FMM products, preconditioner, FGMRES, port reduction to R and L).
The metric is seconds per (frequency, port) solve (lower is better); FMM
product throughput in panel-columns per second is reported beside it.

Arms, each autotuned for its own precision and timed the same way (W warm-up
sweeps, then K sweeps between CUDA events on the context's stream):
  chosen      mixed precision (FP32 tensor-core FMM inside FP64 FGMRES-IR)
  fp64_tc     FP64-accurate products throughout on the tensor cores and FP32
              pipes (integer-slice M2L/M2M/near field, double-float P2M/L2P),
              no FP32 inner iterations
  plain_fp64  FP64 CUDA-core kernels throughout

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--no-autotune --fmm-order P --leaf-target L]
  python bench.py --impl reference     # the CPU oracle on a bounded sample

Under torchrun each rank solves its own frequency chunk of an N-times longer
sweep (weak scaling, no collective on the data path); the step time is the
maximum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per (freq,port) solve & FMM MVM panels/s: chosen vs plain FP64, RL err<=1e-4"
UNIT = "s/(freq*port)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison step")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the preconditioner comparison (diagonal-of-P vs diagonal-of-L, untimed)")
    ap.add_argument("--fmm-order", type=int, default=None,
                    help="expansion order p of the FMM with --no-autotune (default 7: the autotuner's choice on the "
                         "coils)")
    ap.add_argument("--leaf-target", type=int, default=None,
                    help="target panels per octree leaf (default 32; 64 on the PoP stack)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --fmm-order/--leaf-target as given instead of xrl_autotune's choice (FP64 product "
                         "within 1e-6 of the direct sum, fastest inner product at the sweep's column count); the "
                         "PoP stack never autotunes (one setup per candidate is 1.5 min there)")
    ap.add_argument("--workload", default="pop", choices=["coils", "package", "package_crop", "pop"],
                    help="pop (default): the package-on-package stack (~2.1M triangles, 16 ports), the largest "
                         "configuration that fits one GPU, at --freqs of its 64 frequencies; coils: the two-coil "
                         "sweep (2 ports x 32 freqs, one 64-RHS block) with the comparison arms; package: the "
                         "BGA-like package (~250k triangles, 8 ports x 16 freqs); package_crop: its 2.8 mm window")
    ap.add_argument("--restart", type=int, default=None, help="FGMRES restart of the package workloads "
                                                              "(default 150; 100 on the PoP stack)")
    ap.add_argument("--tol", type=float, default=1e-6, help="relative residual of the package workloads")
    ap.add_argument("--freqs", type=int, default=None,
                    help="package workloads: solve the first N frequencies of the sweep (default: all; 2 on the PoP "
                         "stack: 1 kHz and 1.29 kHz, one 16-system chunk each)")
    ap.add_argument("--spread", action="store_true",
                    help="with --freqs: N frequencies spread evenly over the sweep, both ends included, instead of "
                         "the first N")
    ap.add_argument("--fp64tc-arm", action="store_true", help="package workloads: one FP64-accurate sweep too")
    ap.add_argument("--precond-ablation", action="store_true",
                    help="package workloads: one more sweep (untimed by the bench clock) with the diagonal-of-L "
                         "preconditioner, against the chosen diagonal-of-P (Table IV's comparison)")
    ap.add_argument("--chunk", type=int, default=None, help="package workloads: systems per frequency chunk when "
                                                             "the sweep has more than 128 (default 64; 16 on the "
                                                             "PoP stack)")
    ap.add_argument("--mac", type=float, default=None, help="package workloads: bounding-sphere separation theta "
                                                            "(0: the cell-distance rule; default 0, 0.6 on the PoP "
                                                            "stack)")
    ap.add_argument("--sweep-case", action="store_true",
                    help="profiling case: one warm-up and one timed sweep of the coils at --fmm-order/--leaf-target "
                         "(mixed precision), no autotune, no comparison arms")
    ap.add_argument("--kernel-case", action="store_true",
                    help="profiling case: only the FMM products of one sweep's launch configuration "
                         "(FP32 inner product and the mixed mode's FP64 residual operator, 64 systems), 3 each")
    a = ap.parse_args()
    pop = a.workload == "pop" and not (a.sweep_case or a.kernel_case)
    for k, v in (("fmm_order", 7), ("leaf_target", 64 if pop else 32), ("restart", 100 if pop else 150),
                 ("freqs", 2 if pop else 0), ("chunk", 16 if pop else 64), ("mac", 0.6 if pop else 0.0)):
        if getattr(a, k) is None:
            setattr(a, k, v)
    if pop:
        a.no_autotune = True
    return a


def spread(freqs, n, world=1, rank=0, even=False):
    """n * world frequencies of a sweep, the first ones or (even) spread evenly
    over it with both ends included; rank r takes every world-th of them (weak
    scaling: n per rank)."""
    freqs = np.asarray(freqs)
    if not n:
        return freqs[rank::world]
    k = min(len(freqs), n * world)
    if even:
        idx = np.unique(np.round(np.linspace(0, len(freqs) - 1, k)).astype(int))
        return freqs[idx][rank::world]
    return freqs[:k][rank::world]


# ---------------------------------------------------------------- workload
def workload(rank=0, world=1):
    import meshgen
    m = meshgen.coils()
    # weak scaling: rank r takes every world-th frequency of a world-times longer sweep
    allf = np.geomspace(100.0, 1e10, 32 * world)
    m.freqs = allf[rank::world]
    return m


def gather_sweep(R, L, world):
    """R, L of the whole sweep on every rank, in frequency order: rank r
    solved frequencies r, r + world, ... of the longer sweep (workload())."""
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, (np.asarray(R), np.asarray(L)))
    nf = sum(p[0].shape[0] for p in parts)
    Ra = np.empty((nf,) + parts[0][0].shape[1:])
    La = np.empty_like(Ra)
    for r, (Rr, Lr) in enumerate(parts):
        Ra[r::world] = Rr
        La[r::world] = Lr
    return Ra, La


def config_dict(m, precision, opts):
    return {"workload": "two 4-turn square planar copper coils, %d triangles, 2 ports x %d freqs "
                        "(100 Hz-10 GHz), one 64-RHS block, tol 1e-8" % (m.n_tri, len(m.freqs)),
            "n_panels": int(m.n_tri), "n_ports": 2, "n_freqs": int(len(m.freqs)),
            "precision": precision, "fmm_order": opts["fmm_order"], "separation": opts["separation"],
            "leaf_target": opts["leaf_target"], "tol": 1e-8,
            "l2": "working set > L2 (near field + expansions + Krylov basis, several GB): no flush needed"}


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(m, n_loops, budget_rows=24):
    """Time the CPU oracle on a bounded sample of this workload and scale it to
    seconds per (frequency, port) solve of the full workload.

    The oracle's dense direct path is: P by the rule table (N^2/2 entries),
    G = sum_t (M A_t) P (M A_t)^T (real GEMMs), then one dense complex LU
    solve of the n_loops x n_loops loop system per frequency.  Sample: P rows
    for `budget_rows` random panels with the oracle's own rule table, and the
    oracle's two library primitives (np.matmul real, np.linalg.solve complex)
    at n = 2048; each measured rate is scaled to the full sizes.  n_loops is
    the loop count of this mesh (the cycle-space dimension, the same for the
    oracle's fundamental cycles and the library's basis)."""
    from oracle import panels
    G = panels.Geometry(m.xyz, m.tri)
    N = G.n
    rng = np.random.default_rng(0)
    rows = rng.choice(N, budget_rows, replace=False)
    t0 = time.perf_counter()
    panels.rows_P(G, rows)
    t_rows = time.perf_counter() - t0
    t_entry = t_rows / (budget_rows * N)
    n = 2048
    a = rng.standard_normal((n, n))
    t0 = time.perf_counter()
    a @ a
    gemm_rate = 2.0 * n ** 3 / (time.perf_counter() - t0)
    z = a + 1j * rng.standard_normal((n, n)) + n * np.eye(n)
    bb = np.ones((n, 2), complex)
    t0 = time.perf_counter()
    np.linalg.solve(z, bb)
    lu_time = time.perf_counter() - t0
    n_live = int(np.sum(np.asarray(m.term) < 0))
    n_f = len(m.freqs)
    n_p = len(m.ports)
    t_P = t_entry * N * N / 2.0
    # G and the per-material resistive matrix: 3 x (MA P, (MA P) MA^T, (MA w) MA^T)
    t_G = 3 * (2.0 * n_loops * n_live * n_live + 4.0 * n_loops * n_loops * n_live) / gemm_rate
    t_LU = n_f * lu_time * (n_loops / n) ** 3
    total = t_P + t_G + t_LU
    return {"value": total / (n_f * n_p), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": ("oracle P rows for %d random panels (%.1f s, %.3g s/entry, scaled to N^2/2 = %.3g "
                       "entries), np.matmul and np.linalg.solve (the oracle's G and LU primitives) at n=2048 "
                       "scaled to n_loops=%d, %d frequencies; estimated full oracle solve %.0f s "
                       "(P %.0f s, G %.0f s, LU %.0f s)" % (budget_rows, t_rows, t_entry, N * N / 2.0,
                                                          n_loops, n_f, total, t_P, t_G, t_LU)),
            "measured_s": t_rows + lu_time, "estimated_total_s": total}


def oracle_c1_full():
    """The full oracle on the small case (the 2,100-triangle bar, 1 port, 4
    frequencies) timed for real: P by the rule table over every host core
    (process pool), the fundamental-cycle loop system and its dense solves."""
    import meshgen
    from oracle import circuit, panels
    m = meshgen.bar()
    w = os.cpu_count() or 1
    t0 = time.perf_counter()
    P = panels.dense_P_parallel(m.xyz, m.tri, w)
    t1 = time.perf_counter()
    circuit.Circuit(m).solve(m.freqs, P)
    t2 = time.perf_counter()
    return {"workload": "bar 1x1x10 mm, %d triangles, 1 port x %d freqs" % (m.n_tri, len(m.freqs)),
            "s_per_freq_port": (t2 - t0) / len(m.freqs), "total_s": t2 - t0, "P_s": t1 - t0,
            "solve_s": t2 - t1, "cores": w}


def oracle_c2_recorded():
    """The full oracle's time on the benchmark's coils, measured once by
    tests/golden/make_coils_rl.py (its host is named in the record)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "coils_rl_c2.json")) as f:
            g = json.load(f)
    except Exception:
        return None
    nsys = len(g["freqs_hz"]) * g["n_ports"]
    return {"s_per_freq_port": g["oracle_seconds"]["total"] / nsys, "total_s": g["oracle_seconds"]["total"],
            "host": g["host"], "command": g["command"]}


# ---------------------------------------------------------------- peaks
def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except Exception:
        pass
    sm_max = float(p.get("sm_max_mhz", 2070.0))
    return {
        "hbm_gbs": float(p.get("hbm_gbs", 6800.0)),
        "hbm_src": "measured (MEASURED_PEAKS.json)" if "hbm_gbs" in p else "fallback",
        # FP32 SIMT peak from unit counts and the maximum SM clock: 152 SMs x
        # 128 FP32 lanes x 2 flops
        "fp32_tflops": 152 * 128 * 2 * sm_max * 1e6 / 1e12,
        "bf16_sust": float(p.get("bf16_tflops_sustained", 1700.0)),
        "bf16_src": "measured bf16 sustained (MEASURED_PEAKS.json)" if "bf16_tflops_sustained" in p
        else "fallback",
    }


def measure_fp64_peak():
    """FP64 rate of this GPU, measured: the best of 5 cuBLAS DGEMMs (torch.matmul,
    float64, 8192^3) timed with CUDA events."""
    import torch
    n = 8192
    a = torch.randn(n, n, device="cuda", dtype=torch.float64)
    b = torch.randn(n, n, device="cuda", dtype=torch.float64)
    c = a @ b
    best = None
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


# ---------------------------------------------------------------- rooflines
# ncu DRAM bytes (read + write) per launch of the dominant kernels at one
# configuration: (order, stored near-field entries (the tree), targets per CTA,
# columns) -> {phase: bytes}.  Reported only when the bench runs that
# configuration with the kernels the counters were taken of; on the coils the
# leaf targets 16, 32 and 64 give the same tree.
NCU_TRAFFIC = {(7, 51031728, 2, 384): {"m2l": 56.103168e6 + 21.513216e6,     # k_xlate_tc2<0>
                                        "p2p": 437.047552e6 + 32.495872e6}}   # k_xlate_tc2<1>


def m2l_products(p, targets):
    """Tensor-core products per algorithmic flop of the FP32 M2L: the two-target
    kernel (64-coefficient tiles) runs 2-piece FP16 operands, 3 products; the
    one-target kernel 3-piece BF16, 6 products."""
    np_ = ((p + 1) ** 2 + 15) // 16 * 16
    return 3 if (np_ == 64 and targets == 2) else 6


def phase_kernel(name, p, targets=2):
    """Kernels behind a profiling phase of the mixed-precision sweep at order p."""
    np_ = ((p + 1) ** 2 + 15) // 16 * 16
    tc = "k_xlate_tc<%d>" % (64 if np_ <= 64 else 96)
    return {
        "p2p": "k_tcp_pack_x + k_xlate_tc2<1> (tcgen05 near field, two sibling leaves per CTA, 3-piece BF16)",
        "m2l": ("k_tch_pack_a + k_xlate_tc2<0> (tcgen05, two sibling targets per CTA, N = 128, 2-piece FP16, "
                "3 products)" if m2l_products(p, targets) == 3 else
                "k_tc_pack_a + %s (tcgen05, one target per CTA, 3-piece BF16, 6 products)" % tc),
        "p2m": tc + " mode 2 (tcgen05 P2M from the near field's transposed-X image) + k_p2m_df64 (residuals)",
        "m2m": "k_tc_pack_a + " + tc + " mode 0 over the 8 M2M tables (tcgen05) + k_m2l_df64<0> (residuals)",
        "p2p64": "k_ozp_pack_x + k_xlate_oz (tcgen05 near field, 5 integer slices)",
        "m2l64": "k_oz_pack_a + k_xlate_oz (tcgen05, 5 integer slices, 15 products)",
        "precond": "k_spike_y/z/x/out apply + k_band_factor_blk/k_spike_cols/k_spike_reduce factor",
        "operator": "k_gather + k_scatter + k_loop_reduce(_long)",
        "l2p": "k_l2p_tiled + k_l2p_df64 (residuals)",
        "l2l": "k_m2l_tiled<%d,1> list form + k_m2l_df64<1> (residuals)" % ((np_ + 15) // 16)}.get(name, name)


def phase_roofline(name, d, pk, precision, p, nc, near_pad=0.0, traffic=None, targets=2):
    """Roofline entry of one profiling phase: ALGORITHMIC flops (or bytes) per
    launch over the phase's CUDA-event time per launch, against the peak of the
    unit that executes them.  For the tensor-core phases the FP32 (or
    FP64-accurate) contraction runs as several BF16 products; the rate of
    those issued products is reported beside it, not as `achieved`."""
    avg_ms = d["ms"] / max(1, d["launches"])
    mixed = precision == "mixed"
    alg = d["flops"] / (d["ms"] * 1e-3) / 1e12          # algorithmic TFLOP/s
    out = {"kernel": phase_kernel(name, p, targets), "avg_launch_ms": avg_ms, "launches": d["launches"],
           "traffic": traffic.get(name) if traffic else None}
    ncoef = (p + 1) ** 2
    pad = lambda v: (v + 15) // 16 * 16
    tile_pad = (pad(ncoef) * pad(ncoef)) / float(ncoef * ncoef) * (128 * ((nc + 127) // 128)) / float(nc)
    col_pad = (128 * ((nc + 127) // 128)) / float(nc)
    if mixed and (name in ("m2l", "m2l64") or (name in ("p2p", "p2p64") and near_pad > 0)):
        products = m2l_products(p, targets) if name == "m2l" else (6 if name == "p2p" else 15)
        padf = tile_pad if name.startswith("m2l") else near_pad * col_pad
        issued = alg * products * padf                    # BF16 MMA TFLOP/s actually issued
        out.update({"bound": "tensor", "achieved": alg, "peak": pk["bf16_sust"], "unit": "TFLOP/s",
                    "frac": alg / pk["bf16_sust"], "peak_src": pk["bf16_src"],
                    "issued_mma_tflops": issued, "issued_frac": issued / pk["bf16_sust"],
                    "note": "achieved = algorithmic FP%s flops/s; the tensor pipe issues %d 16-bit products x "
                            "padding %.3f per algorithmic flop" % ("32" if name in ("m2l", "p2p") else "64",
                                                                   products, padf)})
    elif name in ("precond", "operator"):
        gbs = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / pk["hbm_gbs"], "peak_src": pk["hbm_src"],
                    "note": "latency-bound chains (sequential substitutions); bytes are algorithmic"
                    if name == "precond" else "gathers over the loop matrix"})
    else:
        fp64 = not mixed or name.endswith("64")
        peak = pk["fp64_tflops"] if fp64 else pk["fp32_tflops"]
        if mixed and fp64:
            # FP64-accurate work on the FP32 pipes (double-float): ~11 FP32 operations per multiply-add
            peak = pk["fp32_tflops"] * 2.0 / 11.0
            src = "derived: FP32 SIMT peak x 2/11 (double-float multiply-add on the FP32 pipes)"
        else:
            src = pk["fp64_src"] if fp64 else "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"
        out.update({"bound": "alu", "achieved": alg, "peak": peak, "unit": "TFLOP/s", "frac": alg / peak,
                    "peak_src": src})
    return out


def product_roofline(flops, byts, ms, pk):
    """FP64 product: algorithmic flops and bytes over its event time, against
    the measured FP64 rate and HBM bandwidth; `frac` is that of the binding one
    (the larger of the two lower bounds on the time)."""
    tf = flops / (ms * 1e-3) / 1e12
    gbs = byts / (ms * 1e-3) / 1e9
    ff, fb = tf / pk["fp64_tflops"], gbs / pk["hbm_gbs"]
    return {"achieved_tflops": tf, "peak_tflops": pk["fp64_tflops"], "flop_frac": ff,
            "achieved_gbs": gbs, "peak_gbs": pk["hbm_gbs"], "hbm_frac": fb,
            "bound": "fp64" if ff >= fb else "hbm", "frac": max(ff, fb), "ms": ms,
            "algorithmic_gflop": flops / 1e9, "algorithmic_gb": byts / 1e9, "peak_src": pk["fp64_src"]}


# ---------------------------------------------------------------- reference arm
def loop_count(m):
    """Dimension of the loop space of a mesh's PEEC graph (branches - nodes +
    connected components): nodes are the live panels and one node per
    terminal, branches the edges between two live panels, the rim edges from
    a live panel to a terminal, and one external branch per port."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    tri = np.asarray(m.tri)
    term = np.asarray(m.term)
    e, own = [], []
    for k in range(tri.shape[1]):
        a_ = tri[:, k]
        b_ = tri[:, (k + 1) % tri.shape[1]]
        if tri.shape[1] == 4:      # hybrid panels: a triangle's 4th slot is -1
            b_ = np.where(b_ < 0, tri[:, 0], b_)
            ok = a_ >= 0
        else:
            ok = np.ones(tri.shape[0], bool)
        e.append(np.sort(np.stack([a_[ok], b_[ok]], 1), axis=1))
        own.append(np.flatnonzero(ok))
    e = np.vstack(e)
    own = np.concatenate(own)
    _, inv = np.unique(e, axis=0, return_inverse=True)
    order = np.argsort(inv.ravel(), kind="stable")
    pan = own[order].reshape(-1, 2)
    n_live = int(np.sum(term < 0))
    n_term = int(term.max()) + 1 if term.max() >= 0 else 0
    node = np.full(tri.shape[0], -1)
    node[term < 0] = np.arange(n_live)
    node[term >= 0] = n_live + term[term >= 0]
    tp, tq = term[pan[:, 0]], term[pan[:, 1]]
    keep = (tp < 0) | (tq < 0)
    u = np.concatenate([node[pan[keep, 0]], [n_live + s_ for s_, _ in m.ports]])
    v = np.concatenate([node[pan[keep, 1]], [n_live + k_ for _, k_ in m.ports]])
    nn = n_live + n_term
    g = coo_matrix((np.ones(u.shape[0]), (u, v)), shape=(nn, nn))
    ncomp = connected_components(g, directed=False)[0]
    return int(u.shape[0] - nn + ncomp)


def run_reference(args):
    """The reference arm: the CPU oracle (this repository's dense FP64 solver,
    as it stands) timed on the host cores on a bounded sample of the same
    workload (oracle_sample), each step one sample; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "coils":
        m = workload(0, 1)
        rows = 8
        cfg = config_dict(m, "fp64 (CPU oracle)", {"fmm_order": None, "separation": None, "leaf_target": None})
    else:
        import meshgen
        m = {"package": meshgen.package, "package_crop": meshgen.package_crop, "pop": meshgen.pop}[args.workload]()
        m.freqs = spread(m.freqs, args.freqs, world, 0, args.spread)
        rows = max(1, int(2e6 // m.n_tri))
        cfg = {"workload": "%s: %d triangles, %d conductors, %d ports x %d freqs per GPU (%s of its sweep)"
                           % (args.workload, m.n_tri, int(m.cond.max()) + 1, len(m.ports), len(m.freqs),
                              "spread over" if args.spread else "the first"),
               "freqs_hz_rank0": [float(f) for f in m.freqs], "precision": "fp64 (CPU oracle)"}
    n_loops = loop_count(m)
    t0 = time.perf_counter()
    samples = []
    for _ in range(max(1, args.steps)):
        samples.append(oracle_sample(m, n_loops, budget_rows=rows))
    wall = time.perf_counter() - t0
    v = float(np.median([s_["value"] for s_ in samples]))
    cb = dict(samples[-1])
    cb["value"] = v
    if args.workload == "coils":
        cb["c2_full_oracle_recorded"] = oracle_c2_recorded()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- profiling case
def kernel_case(args):
    """The bench workload's context and its two product kinds at the solver's
    launch configuration (384 columns = 64 systems x 6), a few GB on the device:
    3 FP32 FMM products (tensor-core M2L, FP32 near field) and 3 applications of
    the FP64 residual operator (integer-slice tensor-core M2L, double-float near
    field)."""
    import torch
    import paper_2409_12375_gb300 as pkg
    m = workload(0, 1)
    x = pkg.XRL.from_mesh(m, fmm_order=args.fmm_order, separation=2, leaf_target=args.leaf_target, precision=1)
    nsys = len(m.freqs) * len(m.ports)
    g = torch.Generator(device="cuda").manual_seed(1)
    xv = torch.randn(6 * nsys, m.n_tri, device="cuda", dtype=torch.float32, generator=g)
    yv = torch.empty_like(xv)
    n = x.stats()["n_loops"]
    rng = np.random.default_rng(2)
    v = rng.standard_normal((nsys, n)) + 1j * rng.standard_normal((nsys, n))
    f = np.repeat(m.freqs, len(m.ports))
    for _ in range(3):
        x.fmm_mvm32_device(xv, yv)
    torch.cuda.synchronize()
    for _ in range(3):
        x.apply_operator(f, v)
    torch.cuda.synchronize()
    x.close()
    print(json.dumps({"kernel_case": "ok", "n_panels": int(m.n_tri), "n_cols": 6 * nsys}))
    return 0


# ---------------------------------------------------------------- our arm
PREC = {"fp64": 0, "mixed": 1, "fp64_tc": 2}


def make_ctx(pkg, m, opts, precision, autotune, nsys):
    """Context for one arm; autotuned for its own precision unless disabled."""
    x = pkg.XRL.from_mesh(m, **dict(opts, precision=PREC[precision]))
    tuned = None
    if autotune:
        leaf, order, ms, err = x.autotune(6 * nsys, 1e-6, PREC[precision])
        tuned = {"leaf_target": leaf, "fmm_order": order, "product_ms": ms, "product_err": err,
                 "tc_targets_per_cta": x.stats()["tc_targets_per_cta"]}
    return x, tuned


def time_sweeps(x, freqs, warmup, steps, clocks=None, barrier=lambda: None):
    """W untimed sweeps, then K sweeps between CUDA events on the context's
    stream (device time) and host clocks around each call (end to end: host
    frequencies in, host R and L out)."""
    import torch
    ext = torch.cuda.ExternalStream(x.stream_handle())
    for _ in range(warmup):
        x.solve(freqs)
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    l0 = x.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    host = []
    e0.record(ext)
    R = L = None
    for _ in range(steps):
        t0 = time.perf_counter()
        R, L = x.solve(freqs)
        host.append(time.perf_counter() - t0)
    e1.record(ext)
    torch.cuda.synchronize()
    barrier()
    st = x.stats()
    return {"dev_ms": e0.elapsed_time(e1), "host_s": float(np.sum(host)), "R": R, "L": L,
            "launches": x.kernel_launches() - l0, "iters": st["total_iters"], "res": st["max_rel_res"]}


def rl_diff(R, L, Rr, Lr):
    """Per frequency: max |a - b| over the port matrix / max |b|; worst frequency."""
    nf = R.shape[0]
    eR = np.max(np.abs(R - Rr).reshape(nf, -1).max(1) / np.abs(Rr).reshape(nf, -1).max(1))
    eL = np.max(np.abs(L - Lr).reshape(nf, -1).max(1) / np.abs(Lr).reshape(nf, -1).max(1))
    return float(eR), float(eL)


def oracle_rl_error(m, R, L):
    """Element-wise relative error of R11, R22, L11, L22, L12 against the dense
    FP64 oracle of the coils (tests/golden/coils_rl_c2.json), worst over the sweep."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "coils_rl_c2.json")) as f:
            g = json.load(f)
    except Exception:
        return None
    if g["n_panels"] != m.n_tri or len(g["freqs_hz"]) != len(m.freqs) or \
            not np.allclose(g["freqs_hz"], m.freqs, rtol=1e-12, atol=0):
        return None
    Ro, Lo = np.asarray(g["R"]), np.asarray(g["L"])
    out = {}
    for name, a, b in (("R11", R[:, 0, 0], Ro[:, 0, 0]), ("R22", R[:, 1, 1], Ro[:, 1, 1]),
                       ("L11", L[:, 0, 0], Lo[:, 0, 0]), ("L22", L[:, 1, 1], Lo[:, 1, 1]),
                       ("L12", L[:, 0, 1], Lo[:, 0, 1])):
        out[name] = float(np.max(np.abs(a - b) / np.abs(b)))
    return out


def fp64_products(pkg, x, m, pk, ext):
    """The raw FP64 product (xrl_fmm_mvm_device) at 1, 6 and 384 columns:
    panel-columns/s from CUDA events over repeated products, and its roofline
    from the library's algorithmic flops and bytes (profiler counters of one
    product)."""
    import torch
    out = {}
    for nc in (1, 6, 384):
        xv = torch.randn(nc, m.n_tri, device="cuda", dtype=torch.float64)
        yv = torch.empty_like(xv)
        x.reset_profile()
        x.set_profiling(True)
        x.fmm_mvm_device(xv, yv)
        torch.cuda.synchronize()
        prof = x.profile()
        x.set_profiling(False)
        flops = sum(v["flops"] for v in prof.values())
        byts = sum(v["bytes"] for v in prof.values())
        x.fmm_mvm_device(xv, yv)
        torch.cuda.synchronize()
        a_ = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        reps = 3 if nc == 384 else 20
        a_.record(ext)
        for _ in range(reps):
            x.fmm_mvm_device(xv, yv)
        b_.record(ext)
        torch.cuda.synchronize()
        ms = a_.elapsed_time(b_) / reps
        out["nc%d" % nc] = dict(product_roofline(flops, byts, ms, pk), panel_cols_per_s=m.n_tri * nc / (ms * 1e-3),
                                phases_ms={k: round(v["ms"], 4) for k, v in prof.items() if v["ms"] > 0})
        del xv, yv
    return out


def package_run(args):
    """The package workloads (Sec. III-B, III-C stand-ins): the chosen
    configuration (mixed precision, batched multi-RHS frequency chunks, the
    multigrid-applied diagonal-of-P preconditioner), W untimed and K timed
    sweeps of the frequency slice between CUDA events on the library's stream,
    max over ranks (each rank its own slice: weak scaling, no collective on the
    data path).  Then, untimed: one profiled sweep for the phase rooflines, the
    FP64 and FP32 product rates, the plain FP64 product at the sweep's column
    count (the plain FP64 sweep itself is not run: hundreds of those products),
    and the CPU oracle on a bounded sample."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import meshgen
    m = {"package": meshgen.package, "package_crop": meshgen.package_crop, "pop": meshgen.pop}[args.workload]()
    m.freqs = spread(m.freqs, args.freqs, world, rank, args.spread)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before the first GPU call; rows bounded to ~2e6 oracle entries
        cb = oracle_sample(m, loop_count(m), budget_rows=max(1, int(2e6 // m.n_tri)))
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2409_12375_gb300 as pkg

    def barrier():
        if world > 1:
            dist.barrier()

    nport = len(m.ports)
    nsys = len(m.freqs) * nport
    chunk = args.chunk if nsys > 128 or args.freqs else 0
    chunk = chunk if chunk and chunk < nsys else 0
    opts = dict(fmm_order=args.fmm_order, leaf_target=args.leaf_target, precision=1, precond=1, mac_theta=args.mac,
                restart=args.restart, tol=args.tol, max_iters=2000, rhs_chunk=chunk, warm_start=1 if chunk else 0,
                device=local)
    t0 = time.perf_counter()
    x = pkg.XRL.from_mesh(m, **opts)
    setup_s = time.perf_counter() - t0
    ncols = 6 * (min(nsys, chunk) if chunk else nsys)
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        leaf, order, ms, err = x.autotune(ncols, 1e-6, 1)
        tuned = {"leaf_target": leaf, "fmm_order": order, "product_ms": ms, "product_err": err,
                 "tc_targets_per_cta": x.stats()["tc_targets_per_cta"], "autotune_s": time.perf_counter() - t0}
    st = x.stats()
    print("setup %.1f s: %d panels, %d loops, %d leaves, %d near entries, peak %.1f GB; %.1f GB held, %.1f GB cached"
          % (setup_s, st["n_panels"], st["n_loops"], st["n_leaves"], st["near_nnz"], st["peak_device_bytes"] / 1e9,
             st["device_bytes"] / 1e9, st["cached_device_bytes"] / 1e9), file=sys.stderr, flush=True)
    clocks = Clocks()
    try:
        tm = time_sweeps(x, m.freqs, args.warmup, args.steps, clocks, barrier)
    except Exception:
        sf = x.stats()
        print("solve failed: %.1f GB held, %.1f GB cached, peak %.1f GB" %
              (sf["device_bytes"] / 1e9, sf["cached_device_bytes"] / 1e9, sf["peak_device_bytes"] / 1e9),
              file=sys.stderr, flush=True)
        raise
    ck = clocks.stop(local)
    t_dev = torch.tensor([tm["dev_ms"], tm["host_s"]], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t_dev, op=dist.ReduceOp.MAX)
    dev_ms, host_s = float(t_dev[0]), float(t_dev[1])
    units = args.steps * nsys * world
    value = dev_ms / 1e3 / units
    st = x.stats()
    order, leaf = x.opts.fmm_order, x.opts.leaf_target

    # phase breakdown: one more sweep with the phase profiler on
    x.reset_profile()
    x.set_profiling(True)
    x.solve(m.freqs)
    torch.cuda.synchronize()
    prof = x.profile()
    x.set_profiling(False)
    pk = peaks()
    pk["fp64_tflops"] = measure_fp64_peak()
    pk["fp64_src"] = "measured: cuBLAS DGEMM 8192^3 (torch.matmul float64), best of 5, CUDA events"
    near_pad = st["near_nnz_padded"] / float(st["near_nnz"]) if st.get("near_nnz_padded") else 0.0
    tct = st["tc_targets_per_cta"]
    traffic = NCU_TRAFFIC.get((order, st["near_nnz"], tct, ncols))
    roofs = {k: phase_roofline(k, prof[k], pk, "mixed", order, ncols, near_pad, traffic, tct)
             for k in ("p2p", "m2l", "p2p64", "m2l64", "precond", "operator", "p2m", "l2p", "m2m", "l2l")
             if k in prof and prof[k]["ms"] > 0}
    dom = max(roofs, key=lambda k: prof[k]["ms"])

    # product rates (untimed by the bench clock): FP64 at 1 and 6 columns, FP32 and the
    # plain FP64 product at the sweep's column count (one each)
    ext = torch.cuda.ExternalStream(x.stream_handle())
    prod = {}
    for nc, prec in ((1, 64), (6, 64), (ncols, 32), (ncols, 64)):
        dt = torch.float64 if prec == 64 else torch.float32
        a = torch.randn(nc, m.n_tri, device="cuda", dtype=dt)
        b = torch.empty_like(a)
        fn = x.fmm_mvm_device if prec == 64 else x.fmm_mvm32_device
        fn(a, b)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 1 if (prec == 64 and nc > 6) else 3
        e0.record(ext)
        for _ in range(reps):
            fn(a, b)
        e1.record(ext)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prod["fp%d_nc%d" % (prec, nc)] = {"ms": ms, "panel_cols_per_s": m.n_tri * nc / (ms * 1e-3)}
        del a, b
    prod["plain_fp64_over_fp32_product_at_%d_cols" % ncols] = (prod["fp64_nc%d" % ncols]["ms"] /
                                                               prod["fp32_nc%d" % ncols]["ms"])
    ora = None
    if args.workload == "package_crop":
        with open(os.path.join(ROOT, "tests", "golden", "package_crop_rl.json")) as f:
            g = json.load(f)
        fo = np.asarray(g["freqs_hz"]) if "freqs_hz" in g and isinstance(g["freqs_hz"], list) else None
        Ro, Lo = np.asarray(g["R"]), np.asarray(g["L"])
        if fo is not None:
            sel = [int(np.argmin(np.abs(fo - f))) for f in m.freqs]
            Ro, Lo = Ro[sel], Lo[sel]
        R, L = tm["R"], tm["L"]
        ora = {"R_self": float(max(np.max(np.abs(R[:, i, i] - Ro[:, i, i]) / np.abs(Ro[:, i, i])) for i in range(nport))),
               "L_self": float(max(np.max(np.abs(L[:, i, i] - Lo[:, i, i]) / np.abs(Lo[:, i, i])) for i in range(nport)))}
    arm = None
    st2 = x.stats()
    mg = x.opts.mg_cycles
    x.close()                         # frees its device memory (and allocation cache) before the next context
    abl = None
    if args.precond_ablation and world == 1:
        # Table IV on the package: diagonal-of-P (the chosen sweep above) against diagonal-of-L,
        # same FMM, tolerance and chunks; host wall time of one sweep after the setup
        abl = {"diag_P": {"fgmres_iters": tm["iters"], "s_per_freq_port": tm["host_s"] / (args.steps * nsys),
                          "precond_setup_ms": st["precond_setup_ms"], "max_rel_residual": tm["res"]}}
        xl = pkg.XRL.from_mesh(m, **dict(opts, precond=3, fmm_order=order, leaf_target=leaf))
        sl = xl.stats()
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            xl.solve(m.freqs)
            tl = time.perf_counter() - t0
            sl2 = xl.stats()
            abl["diag_L"] = {"fgmres_iters": sl2["total_iters"], "s_per_freq_port": tl / nsys,
                             "precond_setup_ms": sl["precond_setup_ms"], "max_rel_residual": sl2["max_rel_res"]}
        except pkg.XRLError as e:
            abl["diag_L"] = {"error": str(e), "precond_setup_ms": sl["precond_setup_ms"]}
        xl.close()
    if args.fp64tc_arm and world == 1:
        xa = pkg.XRL.from_mesh(m, **dict(opts, precision=2, fmm_order=order, leaf_target=leaf))
        ra = time_sweeps(xa, m.freqs, 0, 1)
        eR, eL = rl_diff(tm["R"], tm["L"], ra["R"], ra["L"])
        arm = {"s_per_freq_port": ra["dev_ms"] / 1e3 / nsys, "fgmres_iters": ra["iters"], "max_rel_residual": ra["res"],
               "rel_err_R_chosen_vs_this": eR, "rel_err_L_chosen_vs_this": eL}
        xa.close()
    if rank == 0:
        if cb is not None:
            cb["sample"] = "%s workload: %s" % (args.workload, cb["sample"])
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 mixed (FP32 FMM in FP64 FGMRES-IR)",
                "data": "synthetic",
                "config": {"workload": "%s: %d triangles, %d conductors, %d ports x %d freqs per GPU (%s of its "
                                       "sweep), tol %g, restart %d%s"
                                       % (args.workload, m.n_tri, int(m.cond.max()) + 1, nport, len(m.freqs),
                                          "spread over" if args.spread else "the first", args.tol, args.restart,
                                          ", chunks of %d systems" % chunk if chunk else ""),
                           "freqs_hz_rank0": [float(f) for f in m.freqs], "mac_theta": args.mac, "mg_cycles": mg,
                           "autotune": tuned, "fmm_order": order, "leaf_target": leaf, "precision": "mixed",
                           "parallelism": "replicas over frequencies" if world > 1 else "1 GPU",
                           "l2": "working set > L2 (near field and Krylov basis, tens of GB): no flush needed"},
                "e2e": {"value": host_s / units, "unit": UNIT, "h2d_bytes_per_step": 8 * len(m.freqs),
                        "d2h_bytes_per_step": 2 * 8 * len(m.freqs) * nport ** 2},
                "gpu_launches": tm["launches"], "clocks": ck, "roofline": roofs[dom], "roofline_phases": roofs,
                "cpu_baseline": cb, "products": prod, "oracle_rl_error": ora, "fp64_tc": arm,
                "precond_ablation": abl,
                "plain_fp64": {"run": False, "why": "its product at the sweep's column count is timed instead "
                                                    "(products.fp64_nc%d); the sweep takes hundreds of them" % ncols},
                "solve": {"fgmres_iters": tm["iters"], "max_rel_residual": tm["res"], "setup_s": setup_s,
                          "setup_phase_ms": st["setup_phase_ms"], "n_loops": st["n_loops"],
                          "n_global_loops": st["n_global_loops"], "near_per_panel": st["near_nnz"] / st["n_panels"],
                          "mg_levels": st["mg_levels"], "mg_coarse_n": st["mg_coarse_n"],
                          "peak_device_bytes": st2["peak_device_bytes"]},
                "phases_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_case:
        return kernel_case(args)
    if args.workload != "coils" and not args.sweep_case:
        return package_run(args)
    if args.sweep_case:
        import paper_2409_12375_gb300 as pkg
        m = workload(0, 1)
        x = pkg.XRL.from_mesh(m, fmm_order=args.fmm_order, leaf_target=args.leaf_target, precision=1)
        x.solve(m.freqs)
        x.solve(m.freqs)
        print(json.dumps({"sweep_case": "ok", "iters": x.stats()["total_iters"]}))
        x.close()
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    c1_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c1_oracle = oracle_c1_full()          # process pool started before the first GPU call
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2409_12375_gb300 as pkg

    def barrier():
        if world > 1:
            dist.barrier()

    m = workload(rank, world)
    nsys = len(m.freqs) * len(m.ports)
    opts = dict(fmm_order=args.fmm_order, separation=2, leaf_target=args.leaf_target, device=local)
    x, tuned = make_ctx(pkg, m, opts, args.precision, not args.no_autotune, nsys)
    st = x.stats()
    cfg_opts = dict(opts, fmm_order=x.opts.fmm_order, leaf_target=x.opts.leaf_target)
    # ---- timed region (chosen arm)
    clocks = Clocks()
    tm = time_sweeps(x, m.freqs, args.warmup, args.steps, clocks, barrier)
    ck = clocks.stop(local)
    R, L = tm["R"], tm["L"]
    # phase breakdown: the same K sweeps again with the phase profiler on (CUDA
    # events per phase on the library's stream; the near field then runs in
    # sequence with the far field instead of beside it, so each phase is timed alone)
    x.reset_profile()
    x.set_profiling(True)
    for _ in range(args.steps):
        x.solve(m.freqs)
    torch.cuda.synchronize()
    prof = x.profile()
    x.set_profiling(False)
    t_dev = torch.tensor([tm["dev_ms"], tm["host_s"]], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t_dev, op=dist.ReduceOp.MAX)
    dev_ms, host_s = float(t_dev[0]), float(t_dev[1])
    gathered = None
    if world > 1:
        Ra, La = gather_sweep(R, L, world)
        gathered = {"n_freqs": int(Ra.shape[0]), "R_fmax": Ra[-1].tolist(), "L_fmax": La[-1].tolist()}
    units = args.steps * nsys * world
    value = (dev_ms / 1e3) / units
    e2e = host_s / units

    # roofline of every major phase; "roofline" is the dominant one
    pk = peaks()
    pk["fp64_tflops"] = measure_fp64_peak()
    pk["fp64_src"] = "measured: cuBLAS DGEMM 8192^3 (torch.matmul float64), best of 5, CUDA events"
    near_pad = st["near_nnz_padded"] / float(st["near_nnz"]) if st.get("near_nnz_padded") else 0.0
    key = (cfg_opts["fmm_order"], st["near_nnz"], x.stats()["tc_targets_per_cta"], 6 * nsys)
    traffic = NCU_TRAFFIC.get(key) if args.precision == "mixed" else None
    tct = x.stats()["tc_targets_per_cta"]
    roofs = {k: phase_roofline(k, prof[k], pk, args.precision, cfg_opts["fmm_order"], 6 * nsys, near_pad, traffic,
                               tct)
             for k in ("p2p", "m2l", "p2p64", "m2l64", "precond", "operator", "p2m", "l2p", "m2m", "l2l")
             if k in prof and prof[k]["ms"] > 0}
    dom = max(roofs, key=lambda k: prof[k]["ms"])
    roof = roofs[dom]

    # the raw FP64 product (the paper's fmm_mvm) at 1, 6 and 384 columns
    ext = torch.cuda.ExternalStream(x.stream_handle())
    mvm = fp64_products(pkg, x, m, pk, ext)

    # comparison arms, each autotuned for its own precision, timed like the chosen arm
    arms = {}
    if world == 1 and not args.no_plain and args.precision == "mixed":
        for name in ("fp64_tc", "fp64"):
            xa, ta = make_ctx(pkg, m, opts, name, not args.no_autotune, nsys)
            ra = time_sweeps(xa, m.freqs, args.warmup, args.steps)
            spf = ra["dev_ms"] / 1e3 / (args.steps * nsys)
            eR, eL = rl_diff(R, L, ra["R"], ra["L"])
            arms["plain_fp64" if name == "fp64" else name] = {
                "s_per_freq_port": spf, "e2e_s_per_freq_port": ra["host_s"] / (args.steps * nsys),
                "fgmres_iters": ra["iters"], "max_rel_residual": ra["res"], "autotune": ta,
                "speedup_chosen_vs_this": spf / value,
                "rel_err_R_chosen_vs_this": eR, "rel_err_L_chosen_vs_this": eL,
                "oracle_rl_error": oracle_rl_error(m, ra["R"], ra["L"])}
            xa.close()

    # preconditioner comparison outside the timed region (Sec. II-D, Table IV): the same sweep with
    # the diagonal-of-P (eq. 10) and the diagonal-of-L preconditioners at the table's tolerance 1e-6
    # and at the bench's 1e-8; setup = the pencil build (P entries, pattern, band ordering)
    abl = None
    po = dict(cfg_opts, precision=PREC[args.precision])
    if not args.no_ablation and world == 1:
        abl = {}
        for tol in (1e-6, 1e-8):
            row = {}
            for name, pc in (("diag_P", 1), ("diag_L", 3)):
                xa = pkg.XRL.from_mesh(m, **dict(po, precond=pc, tol=tol))
                sa = xa.stats()
                try:
                    xa.solve(m.freqs)
                    xa.reset_profile()
                    xa.set_profiling(True)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    xa.solve(m.freqs)
                    ta = time.perf_counter() - t0
                    pa = xa.profile()
                    sb = xa.stats()
                    row[name] = {"fgmres_iters": sb["total_iters"], "s_per_freq_port": ta / nsys,
                                 "precond_setup_ms": sa["precond_setup_ms"],
                                 "precond_factor_apply_ms": pa["precond"]["ms"] if "precond" in pa else None,
                                 "max_rel_residual": sb["max_rel_res"]}
                except pkg.XRLError as e:
                    row[name] = {"error": str(e), "precond_setup_ms": sa["precond_setup_ms"]}
                xa.close()
            abl["tol_%g" % tol] = row

    # the same coils meshed with rectangles on the straight runs (Sec. II-A hybrid panels), untimed:
    # same FMM configuration and frequencies; R, L against the triangle sweep above
    hyb = None
    if not args.no_ablation and world == 1:
        import meshgen
        mh = meshgen.coils(rect=True)
        mh.freqs = m.freqs
        xh = pkg.XRL.from_mesh(mh, **po)
        xh.solve(mh.freqs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Rh, Lh = xh.solve(mh.freqs)
        th = time.perf_counter() - t0
        sh = xh.stats()
        dR, dL = rl_diff(Rh, Lh, R, L)
        hyb = {"n_panels": sh["n_panels"], "n_rectangles": int(np.sum(mh.tri[:, 3] >= 0)), "n_loops": sh["n_loops"],
               "fgmres_iters": sh["total_iters"], "s_per_freq_port": th / nsys,
               "rel_diff_R_vs_triangles": dR, "rel_diff_L_vs_triangles": dL}
        xh.close()

    if rank == 0:
        cb = None
        if world == 1 and not args.no_cpu_baseline:
            cb = oracle_sample(m, st["n_loops"])
            cb["c1_full_oracle"] = c1_oracle
            cb["c2_full_oracle_recorded"] = oracle_c2_recorded()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32/f64 mixed (FP32 FMM in FP64 FGMRES-IR)" if args.precision == "mixed" else "f64",
                "data": "synthetic", "config": dict(config_dict(m, args.precision, cfg_opts), autotune=tuned),
                "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * len(m.freqs),
                        "d2h_bytes_per_step": 2 * 8 * len(m.freqs) * len(m.ports) ** 2},
                "gpu_launches": tm["launches"], "clocks": ck, "roofline": roof, "roofline_phases": roofs,
                "cpu_baseline": cb, "fmm_mvm_fp64": mvm, "arms": arms,
                "oracle_rl_error": oracle_rl_error(m, R, L), "sweep_gathered": gathered,
                "precond_ablation": abl, "hybrid_panels": hyb,
                "solve": {"fgmres_iters": tm["iters"], "max_rel_residual": tm["res"], "setup_ms": st["setup_ms"],
                          "n_loops": st["n_loops"], "near_nnz": st["near_nnz"],
                          "near_per_panel": st["near_nnz"] / float(st["n_panels"]),
                          "peak_device_bytes": x.stats()["peak_device_bytes"]},
                "phases_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}
        print(json.dumps(line))
    x.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
