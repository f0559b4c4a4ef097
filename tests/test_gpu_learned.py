"""The learned initial guess: network gradients against the FP64 oracle, the
projection of exact current shapes, and what a trained network gains over
the zero initial guess on a geometry it was not trained on."""
import numpy as np
import pytest

import meshgen
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as p
    if not os.path.exists(p.library_path()):
        __graft_entry__.build()
    return p


def small_coils(outer, seed_gap=0.4e-3):
    return meshgen.coils(outer=outer, w=0.15e-3, s=0.15e-3, turns=3, gap=seed_gap, step=0.1e-3, n_freq=12,
                         fmin=1e3, fmax=1e10)


def test_mlp_gradients_match_fp64_oracle(pkg):
    import torch
    net = pkg.MLP(n_in=24, width=128, n_hidden=3, n_out=6, seed=3)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((300, 24)).astype(np.float32)
    t = rng.standard_normal((300, 6)).astype(np.float32)
    g, loss = net.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    p = net.get_params()
    dims = [24, 128, 128, 128, 6]
    lo, go = omlp.loss_and_grad(p, dims, x.astype(np.float64), t.astype(np.float64), round_weights=True)
    assert abs(loss - lo) / lo < 1e-5
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-4
    y = net.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    yo, _, _ = omlp.forward(p, dims, x.astype(np.float64))
    assert np.max(np.abs(y - yo)) < 1e-4 * max(1.0, np.max(np.abs(yo)))
    net.close()


def test_mlp_training_reduces_loss(pkg):
    import torch
    net = pkg.MLP(n_in=24, width=128, n_hidden=3, n_out=6, seed=4)
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.standard_normal((8192, 24)), device="cuda", dtype=torch.float32)
    w = torch.tensor(rng.standard_normal((24, 6)), device="cuda", dtype=torch.float32)
    t = torch.tanh(x @ w).contiguous()
    first = net.train_step(x, t, lr=3e-3)
    for _ in range(150):
        last = net.train_step(x, t, lr=3e-3)
    assert last < 0.1 * first
    net.close()


def test_exact_shape_guess_converges_immediately(pkg):
    """Projecting the exact panel currents of a solved sweep recovers the
    solution: every guess is accepted and FGMRES stops at once."""
    import torch
    m = small_coils(2.4e-3)
    ctx = pkg.XRL.from_mesh(m, fmm_order=8)
    R0, L0 = ctx.solve(m.freqs)
    it0 = ctx.stats()["total_iters"]
    shape = torch.tensor(ctx.panel_currents(normalize=True), device="cuda", dtype=torch.float32)
    R, L, acc, gres = ctx.solve_guess(m.freqs, shape)
    assert acc.min() == 1
    assert gres.max() < 1e-3          # FP32 shapes: residual at the FP32 level
    assert ctx.stats()["total_iters"] < it0 / 2
    assert np.max(np.abs(R - R0)) < 1e-6 * np.max(np.abs(R0))
    assert np.max(np.abs(L - L0)) < 1e-6 * np.max(np.abs(L0))
    ctx.close()


def test_learned_guess_gains_on_held_out_geometry(pkg):
    from paper_2409_12375_gb300 import warmstart
    net = pkg.MLP(n_in=24, width=128, n_hidden=3, n_out=6, seed=5)
    data = []
    for outer in (2.2e-3, 2.6e-3, 3.0e-3):
        m = small_coils(outer)
        ctx = pkg.XRL.from_mesh(m, fmm_order=8)
        data.append(warmstart.training_data(ctx, m.freqs, float(m.freqs[0])))
        ctx.close()
    hist = warmstart.train(net, data, steps=600, batch=32768, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    m = small_coils(2.8e-3)                        # not in the training set
    ctx = pkg.XRL.from_mesh(m, fmm_order=8)
    ctx.solve(m.freqs)
    it_zero = ctx.stats()["total_iters"]
    R, L, acc, gres = warmstart.solve_learned(ctx, net, m.freqs)
    it_learned = ctx.stats()["total_iters"]
    print("iterations zero guess %d, learned guess %d; accepted %d/%d; median guess residual %.3g"
          % (it_zero, it_learned, acc.sum(), acc.size, np.median(gres)))
    assert np.median(gres) < 0.5
    assert it_learned < it_zero
    ctx.close()
    net.close()
