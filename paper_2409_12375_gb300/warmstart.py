"""Learned initial guess for broadband sweeps (driver around the C ABI).

Flow for one geometry (all arithmetic runs in the library's kernels):
  1. solve the reference (lowest) frequency f0 for every port and read the
     panel currents per unit port current (xrl_get_panel_currents);
  2. build per-panel features for every frequency of the sweep
     (xrl_panel_features) and run the network on them (xrl_mlp_forward);
  3. solve the whole sweep from the predicted shapes (xrl_solve_guess), which
     projects them onto loop space, fits one complex scale per system and
     keeps a guess only where the FP64 residual says it helps.
Training data come from sweeps the solver itself produced (steps 1-2 with
the solved currents as targets, scaled like the features).
"""
import numpy as np


def reference(ctx, f0):
    """Per-unit-port-current panel currents at f0: torch CUDA float64 [n_ports][n_panels][6]."""
    import torch
    ctx.solve(np.array([f0]))
    return torch.tensor(ctx.panel_currents(normalize=True), device="cuda", dtype=torch.float64)


def training_data(ctx, freqs, f0):
    """(features [rows][24], targets [rows][6]) from solves of this context's mesh."""
    import torch
    ip0 = reference(ctx, f0)
    ctx.solve(np.asarray(freqs))
    ip = ctx.panel_currents(normalize=True)                      # [nf*np][N][6]
    feat, scale = ctx.features(freqs, f0, ip0)
    npt = ip0.shape[0]
    ip = ip.reshape(len(freqs), npt, -1, 6) * scale[None, :, None, None]
    tgt = torch.tensor(ip.reshape(-1, 6), device="cuda", dtype=torch.float32)
    return feat.reshape(-1, 24).contiguous(), tgt.contiguous()


def train(mlp, data, steps=400, batch=32768, lr=2e-3, weight_decay=1e-4, seed=0):
    """Minibatch AdamW on the concatenated (features, targets) pairs; returns the loss history."""
    import torch
    X = torch.cat([d[0] for d in data])
    T = torch.cat([d[1] for d in data])
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (min(batch, X.shape[0]),), generator=g).to(X.device)
        hist.append(mlp.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=lr, weight_decay=weight_decay))
    return hist


def predict(ctx, mlp, freqs, f0, ip0):
    """Predicted current shapes [n_freq * n_ports][n_panels][6] (torch CUDA float32)."""
    feat, _ = ctx.features(freqs, f0, ip0)
    nsys, n = feat.shape[0], feat.shape[1]
    y = mlp.forward(feat.reshape(-1, 24).contiguous())
    return y.reshape(nsys, n, 6).contiguous()


def solve_learned(ctx, mlp, freqs, f0=None):
    """Sweep solve started from the network's prediction; returns R, L, accepted, guess residuals."""
    f0 = float(np.min(freqs)) if f0 is None else f0
    ip0 = reference(ctx, f0)
    shape = predict(ctx, mlp, freqs, f0, ip0)
    return ctx.solve_guess(np.asarray(freqs), shape)
