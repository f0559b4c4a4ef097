"""FP64 reference of the per-panel network (oracle, test infrastructure only).

Same network as the library's: h_0 = x, h_{l+1} = GELU(h_l W_l + b_l) for
the hidden layers (exact GELU, 0.5 a (1 + erf(a / sqrt 2))), output
y = h W_L + b_L, loss = mean((y - t)^2).  The weights used in the forward
and backward pass are the FP32 master weights rounded to BF16 (round to
nearest, ties to even), as in the library; everything else is FP64.
Parameter layout per layer: W_l [in][out] row-major, then b_l [out].
Pinned by central finite differences in tests/test_oracle_mlp.py.
"""
import numpy as np
from scipy.special import erf


def bf16_round(w):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    u = np.asarray(w, np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((u >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)
    r = ((u + rounding) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layout(dims):
    out = []
    off = 0
    for a, b in zip(dims[:-1], dims[1:]):
        out.append((off, off + a * b, a, b))
        off += a * b + b
    return out, off


def unpack(params, dims, round_weights=True):
    lay, _ = layout(dims)
    Ws, bs = [], []
    for w0, b0, a, b in lay:
        W = np.asarray(params[w0:w0 + a * b]).reshape(a, b)
        Ws.append(bf16_round(W.astype(np.float32)) if round_weights else W.astype(np.float64))
        bs.append(np.asarray(params[b0:b0 + b], np.float64))
    return Ws, bs


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / np.sqrt(2.0)))


def gelu_d(a):
    return 0.5 * (1.0 + erf(a / np.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / np.sqrt(2.0 * np.pi)


def forward(params, dims, x, round_weights=True):
    Ws, bs = unpack(params, dims, round_weights)
    h = np.asarray(x, np.float64)
    pre = []
    acts = [h]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        a = h @ W + b
        pre.append(a)
        h = gelu(a) if l + 1 < len(Ws) else a
        acts.append(h)
    return h, pre, acts


def loss_and_grad(params, dims, x, t, round_weights=True):
    """Mean squared error and its gradient w.r.t. the (rounded) weights and biases."""
    Ws, bs = unpack(params, dims, round_weights)
    y, pre, acts = forward(params, dims, x, round_weights)
    n = y.size
    d = 2.0 * (y - t) / n
    lay, total = layout(dims)
    g = np.zeros(total)
    for l in range(len(Ws) - 1, -1, -1):
        w0, b0, a, b = lay[l]
        g[w0:w0 + a * b] = (acts[l].T @ d).ravel()
        g[b0:b0 + b] = d.sum(axis=0)
        if l > 0:
            d = (d @ Ws[l].T) * gelu_d(pre[l - 1])
    return float(np.mean((y - t) ** 2)), g
