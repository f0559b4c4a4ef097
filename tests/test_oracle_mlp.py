"""Pins for oracle/mlp.py: the analytic gradient matches central finite
differences (FP64, weights not rounded), and BF16 rounding matches the
bfloat16 definition on known values."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = [5, 7, 7, 3]
    _, n = mlp.layout(dims)
    p = rng.standard_normal(n) * 0.5
    x = rng.standard_normal((11, 5))
    t = rng.standard_normal((11, 3))
    _, g = mlp.loss_and_grad(p, dims, x, t, round_weights=False)
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, dims, x, t, round_weights=False)
        lm, _ = mlp.loss_and_grad(p - e, dims, x, t, round_weights=False)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-6 * max(1.0, np.max(np.abs(g)))


def test_bf16_rounding():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to even (1.0);
    # 1 + 3 * 2^-8 ties between 1 + 2^-7 and 1 + 2^-6... rounds to 1 + 2^-6 (even mantissa)
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-3], np.float32)
    r = mlp.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6
    assert r[3] == -2.5
    assert abs(r[4] - 3.0e-3) / 3.0e-3 < 2.0 ** -8
