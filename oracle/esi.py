"""Equivalent surface impedance, the double-plane model of eq. 3 (Sec. II-A).

Z_s(f) = (1+j) R_RF sqrt(f) / (1 - exp(-(1+j) R_RF sqrt(f) / R_DC)),
R_DC = 2 / (sigma * thickness),  R_RF = sqrt(pi * mu0 / sigma).

Written as Z_s = R_DC * x / (1 - exp(-x)) with x = (1+j) R_RF sqrt(f) / R_DC,
which is the same expression; the quotient x / (1 - e^{-x}) is evaluated with
expm1 and, for |x| < 1e-3, with its Taylor series 1 + x/2 + x^2/12 - x^4/720
(the Bernoulli-number generating function), so that Z_s(0) = R_DC exactly.
"""
import numpy as np

MU0 = 4e-7 * np.pi


def zs(f, sigma, thickness):
    f = np.asarray(f, float)
    rdc = 2.0 / (sigma * thickness)
    rrf = np.sqrt(np.pi * MU0 / sigma)
    x = (1.0 + 1.0j) * rrf * np.sqrt(f) / rdc
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    q_big = xs / (-np.expm1(-xs))
    q_small = 1.0 + x / 2.0 + x * x / 12.0 - x ** 4 / 720.0
    return rdc * np.where(small, q_small, q_big)
