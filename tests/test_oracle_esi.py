"""Pins for the ESI model (eq. 3) in oracle/esi.py."""
import os

import numpy as np

from oracle.esi import MU0, zs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "skin_depths.txt")


def test_dc_limit_is_rdc():
    sig, t = 5.8e7, 0.5e-3
    rdc = 2.0 / (sig * t)
    assert zs(0.0, sig, t) == rdc
    z = zs(1e-10, sig, t)      # |x| ~ 1e-8: Z_s = R_DC (1 + x/2 + ...)
    assert abs(z - rdc) / rdc < 1e-7


def test_small_x_series_matches_closed_form():
    # continuity across the |x| = 1e-3 switch
    sig, t = 5.8e7, 0.5e-3
    rdc = 2.0 / (sig * t)
    rrf = np.sqrt(np.pi * MU0 / sig)
    f_switch = (1e-3 * rdc / (np.sqrt(2) * rrf)) ** 2
    a = zs(f_switch * (1 - 1e-9), sig, t)
    b = zs(f_switch * (1 + 1e-9), sig, t)
    assert abs(a - b) / abs(a) < 1e-12


def test_high_frequency_limit_is_skin_effect_impedance():
    # for thickness >> skin depth, Z_s -> (1+j) / (sigma * delta): a good conductor half-space
    sig, t = 5.8e7, 1e-3
    f = 1e10
    delta = 1.0 / np.sqrt(np.pi * f * MU0 * sig)
    z = zs(f, sig, t)
    ref = (1 + 1j) / (sig * delta)
    assert abs(z - ref) / abs(ref) < 1e-12
    assert abs(z.real - z.imag) / z.real < 1e-12


def test_low_frequency_first_order_term():
    # Z_s = R_DC (1 + x/2 + O(x^2)) with x = (1+j) R_RF sqrt(f) / R_DC
    sig, t = 5.8e7, 0.5e-3
    rdc = 2.0 / (sig * t)
    rrf = np.sqrt(np.pi * MU0 / sig)
    f = 1.0
    x = (1 + 1j) * rrf * np.sqrt(f) / rdc
    z = zs(f, sig, t)
    assert abs(z - rdc * (1 + x / 2)) / rdc < 2 * abs(x) ** 2


def test_paper_skin_depths_pin_constants():
    # the printed skin depths imply sigma ~ 5.96e7 S/m with mu0 = 4 pi 1e-7 (Sec. III)
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    sig = []
    for r in rows:
        f, d = float(r[0]), float(r[1])
        sig.append(1.0 / (np.pi * f * MU0 * d * d))
    sig = np.array(sig)
    assert np.all(np.abs(sig / 5.96e7 - 1) < 2e-3), sig
    # and R_RF sqrt(f) is the skin resistance 1/(sigma delta)
    f, d = float(rows[0][0]), float(rows[0][1])
    s = sig[0]
    assert abs(np.sqrt(np.pi * MU0 / s) * np.sqrt(f) - 1.0 / (s * d)) < 1e-9 / (s * d)
