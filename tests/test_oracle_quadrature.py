"""Pins for oracle/quadrature.py: exact integration of monomials.

On the unit right triangle T = {x, y >= 0, x + y <= 1},
int_T x^a y^b dA = a! b! / (a + b + 2)!  (Beta-function identity), so the
panel average is 2 a! b! / (a + b + 2)!.
"""
from math import factorial

import numpy as np
import pytest

from oracle import quadrature as qd

V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


def avg_exact(a, b):
    return 2.0 * factorial(a) * factorial(b) / factorial(a + b + 2)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 8])
def test_collapsed_exact_to_degree(q):
    coef, w = qd.collapsed(q)
    assert abs(w.sum() - 1.0) < 1e-14
    p = coef @ V
    for a in range(2 * q - 1):
        for b in range(2 * q - 1 - a):
            got = np.sum(w * p[:, 0] ** a * p[:, 1] ** b)
            assert abs(got - avg_exact(a, b)) < 1e-13, (q, a, b)


def test_collapsed_not_exact_beyond_degree():
    # a plausible off-by-one in the Jacobian would make degree 2q-1 "exact" too
    coef, w = qd.collapsed(2)
    p = coef @ V
    errs = [abs(np.sum(w * p[:, 0] ** a * p[:, 1] ** (4 - a)) - avg_exact(a, 4 - a)) for a in range(5)]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("kind", ["edge", "vertex"])
def test_graded_rules_integrate_polynomials(kind):
    # graded maps are polynomial, so low-degree monomials are integrated exactly
    coef, w = qd.edge_graded(10, 3) if kind == "edge" else qd.vertex_graded(10, 3)
    assert abs(w.sum() - 1.0) < 1e-13
    # vertex roles: edge rule takes (o, a, b), vertex rule (a, b, o); any
    # assignment of the reference triangle's vertices must give the same average
    for perm in ([0, 1, 2], [1, 2, 0], [2, 0, 1]):
        p = coef @ V[perm]
        for a in range(4):
            for b in range(4 - a):
                got = np.sum(w * p[:, 0] ** a * p[:, 1] ** b)
                assert abs(got - avg_exact(a, b)) < 1e-12, (kind, perm, a, b)
