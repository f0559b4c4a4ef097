"""Triangle quadrature rules for the oracle (test infrastructure only).

All rules return barycentric-free data: for a triangle (v0, v1, v2) the
points are affine combinations of the vertices and the weights are
normalised to sum to one, so a rule computes the panel AVERAGE of a function.

* collapsed(q): the Duffy/Stroud conical product of q-point Gauss-Legendre
  rules.  p = v0 + s (v1 - v0) + t (1 - s) (v2 - v0), weight 2 W_s W_t (1 - s).
  Exact for polynomials of total degree 2q - 2.
* edge_graded(n, k): Duffy map with the singular EDGE (a, b) at u = 1,
  p = o + u [(a - o) + w (b - a)], u = 1 - (1 - xi)^k, used when the outer
  panel shares an edge with the source panel.
* vertex_graded(n, k): Duffy map with the singular VERTEX a at u = 0,
  p = a + u [(b - a) + w (o - b)], u = xi^k, used for a shared vertex.

The near-field rule table (which rule for which pair) lives in panels.py.
"""
import numpy as np


def gauss01(q):
    """q-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def collapsed(q):
    """Coefficients (c0, c1, c2) per point with p = c0 v0 + c1 v1 + c2 v2, and weights."""
    s, ws = gauss01(q)
    t, wt = gauss01(q)
    S, T = np.meshgrid(s, t, indexing="ij")
    W = 2.0 * np.outer(ws, wt) * (1.0 - S)
    S = S.ravel()
    T = T.ravel()
    c1 = S
    c2 = T * (1.0 - S)
    c0 = 1.0 - c1 - c2
    return np.stack([c0, c1, c2], axis=1), W.ravel()


def edge_graded(n, k):
    """Coefficients on (o, a, b) and weights; singular edge a-b."""
    xi, wx = gauss01(n)
    pts = []
    wts = []
    for i in range(n):
        u = 1.0 - (1.0 - xi[i]) ** k
        du = k * (1.0 - xi[i]) ** (k - 1) * wx[i]
        for j in range(n):
            w = xi[j]
            # p = o + u (a - o) + u w (b - a) = (1-u) o + u (1-w) a + u w b
            pts.append((1.0 - u, u * (1.0 - w), u * w))
            wts.append(2.0 * u * du * wx[j])
    return np.array(pts), np.array(wts)


def vertex_graded(n, k):
    """Coefficients on (a, b, o) and weights; singular vertex a."""
    xi, wx = gauss01(n)
    pts = []
    wts = []
    for i in range(n):
        u = xi[i] ** k
        du = k * xi[i] ** (k - 1) * wx[i]
        for j in range(n):
            w = xi[j]
            # p = a + u (b - a) + u w (o - b) = (1-u) a + u (1-w) b + u w o
            pts.append((1.0 - u, u * (1.0 - w), u * w))
            wts.append(2.0 * u * du * wx[j])
    return np.array(pts), np.array(wts)
