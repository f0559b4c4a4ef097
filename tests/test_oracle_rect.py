"""Pins for the rectangular panels of the hybrid meshes (Sec. II-A, Figs. 1-2):
the sub-triangle decomposition of P against the closed-form self and
edge-adjacent integrals of coplanar rectangles and against a reduced 2-D
quadrature for other aligned pairs; the centroid-midpoint transform on
rectangles (uniform current, DC resistance) and the loop basis on a hybrid
triangle/rectangle mesh."""
import numpy as np
import pytest
from scipy import integrate

import meshgen
from oracle import circuit as C
from oracle import panels as P


def _F(a, b):
    """int int over an a x b rectangle of int int 1/|r - r'| (the closed form
    of 4 int_0^a int_0^b (a - u)(b - v) / sqrt(u^2 + v^2) du dv)."""
    d = np.hypot(a, b)
    return (2 * a**3 / 3 + 2 * b**3 / 3 - 2 * (a * a + b * b) * d / 3
            + 2 * a * a * b * np.arcsinh(b / a) + 2 * a * b * b * np.arcsinh(a / b))


def _overlap(x0, x1, y0, y1):
    """g(u) = length of {x in [x0, x1] : x + u in [y0, y1]} and its kinks."""
    g = lambda u: max(0.0, min(x1, y1 - u) - max(x0, y0 - u))
    kinks = sorted({y0 - x1, y0 - x0, y1 - x1, y1 - x0})
    return g, kinks


def _aligned_pair(r1, r2):
    """int_R1 int_R2 1/|r - r'| for axis-aligned coplanar rectangles
    r = (x0, x1, y0, y1), reduced to int int g(u) h(v) / sqrt(u^2 + v^2)."""
    g, ku = _overlap(r1[0], r1[1], r2[0], r2[1])
    h, kv = _overlap(r1[2], r1[3], r2[2], r2[3])
    tot = 0.0
    for u0, u1 in zip(ku[:-1], ku[1:]):
        for v0, v1 in zip(kv[:-1], kv[1:]):
            if u1 <= u0 or v1 <= v0:
                continue
            f = lambda v, u: g(u) * h(v) / np.hypot(u, v)
            tot += integrate.dblquad(f, u0, u1, v0, v1, epsabs=0, epsrel=1e-12)[0]
    return tot


def _frame(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q, np.random.default_rng(seed + 1).standard_normal(3) * 1e-3


def _rect_mesh(rects, seed):
    """Panels for axis-aligned rectangles (x0, x1, y0, y1) in z = 0 with shared
    corner vertices, rotated and shifted rigidly."""
    key = {}
    pts = []
    pan = []
    for x0, x1, y0, y1 in rects:
        row = []
        for xy in ((x0, y0), (x1, y0), (x1, y1), (x0, y1)):
            k = (round(xy[0] * 1e12), round(xy[1] * 1e12))
            if k not in key:
                key[k] = len(pts)
                pts.append((xy[0], xy[1], 0.0))
            row.append(key[k])
        pan.append(row)
    R, o = _frame(seed)
    return np.array(pts) @ R.T + o, np.array(pan)


@pytest.mark.parametrize("a,b", [(1e-3, 1e-3), (1e-3, 0.3e-3), (0.2e-3, 75e-6)])
def test_rectangle_self_term_closed_form(a, b):
    xyz, pan = _rect_mesh([(0, a, 0, b)], 3)
    p = P.dense_P_panels(P.Panels(xyz, pan))[0, 0]
    assert abs(p / (_F(a, b) / (a * b) ** 2) - 1) < 3e-8


@pytest.mark.parametrize("a,b,c", [(1e-3, 1e-3, 0.7e-3), (1e-3, 0.3e-3, 1e-3)])
def test_edge_adjacent_rectangles_closed_form(a, b, c):
    # F(R1 u R2) = F(R1) + F(R2) + 2 I(R1, R2) for R1 = [0,a]x[0,b], R2 = [a,a+c]x[0,b]
    xyz, pan = _rect_mesh([(0, a, 0, b), (a, a + c, 0, b)], 4)
    Pm = P.dense_P_panels(P.Panels(xyz, pan))
    ref = (_F(a + c, b) - _F(a, b) - _F(c, b)) / 2 / (a * b * c * b)
    assert abs(Pm[0, 1] / ref - 1) < 3e-8
    assert Pm[0, 1] == Pm[1, 0]


@pytest.mark.parametrize("r2", [(1e-3, 1.6e-3, 0.5e-3, 1.2e-3),     # shares a vertex
                                (1.2e-3, 1.9e-3, -0.3e-3, 0.4e-3),   # separated, q < 1.5
                                (4e-3, 4.5e-3, 2e-3, 2.8e-3)])       # separated, far
def test_aligned_rectangle_pairs_brute_force(r2):
    r1 = (0.0, 1e-3, 0.0, 0.5e-3)
    xyz, pan = _rect_mesh([r1, r2], 5)
    Pm = P.dense_P_panels(P.Panels(xyz, pan))
    A1 = (r1[1] - r1[0]) * (r1[3] - r1[2])
    A2 = (r2[1] - r2[0]) * (r2[3] - r2[2])
    ref = _aligned_pair(r1, r2) / (A1 * A2)
    assert abs(Pm[0, 1] / ref - 1) < 3e-8


def test_triangle_and_rectangle_pair_matches_split_rectangle():
    """A triangle against a rectangle equals the area-weighted mean over the
    rectangle's two halves (the definition of the rectangle's entry), and a
    non-parallelogram quad is rejected."""
    xyz = np.array([[0, 0, 0], [1e-3, 0, 0], [1e-3, 1e-3, 0], [0, 1e-3, 0], [2e-3, 0.5e-3, 0]], float)
    H = P.Panels(xyz, np.array([[0, 1, 2, 3], [1, 4, 2, -1]]))
    T = P.Geometry(xyz, np.array([[0, 1, 2], [0, 2, 3], [1, 4, 2]]))
    Pt = P.dense_P(T)
    Ph = P.dense_P_panels(H)
    assert abs(Ph[0, 1] - 0.5 * (Pt[0, 2] + Pt[1, 2])) < 1e-12 * Ph[0, 1]
    bad = xyz.copy()
    bad[3, 1] = 1.3e-3
    with pytest.raises(ValueError):
        P.Panels(bad, np.array([[0, 1, 2, 3]]))


@pytest.fixture(scope="module")
def rect_bar():
    return meshgen.bar(jitter=0.0, rect=True, n_l=20)


def test_rect_bar_uniform_current_and_dc_resistance(rect_bar):
    c = C.Circuit(rect_bar)
    assert np.all(c.geom.nv == 4)
    # uniform J0 in the x = 0 face: edge fluxes give I_p = J0 * area on every interior rectangle
    xyz = np.asarray(rect_bar.xyz)
    J0 = np.array([0.0, 3.0, -2.0])
    ie = np.zeros(c.n_cb)
    for b in range(c.n_cb):
        va, vb = xyz[c.edge_vertices[c.branch_edge[b]]]
        if abs(va[0]) > 1e-12 or abs(vb[0]) > 1e-12 or c.head[b] >= c.n_live:
            continue
        ct, ch = c.geom.c[c.live[c.tail[b]]], c.geom.c[c.live[c.head[b]]]
        ed = vb - va
        nrm = np.cross(ed, np.array([1.0, 0, 0]))
        nrm /= np.linalg.norm(nrm)
        if np.dot(ch - ct, nrm) < 0:
            nrm = -nrm
        ie[b] = np.dot(J0, nrm) * np.linalg.norm(ed)
    ip = np.stack([c.A[t].T @ ie for t in range(3)], axis=1)
    V = xyz[c.geom.pan]
    on = np.all(np.abs(V[:, :, 0]) < 1e-12, axis=1)
    inner = on & np.all((V[:, :, 1] > 1e-12) & (V[:, :, 1] < 1e-3 - 1e-12), axis=1)
    inner &= np.all((V[:, :, 2] > 1e-12) & (V[:, :, 2] < 10e-3 - 1e-12), axis=1)
    ks = np.flatnonzero(inner & (np.asarray(rect_bar.term) < 0))
    assert ks.size >= 20
    np.testing.assert_allclose(ip[c.panel_node[ks]], np.outer(c.geom.area[ks], J0), rtol=0,
                               atol=1e-12 * np.abs(J0).max() * c.geom.area.max())
    # DC resistance of the surface model equals rho l / A (ESI thickness 2A/perimeter)
    Pd = P.dense_P_panels(c.geom)
    R, L, _ = c.solve([0.0], Pd)
    assert abs(R[0, 0, 0] / (10e-3 / (5.8e7 * 1e-6)) - 1) < 1e-12


def test_hybrid_coil_topology_and_P():
    m = meshgen.coils(outer=2e-3, turns=1, n_w=2, step=0.2e-3, n_coils=1, rect=True, n_freq=4)
    c = C.Circuit(m)
    assert 0 < np.sum(c.geom.nv == 4) < c.geom.n
    Bm = c.incidence()
    assert np.abs(c.M @ Bm.T).max() == 0.0
    assert c.M.shape[0] == c.n_branch - c.n_nodes + 1
    assert np.linalg.matrix_rank(c.M) == c.M.shape[0]
    Pd = P.dense_P_panels(c.geom)
    assert np.array_equal(Pd, Pd.T)
    assert np.linalg.eigvalsh(Pd).min() > 0


def test_rect_grid_null_loop_mode_carries_no_panel_current(rect_bar):
    """On a grid of rectangles the pulse basis (eq. 4) cannot see the
    checkerboard circulation: the loop matrix Z of eq. 7 is singular, its
    null vector gives zero current on every panel (so Z_s and P both miss
    it), and the port right-hand side is orthogonal to it (the system stays
    consistent).  The triangulated bar has no such mode."""
    c = C.Circuit(rect_bar)
    Pd = P.dense_P_panels(c.geom)
    Z = c.loop_matrix(1e5, c.potential_part(Pd[np.ix_(c.live, c.live)]))
    u, s, vh = np.linalg.svd(Z)
    assert s[-1] < 1e-14 * s[0] and s[-2] > 1e-8 * s[0]
    x = vh[-1].conj()
    ip = c.panel_currents(x[:, None])[:, :, 0]          # [3, n_live]
    ie = c.M[:, :c.n_cb].T @ x
    assert np.abs(ip).max() < 1e-10 * np.abs(ie).max() * np.abs(c.A).max()
    assert abs(c.port_rhs()[:, 0] @ x) < 1e-12
    tri_bar = meshgen.bar(jitter=0.0, n_l=20)
    ct = C.Circuit(tri_bar)
    Pt = P.dense_P(P.Geometry(tri_bar.xyz, tri_bar.tri))
    st = np.linalg.svd(ct.loop_matrix(1e5, ct.potential_part(Pt[np.ix_(ct.live, ct.live)])), compute_uv=False)
    assert st[-1] > 1e-6 * st[0]


@pytest.mark.parametrize("name", ["bar", "coils", "coil1"])
def test_hybrid_generator_closed_oriented_parallelograms(name):
    """The rect=True meshes: closed and consistently oriented, every 4-vertex
    panel a parallelogram, and the same vertices and loop count as the
    triangulated mesh of the same lattice (the rectangles only merge pairs of
    triangles)."""
    if name == "bar":
        m, t = meshgen.bar(jitter=0.0, rect=True, n_l=10), meshgen.bar(jitter=0.0, n_l=10)
    elif name == "coils":
        m, t = meshgen.coils(rect=True), meshgen.coils()
    else:
        kw = dict(outer=2e-3, turns=1, n_w=2, step=0.2e-3, n_coils=1)
        m, t = meshgen.coils(rect=True, **kw), meshgen.coils(**kw)
    assert meshgen.crop_check(m) == (True, True)
    quad = m.tri[:, 3] >= 0
    V = np.asarray(m.xyz)[np.where(m.tri >= 0, m.tri, 0)]
    d = np.linalg.norm(V[quad, 0] + V[quad, 2] - V[quad, 1] - V[quad, 3], axis=1)
    assert np.all(d <= 1e-9 * np.linalg.norm(V[quad, 2] - V[quad, 0], axis=1))
    assert m.xyz.shape == t.xyz.shape
    assert m.n_tri + int(quad.sum()) == t.n_tri
