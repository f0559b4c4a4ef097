"""Pins for oracle/circuit.py: the CM transform (Algorithm 1, eq. 4), the loop
matrix (Sec. II-B), the loop system (eq. 7-8) and port R, L; plus the
diagonal-of-P preconditioner of eq. 10."""
import numpy as np
import pytest

from oracle import circuit as C
from oracle.esi import MU0


@pytest.fixture(scope="module")
def bar_circ(bar_mesh):
    return C.Circuit(bar_mesh)


@pytest.fixture(scope="module")
def two_circ(two_bars_mesh):
    return C.Circuit(two_bars_mesh)


def _face_interior_panels(circ, axis, value):
    """Live panels lying on the plane x_axis = value whose three neighbours
    are live panels on the same plane."""
    G = circ.geom
    on = np.abs(G.v[:, :, axis] - value).max(axis=1) < 1e-12
    out = []
    tri = circ.geom.tri
    for k in np.flatnonzero(on & (np.asarray(circ.mesh.term) < 0)):
        nb = 0
        for e in range(3):
            a, b = tri[k, e], tri[k, (e + 1) % 3]
            m = np.flatnonzero((np.isin(tri, [a, b]).sum(axis=1) == 2) & (np.arange(len(tri)) != k))
            if on[m[0]] and circ.mesh.term[m[0]] < 0:
                nb += 1
        if nb == 3:
            out.append(k)
    return np.array(out)


def test_uniform_current_reproduced_exactly(bar_circ):
    """Flux of a uniform in-plane J0 through each edge gives I_p = J0 * area."""
    c = bar_circ
    xyz = np.asarray(c.mesh.xyz)
    J0 = np.array([0.0, 3.0, -2.0])          # in the plane x = 0
    ie = np.zeros(c.n_cb)
    G = c.geom
    for b in range(c.n_cb):
        e = c.branch_edge[b]
        va, vb = xyz[c.edge_vertices[e]]
        if abs(va[0]) > 1e-12 or abs(vb[0]) > 1e-12:
            continue
        t_node, h_node = c.tail[b], c.head[b]
        if h_node >= c.n_live:
            continue
        ct, ch = G.c[c.live[t_node]], G.c[c.live[h_node]]
        ed = vb - va
        nrm = np.cross(ed, np.array([1.0, 0, 0]))
        nrm /= np.linalg.norm(nrm)
        if np.dot(ch - ct, nrm) < 0:
            nrm = -nrm
        ie[b] = np.dot(J0, nrm) * np.linalg.norm(ed)
    ip = np.stack([c.A[t].T @ ie for t in range(3)], axis=1)     # [n_live, 3]
    ks = _face_interior_panels(c, 0, 0.0)
    assert ks.size > 50
    nodes = c.panel_node[ks]
    np.testing.assert_allclose(ip[nodes], np.outer(G.area[ks], J0), rtol=0, atol=1e-12 * np.abs(J0).max() * G.area.max())


def test_vertex_loop_gives_rotated_hat_gradient(bar_circ):
    """A unit loop circulating counter-clockwise around an interior vertex v
    gives I_p = (b - a)/2 in each triangle (v, a, b) of its star."""
    c = bar_circ
    tri = c.geom.tri
    xyz = np.asarray(c.mesh.xyz)
    # an interior vertex of the x = 0 face, away from the terminals
    cand = [v for v in range(xyz.shape[0]) if abs(xyz[v, 0]) < 1e-12 and 0.3 < xyz[v, 1] / 1e-3 < 0.7
            and 0.3 < xyz[v, 2] / 1e-2 < 0.7]
    v = cand[0]
    star = np.flatnonzero((tri == v).any(axis=1))
    ie = np.zeros(c.n_cb)
    for b in range(c.n_cb):
        ev = c.edge_vertices[c.branch_edge[b]]
        if v not in ev:
            continue
        a = ev[0] if ev[1] == v else ev[1]
        # source triangle: (v, x, a) in ccw order, i.e. a precedes v
        tp = c.live[c.tail[b]]
        r = list(tri[tp])
        i = r.index(v)
        src_is_tail = r[(i + 2) % 3] == a
        ie[b] = 1.0 if src_is_tail else -1.0
    ip = np.stack([c.A[t].T @ ie for t in range(3)], axis=1)
    for k in star:
        r = list(tri[k])
        i = r.index(v)
        a, b = r[(i + 1) % 3], r[(i + 2) % 3]
        np.testing.assert_allclose(ip[c.panel_node[k]], 0.5 * (xyz[b] - xyz[a]), atol=1e-15)
    others = np.setdiff1d(np.arange(c.n_live), c.panel_node[star])
    assert np.abs(ip[others]).max() == 0.0


def test_loop_matrix_is_a_cycle_basis(bar_circ, two_circ):
    for c in (bar_circ, two_circ):
        Bm = c.incidence()
        assert np.abs(c.M @ Bm.T).max() == 0.0
        # cycle-space dimension B - N + components (ports join each conductor's terminals)
        n_comp = len(set(c.mesh.cond))
        assert c.M.shape[0] == c.n_branch - c.n_nodes + n_comp
        assert np.linalg.matrix_rank(c.M) == c.M.shape[0]


def test_bar_dc_resistance_is_rho_l_over_a(bar_circ, bar_dense_P):
    R, L, _ = bar_circ.solve([0.0, 1e-3], bar_dense_P)
    rho_l_a = 10e-3 / (5.8e7 * 1e-6)
    assert abs(R[0, 0, 0] / rho_l_a - 1) < 1e-12
    # at 1 mHz the ESI excess R_RF sqrt(f) / (2 R_DC) is ~6e-5 (eq. 3 expanded)
    assert abs(R[1, 0, 0] / rho_l_a - 1) < 1e-4


def test_bar_high_frequency_inductance_bracket(bar_circ, bar_dense_P):
    # surface current: below the DC partial self inductance of the solid bar
    # (Grover/Ruehli rectangular-bar formula) by about its internal part mu0 l/(8 pi)
    R, L, _ = bar_circ.solve([1e9], bar_dense_P)
    l, w, t = 10e-3, 1e-3, 1e-3
    L_dc = MU0 * l / (2 * np.pi) * (np.log(2 * l / (w + t)) + 0.5 + 0.2235 * (w + t) / l)
    L_int = MU0 * l / (8 * np.pi)
    assert L_dc - 1.5 * L_int < L[0, 0, 0] < L_dc
    # resistance at 1 GHz is set by the skin depth: within 25 % of rho l / (perimeter * delta)
    delta = 1.0 / np.sqrt(np.pi * 1e9 * MU0 * 5.8e7)
    R_skin = l / (5.8e7 * 4 * w * delta)
    assert abs(R[0, 0, 0] / R_skin - 1) < 0.25


def test_two_bars_reciprocity_pd_and_neumann(two_circ, two_bars_dense_P):
    R, L, _ = two_circ.solve([1e9], two_bars_dense_P)
    R, L = R[0], L[0]
    assert abs(R[0, 1] - R[1, 0]) <= 1e-10 * abs(R[0, 0])
    assert abs(L[0, 1] - L[1, 0]) <= 1e-10 * abs(L[0, 0])
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() > 0
    assert np.linalg.eigvalsh(0.5 * (L + L.T)).min() > 0
    l, d = 2e-3, 0.5e-3
    M_neu = MU0 / (2 * np.pi) * (l * np.arcsinh(l / d) - np.hypot(l, d) + d)
    assert abs(L[0, 1] / M_neu - 1) < 1e-2


@pytest.mark.parametrize("f", [1e3, 1e9])
def test_loop_and_nodal_formulations_agree(two_circ, two_bars_dense_P, f):
    Pl = two_bars_dense_P[np.ix_(two_circ.live, two_circ.live)]
    Gp = two_circ.potential_part(Pl)
    Bp = two_circ.port_rhs()
    Y_loop = Bp.T @ np.linalg.solve(two_circ.loop_matrix(f, Gp), Bp.astype(complex))
    Y_mna = C.mna_port_admittance(two_circ, f, two_bars_dense_P)
    assert np.max(np.abs(Y_loop - Y_mna)) < 1e-9 * np.max(np.abs(Y_loop))


def test_precond_is_operator_with_diagonal_P(two_circ, two_bars_dense_P):
    f = 1e8
    Q = C.precond_matrix(two_circ, f, two_bars_dense_P)
    Pd = np.diag(np.diag(two_bars_dense_P))[np.ix_(two_circ.live, two_circ.live)]
    Zd = two_circ.loop_matrix(f, two_circ.potential_part(Pd))
    assert np.max(np.abs(Q - Zd)) < 1e-12 * np.max(np.abs(Q))
    assert np.linalg.eigvalsh(Q.real).min() > 0
    assert np.linalg.eigvalsh(Q.imag).min() > 0


def _branch_potential_diagonal(circ, P_full):
    """(sum_t A_t P A_t^T)_bb for every conductor branch, written out from the
    geometry: the edge midpoint, the two panel centroids and the orientation
    rule of Algorithm 1 (+rho on the tail panel, -rho on the head panel)."""
    xyz = np.asarray(circ.mesh.xyz, float)
    tri = np.asarray(circ.mesh.tri, np.int64)
    cen = xyz[tri].mean(axis=1)
    g = np.zeros(circ.n_cb)
    for b in range(circ.n_cb):
        ev = circ.edge_vertices[circ.branch_edge[b]]
        mid = 0.5 * (xyz[ev[0]] + xyz[ev[1]])
        sides = []
        for node, sign in ((circ.tail[b], 1.0), (circ.head[b], -1.0)):
            if node < circ.n_live:
                p = circ.live[node]
                sides.append((p, sign * (mid - cen[p])))
        for p, r in sides:
            for q, s in sides:
                g[b] += (r @ s) * P_full[p, q]
    return g


@pytest.mark.parametrize("f", [1e3, 1e9])
def test_precond_L_is_surface_impedance_plus_branch_diagonal(two_circ, two_bars_dense_P, f):
    QL = C.precond_matrix_L(two_circ, f, two_bars_dense_P)
    # the surface-impedance part is the operator's loop-space Z_s, whole (the
    # loop matrix with the potential part switched off)
    n = two_circ.M.shape[0]
    Zs = two_circ.loop_matrix(f, np.zeros((n, n)))
    # the rest keeps one inductive term per branch: j omega mu0/4pi M diag(g) M^T
    g = _branch_potential_diagonal(two_circ, two_bars_dense_P)
    Mc = two_circ.M[:, :two_circ.n_cb]
    Li = 2 * np.pi * f * C.MU0_4PI * (Mc * g[None, :]) @ Mc.T
    assert np.max(np.abs(QL - Zs - 1j * Li)) < 1e-12 * np.max(np.abs(QL))
    assert np.all(g > 0)


def test_precond_L_symmetric_positive_and_distinct_from_diag_P(two_circ, two_bars_dense_P):
    f = 1e8
    QL = C.precond_matrix_L(two_circ, f, two_bars_dense_P)
    Q = C.precond_matrix(two_circ, f, two_bars_dense_P)
    assert np.max(np.abs(QL - QL.T)) == 0.0
    assert np.linalg.eigvalsh(QL.real).min() > 0
    assert np.linalg.eigvalsh(QL.imag).min() > 0
    # the sparsity of eq. 10 (loops touching a common panel), different values
    Mc = np.abs(two_circ.M[:, :two_circ.n_cb])
    touch = (Mc @ np.abs(two_circ.A).sum(axis=0)) > 0          # loop x panel
    S = (touch.astype(float) @ touch.T.astype(float)) > 0
    assert not np.any((QL != 0) & ~S) and not np.any((Q != 0) & ~S)
    assert np.max(np.abs(QL.imag - Q.imag)) > 1e-3 * np.max(np.abs(Q.imag))


def test_both_preconditioners_cut_gmres_iterations(bar_circ, bar_dense_P):
    """Dense restarted GMRES (restart 50, relative residual 1e-8) on the bar's
    loop system at 10 MHz: the diagonal-of-P (eq. 10) and the diagonal-of-L
    preconditioners, applied exactly, each need under a fifth of the
    unpreconditioned iterations.  (Their own counts differ by about one here:
    both keep the loop-space Z_s whole, so they differ only in the inductive
    couplings of branches that share a panel.)"""
    import scipy.linalg as la
    import scipy.sparse.linalg as sla
    c = bar_circ
    f = 1e7
    Pl = bar_dense_P[np.ix_(c.live, c.live)]
    Z = c.loop_matrix(f, c.potential_part(Pl))
    b = c.port_rhs()[:, 0].astype(complex)

    def iters(Q):
        n = [0]
        M = None
        if Q is not None:
            lu = la.lu_factor(Q)
            M = sla.LinearOperator(Z.shape, matvec=lambda v: la.lu_solve(lu, v), dtype=complex)
        x, info = sla.gmres(Z, b, M=M, rtol=1e-8, restart=50, maxiter=20,
                            callback=lambda r: n.__setitem__(0, n[0] + 1), callback_type="pr_norm")
        assert info == 0
        assert np.linalg.norm(Z @ x - b) <= 1e-7 * np.linalg.norm(b)
        return n[0]

    n0 = iters(None)
    nP = iters(C.precond_matrix(c, f, bar_dense_P))
    nL = iters(C.precond_matrix_L(c, f, bar_dense_P))
    assert nP < 0.2 * n0 and nL < 0.2 * n0, (n0, nP, nL)
