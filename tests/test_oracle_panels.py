"""Pins for oracle/panels.py: the triangle potential, the self term and the
rule table for P_kl = (1/(A_k A_l)) int int 1/|r - r'| (eq. 6)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import panels as P
from oracle import quadrature as qd


def brute_potential(x, v):
    """Adaptive 2-D quadrature of int_T 1/|x - r'| dS' (Duffy map, scipy)."""
    v0, v1, v2 = v
    A2 = np.linalg.norm(np.cross(v1 - v0, v2 - v0))

    def f(t, s):
        p = v0 + s * (v1 - v0) + t * (1 - s) * (v2 - v0)
        return (1 - s) * A2 / np.linalg.norm(x - p)
    val, _ = integrate.dblquad(f, 0, 1, 0, 1, epsabs=1e-13, epsrel=1e-12)
    return val


TRI = np.array([[0.1, -0.2, 0.05], [1.2, 0.1, -0.1], [0.3, 0.9, 0.2]])


@pytest.mark.parametrize("x", [
    [2.0, 1.5, -1.0],                      # far off-plane
    [0.5, 0.3, 0.4],                       # near, above
    [0.5, 0.3, -0.01],                     # very near, below
    None,                                  # centroid (in plane, inside)
    "edge",                                # in plane, on an edge's midpoint
    "out",                                 # in plane, outside
])
def test_potential_matches_brute_force(x):
    v = TRI
    if x is None:
        x = v.mean(0)
    elif x == "edge":
        x = 0.5 * (v[0] + v[1])
    elif x == "out":
        x = v[0] + 1.3 * (v[0] - v[2])
    x = np.asarray(x, float)
    got = P.tri_potential(x[None], v[None])[0]
    ref = brute_potential(x, v)
    assert abs(got - ref) / ref < 1e-10


def test_potential_point_charge_limit():
    v = TRI
    A = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    c = v.mean(0)
    errs = []
    for R in [30.0, 300.0]:
        x = c + R * np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
        got = P.tri_potential(x[None], v[None])[0]
        # monopole about the centroid plus an O(R^-2) relative quadrupole term
        errs.append(abs(got * R / A - 1.0))
        assert errs[-1] < 2.0 / R ** 2
    assert errs[1] < errs[0] / 50


def _self_by_edge_identity(v):
    """Independent route to int_T int_T 1/R: scaling the triangle about its
    centroid, d/dlambda I(lambda T) = 3 I = 2 sum_edges h_i int_edge Phi_T ds
    (Reynolds transport), with h_i the centroid-edge distance."""
    c = v.mean(0)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    tot = 0.0
    for i in range(3):
        a, b = v[i], v[(i + 1) % 3]
        L = b - a
        le = np.linalg.norm(L)
        u = np.cross(L / le, n)
        h = np.dot(a - c, u)
        val, _ = integrate.quad(lambda s: P.tri_potential((a + s * L)[None], v[None])[0] * le,
                                0, 1, epsabs=1e-15, epsrel=1e-13, limit=200)
        tot += 2 * h * val
    return tot / 3.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_self_term_matches_edge_identity(seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, 3))
    A = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    got = P.self_term(v[None])[0] * A * A
    ref = _self_by_edge_identity(v)
    assert abs(got - ref) / ref < 1e-9


def _classify(G, k, l):
    nshare = len(set(G.tri[k]) & set(G.tri[l]))
    q = np.linalg.norm(G.c[k] - G.c[l]) / (G.radius[k] + G.radius[l])
    return nshare, q


def _reference_entry(G, k, l):
    """High-accuracy value of P_kl: adaptive outer quadrature of the analytic
    inner potential for touching pairs, a 16x16 collapsed rule otherwise."""
    nshare, q = _classify(G, k, l)
    if nshare > 0:
        vk = G.v[k]
        A2 = 2 * G.area[k]

        def f(t, s):
            p = vk[0] + s * (vk[1] - vk[0]) + t * (1 - s) * (vk[2] - vk[0])
            return (1 - s) * A2 * P.tri_potential(p[None], G.v[l][None])[0]
        val, _ = integrate.dblquad(f, 0, 1, 0, 1, epsabs=1e-16, epsrel=1e-11)
        return val / (G.area[k] * G.area[l])
    coef, w = qd.collapsed(16)
    s1 = P._semi(G.v[[k]], G.v[[l]], G.area[[l]], coef, w)[0]
    s2 = P._semi(G.v[[l]], G.v[[k]], G.area[[k]], coef, w)[0]
    return 0.5 * (s1 + s2)


def test_rule_table_accuracy_by_class(bar_mesh):
    G = P.Geometry(bar_mesh.xyz, bar_mesh.tri)
    rng = np.random.default_rng(5)
    picked = {}
    k0 = 700                       # a panel on a side face, away from the ends
    for l in rng.permutation(G.n):
        nshare, q = _classify(G, k0, l)
        if l == k0:
            continue
        if nshare == 2:
            cls = "edge"
        elif nshare == 1:
            cls = "vertex"
        elif q < P.Q_NEAR:
            cls = "near"
        elif q < P.Q_SEMI:
            cls = "semi"
        elif q < P.Q_FAR:
            cls = "mid"
        else:
            cls = "far"
        if len(picked.setdefault(cls, [])) < 2:
            picked[cls].append(l)
    assert set(picked) == {"edge", "vertex", "near", "semi", "mid", "far"}
    tol = {"edge": 5e-8, "vertex": 5e-8, "near": 2e-8, "semi": 2e-8, "mid": 2e-8, "far": 2e-8}
    for cls, ls in picked.items():
        for l in ls:
            got = P.pair_values(G, [k0], [l])[0]
            ref = _reference_entry(G, k0, l)
            assert abs(got - ref) / ref < tol[cls], (cls, l, got, ref)


def test_dense_P_symmetric_positive_definite(two_bars_dense_P):
    Pm = two_bars_dense_P
    assert np.array_equal(Pm, Pm.T)
    assert np.linalg.eigvalsh(Pm).min() > 0


def test_scaling_and_rigid_motion():
    import meshgen
    m = meshgen.bar(length=2e-3, n_l=10, n_w=2, n_h=2, seed=3)
    G = P.Geometry(m.xyz, m.tri)
    P1 = P.dense_P(G)
    s = 3.7
    # a rotation about an axis plus a translation, then scale by s
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    xyz2 = s * (m.xyz @ R.T) + np.array([1e-3, -2e-3, 5e-4])
    P2 = P.dense_P(P.Geometry(xyz2, m.tri))
    assert np.max(np.abs(P2 * s - P1) / np.abs(P1)) < 1e-11


def test_rows_match_dense(two_bars_mesh, two_bars_dense_P):
    G = P.Geometry(two_bars_mesh.xyz, two_bars_mesh.tri)
    rows = [0, 17, G.n - 1]
    np.testing.assert_array_equal(P.rows_P(G, rows), two_bars_dense_P[rows])


def test_parallel_dense_matches_serial(two_bars_mesh, two_bars_dense_P):
    """The spawn-pool evaluator of the stored package sweep: the serial dense
    P's entries, with a block size that leaves a ragged last block.  The pair
    batches differ in size, and numpy's vectorised sums may round a batch
    differently (seen: 1 ulp on 0.01% of the entries), so rtol 1e-14."""
    Pp = P.dense_P_parallel(two_bars_mesh.xyz, two_bars_mesh.tri, workers=2, block=37)
    np.testing.assert_allclose(Pp, two_bars_dense_P, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(Pp, Pp.T)
