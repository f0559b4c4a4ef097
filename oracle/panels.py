"""Panel geometry and the dense panel potential matrix P (oracle, test only).

P_kl = (1 / (A_k A_l)) * int_{S_k} int_{S_l} 1 / |r - r'| dS' dS      (units 1/m)

is the frequency-independent kernel of eq. 6 after the centroid-midpoint
transformation (Sec. II-A, eq. 4-6; the 1/(A_k A_l) normalisation is the
reading in which the panel current coefficient is J_l * A_l, see circuit.py).
The fast product of Sec. II-C approximates exactly this matrix.

Entries are evaluated by a fixed rule table (the paper names no quadrature):
with d = |c_k - c_l|, r = max centroid-to-vertex distance and
q = d / (r_k + r_l), and (lo, hi) = (min(k, l), max(k, l)):

  k == l            closed form (4/3) sum_sides (1/a) ln(s / (s - 2a)), s = perimeter
  shared edge       average of the two one-sided semi-analytic integrals, outer
                    rule edge_graded(10, 3) on the outer panel
  shared vertex     same, outer rule vertex_graded(10, 3)
  q < 1.5           one-sided semi-analytic: outer rule collapsed(8) on lo,
                    analytic potential of hi
  1.5 <= q < 3      one-sided semi-analytic, outer rule collapsed(5) on lo
  3 <= q < 10       point product rule collapsed(4) x collapsed(4), lo outer
  q >= 10           point product rule collapsed(3) x collapsed(3), lo outer

Rectangular panels (Sec. II-A: "triangular and rectangular supports") are
parallelograms (v0, v1, v2, v3).  The integral over a rectangle is the sum of
the integrals over its two triangles (v0, v1, v2) and (v0, v2, v3), so with
sub-triangle areas a_i and panel areas A_k

  P_kl = sum_{i in k} sum_{j in l} (a_i / A_k) (a_j / A_l) P^tri_ij,

where P^tri is the triangle rule table above applied to the sub-triangles
(numbered panel by panel, so (lo, hi) follows the panel order).  The two
halves of one rectangle share its diagonal and take the shared-edge rule.
For a triangle-only mesh the weights are exactly 1 and P = P^tri.

"Semi-analytic" means the inner integral is the closed-form potential of a
uniformly charged flat triangle (tri_potential) evaluated at the outer rule's
points.  The rule table gives per-entry errors <= 2e-8 relative (measured
against adaptive quadrature in the tests) and an exactly symmetric P: every
entry is computed from the ordered pair (lo, hi), and the two-sided averages
add the same two numbers in the same order for (k, l) and (l, k).
"""
import numpy as np

from . import quadrature as qd

# class boundaries in q = d / (r_k + r_l) and rule orders (see module doc)
Q_NEAR = 1.5
Q_SEMI = 3.0
Q_FAR = 10.0
EDGE_RULE = (10, 3)
VERTEX_RULE = (10, 3)
NEAR_RULE = 8
SEMI_RULE = 5
MID_RULE = 4
FAR_RULE = 3


class Geometry:
    """Per-panel vertices, centroid, area, unit normal and radius (FP64)."""

    def __init__(self, xyz, tri):
        self.tri = np.asarray(tri, np.int64)
        self.v = np.asarray(xyz, float)[self.tri]            # [N, 3, 3]
        self.c = (self.v[:, 0] + self.v[:, 1] + self.v[:, 2]) / 3.0
        cr = np.cross(self.v[:, 1] - self.v[:, 0], self.v[:, 2] - self.v[:, 0])
        nn = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * nn
        self.normal = cr / nn[:, None]
        self.radius = np.max(np.linalg.norm(self.v - self.c[:, None, :], axis=2), axis=1)

    @property
    def n(self):
        return self.v.shape[0]


def tri_potential(x, v):
    """int_T 1/|x - r'| dS' for uniformly charged flat triangles.

    x: [M, 3] points, v: [M, 3, 3] triangles (one per point).  Closed form of
    Wilton et al. (1984) / Graglia (1993): with w0 the height of x over the
    plane, rho its projection, and per edge the signed distance P0 of rho to
    the edge line (positive inside), the edge-parallel coordinates l-, l+ of
    the endpoints relative to rho and the distances R-, R+ to them,
      Phi = sum_edges [ P0 ln((R+ + l+)/(R- + l-))
                        - |w0| (atan(P0 l+/(R0^2 + |w0| R+)) - atan(P0 l-/(R0^2 + |w0| R-))) ],
    R0^2 = P0^2 + w0^2.  ln(R + l) is evaluated as ln(R0^2 / (R - l)) for
    l < 0 to avoid cancellation.
    """
    x = np.asarray(x, float)
    v0, v1, v2 = v[:, 0], v[:, 1], v[:, 2]
    n = np.cross(v1 - v0, v2 - v0)
    n /= np.linalg.norm(n, axis=1)[:, None]
    w0 = np.einsum("ij,ij->i", x - v0, n)
    aw = np.abs(w0)
    rho = x - w0[:, None] * n
    tot = np.zeros(x.shape[0])
    with np.errstate(divide="ignore", invalid="ignore"):
        for i in range(3):
            a = v[:, i]
            b = v[:, (i + 1) % 3]
            L = b - a
            lh = L / np.linalg.norm(L, axis=1)[:, None]
            u = np.cross(lh, n)
            P0 = np.einsum("ij,ij->i", a - rho, u)
            lm = np.einsum("ij,ij->i", a - rho, lh)
            lp = np.einsum("ij,ij->i", b - rho, lh)
            Rm = np.linalg.norm(a - x, axis=1)
            Rp = np.linalg.norm(b - x, axis=1)
            R0s = P0 * P0 + w0 * w0
            lnp = np.where(lp >= 0, np.log(Rp + lp), np.log(R0s / (Rp - lp)))
            lnm = np.where(lm >= 0, np.log(Rm + lm), np.log(R0s / (Rm - lm)))
            tot += np.where(P0 != 0.0, P0 * (lnp - lnm), 0.0)
            beta = (np.arctan(P0 * lp / (R0s + aw * Rp)) -
                    np.arctan(P0 * lm / (R0s + aw * Rm)))
            tot -= np.where(aw > 0.0, aw * beta, 0.0)
    return tot


def self_term(v):
    """P_kk for triangles v [M,3,3]: (1/A^2) int_T int_T 1/|r - r'|.

    Closed form (4/3) sum_{sides a} (1/a) ln(s / (s - 2 a)), s = a + b + c.
    """
    a = np.linalg.norm(v[:, 1] - v[:, 2], axis=1)
    b = np.linalg.norm(v[:, 2] - v[:, 0], axis=1)
    c = np.linalg.norm(v[:, 0] - v[:, 1], axis=1)
    s = a + b + c
    return (4.0 / 3.0) * (np.log(s / (s - 2 * a)) / a + np.log(s / (s - 2 * b)) / b +
                          np.log(s / (s - 2 * c)) / c)


def _semi(vo, vi, ai, coef, w):
    """One-sided semi-analytic entries: average over outer triangles vo
    (rule coef/w applied to the vertex triples given) of the potential of
    inner triangles vi, divided by inner areas ai."""
    M = vo.shape[0]
    Q = coef.shape[0]
    pts = np.einsum("qj,mjk->mqk", coef, vo).reshape(M * Q, 3)
    inner = np.repeat(vi, Q, axis=0)
    phi = tri_potential(pts, inner).reshape(M, Q)
    return (phi @ w) / ai


def _reorder_shared(G, outer, inner, kind):
    """Vertex triples of the outer panels arranged for the graded rules.

    kind 'edge': (o, a, b) with o the vertex not shared, a = next, b = next.
    kind 'vertex': (a, b, o) with a the shared vertex, b = next, o = next.
    """
    to = G.tri[outer]
    ti = G.tri[inner]
    shared = (to[:, :, None] == ti[:, None, :]).any(axis=2)
    if kind == "edge":
        first = np.argmin(shared, axis=1)      # the one vertex not shared
    else:
        first = np.argmax(shared, axis=1)      # the one shared vertex
    idx = (first[:, None] + np.arange(3)[None, :]) % 3
    return np.take_along_axis(G.v[outer], idx[:, :, None], axis=1)


def pair_values(G, K, L):
    """P_kl for arbitrary index pairs (vectors K, L of equal length)."""
    K = np.asarray(K, np.int64)
    L = np.asarray(L, np.int64)
    lo = np.minimum(K, L)
    hi = np.maximum(K, L)
    out = np.empty(K.shape[0])
    tl = G.tri[lo]
    th = G.tri[hi]
    nshare = (tl[:, :, None] == th[:, None, :]).any(axis=2).sum(axis=1)
    d = np.linalg.norm(G.c[lo] - G.c[hi], axis=1)
    q = d / (G.radius[lo] + G.radius[hi])
    is_self = lo == hi
    if np.any((nshare == 3) & ~is_self):
        raise ValueError("duplicate triangles")
    cls_edge = ~is_self & (nshare == 2)
    cls_vert = ~is_self & (nshare == 1)
    free = ~is_self & (nshare == 0)
    cls_near = free & (q < Q_NEAR)
    cls_semi = free & (q >= Q_NEAR) & (q < Q_SEMI)
    cls_mid = free & (q >= Q_SEMI) & (q < Q_FAR)
    cls_far = free & (q >= Q_FAR)

    if np.any(is_self):
        out[is_self] = self_term(G.v[lo[is_self]])

    def symmetric(mask, rule, kind):
        a = lo[mask]
        b = hi[mask]
        coef, w = rule
        if kind is None:
            va = G.v[a]
            vb = G.v[b]
        else:
            va = _reorder_shared(G, a, b, kind)
            vb = _reorder_shared(G, b, a, kind)
        s1 = _semi(va, G.v[b], G.area[b], coef, w)
        s2 = _semi(vb, G.v[a], G.area[a], coef, w)
        out[mask] = (s1 + s2) * 0.5

    if np.any(cls_edge):
        symmetric(cls_edge, qd.edge_graded(*EDGE_RULE), "edge")
    if np.any(cls_vert):
        symmetric(cls_vert, qd.vertex_graded(*VERTEX_RULE), "vertex")
    def one_sided(mask, order):
        a = lo[mask]
        b = hi[mask]
        coef, w = qd.collapsed(order)
        out[mask] = _semi(G.v[a], G.v[b], G.area[b], coef, w)

    def product(mask, order):
        a = lo[mask]
        b = hi[mask]
        coef, w = qd.collapsed(order)
        pa = np.einsum("qj,mjk->mqk", coef, G.v[a])
        pb = np.einsum("qj,mjk->mqk", coef, G.v[b])
        r = np.linalg.norm(pa[:, :, None, :] - pb[:, None, :, :], axis=3)
        out[mask] = np.einsum("i,j,mij->m", w, w, 1.0 / r)

    if np.any(cls_near):
        one_sided(cls_near, NEAR_RULE)
    if np.any(cls_semi):
        one_sided(cls_semi, SEMI_RULE)
    if np.any(cls_mid):
        product(cls_mid, MID_RULE)
    if np.any(cls_far):
        product(cls_far, FAR_RULE)
    return out


def dense_P(G, chunk=200000):
    """Full symmetric P (N x N), FP64."""
    N = G.n
    iu, ju = np.triu_indices(N)
    vals = np.empty(iu.shape[0])
    for s in range(0, iu.shape[0], chunk):
        vals[s:s + chunk] = pair_values(G, iu[s:s + chunk], ju[s:s + chunk])
    P = np.zeros((N, N))
    P[iu, ju] = vals
    P[ju, iu] = vals
    return P


_POOL_G = None


def _pool_init(xyz, tri):
    global _POOL_G
    _POOL_G = Geometry(xyz, tri)


def _pool_rows(args):
    """Upper-triangle entries P[r, r:] for rows r0..r1-1 of the pool's mesh."""
    r0, r1 = args
    N = _POOL_G.n
    K = np.concatenate([np.full(N - r, r, np.int64) for r in range(r0, r1)])
    L = np.concatenate([np.arange(r, N, dtype=np.int64) for r in range(r0, r1)])
    vals = np.empty(K.shape[0])
    for s in range(0, K.shape[0], 100000):
        vals[s:s + 100000] = pair_values(_POOL_G, K[s:s + 100000], L[s:s + 100000])
    return r0, r1, vals


def dense_P_parallel(xyz, tri, workers, block=48):
    """dense_P of a triangle mesh with the upper triangle's rows spread over a
    pool of `workers` processes (multiprocessing 'spawn', so that it may run
    next to a CUDA context); every entry is pair_values of its (row, column)
    pair as in dense_P, and the lower triangle mirrors the upper one."""
    import multiprocessing as mp
    tri = np.asarray(tri, np.int64)
    N = tri.shape[0]
    P = np.zeros((N, N))
    tasks = [(r, min(N, r + block)) for r in range(0, N, block)]
    with mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(xyz, tri)) as pool:
        for r0, r1, vals in pool.imap_unordered(_pool_rows, tasks, chunksize=1):
            o = 0
            for r in range(r0, r1):
                P[r, r:] = vals[o:o + N - r]
                o += N - r
    for r0 in range(0, N, 1024):
        r1 = min(N, r0 + 1024)
        blk = P[r0:r1, r0:r1]
        P[r0:r1, r0:r1] = np.triu(blk) + np.triu(blk, 1).T
        P[r1:, r0:r1] = P[r0:r1, r1:].T
    return P


def rows_P(G, rows, chunk=200000):
    """Selected rows of P, shape [len(rows), N]."""
    rows = np.asarray(rows, np.int64)
    N = G.n
    K = np.repeat(rows, N)
    L = np.tile(np.arange(N), rows.shape[0])
    vals = np.empty(K.shape[0])
    for s in range(0, K.shape[0], chunk):
        vals[s:s + chunk] = pair_values(G, K[s:s + chunk], L[s:s + chunk])
    return vals.reshape(rows.shape[0], N)


class Panels:
    """Hybrid triangle/rectangle panels (Sec. II-A) as sub-triangles.

    pan: [N, 3] triangles, or [N, 4] with -1 in the last column for a
    triangle; a 4-vertex panel must be a parallelogram.  Attributes: c
    (vertex mean = centroid of a triangle or a parallelogram), area, normal,
    radius (max centroid-vertex distance), nv (3 or 4), sub (Geometry of the
    sub-triangles), sub_of (panel of each sub-triangle), w (a_i / A_k).
    """

    def __init__(self, xyz, pan):
        pan = np.asarray(pan, np.int64)
        if pan.shape[1] == 3:
            pan = np.hstack([pan, -np.ones((pan.shape[0], 1), np.int64)])
        self.pan = pan
        self.nv = np.where(pan[:, 3] >= 0, 4, 3)
        xyz = np.asarray(xyz, float)
        quad = self.nv == 4
        V = xyz[np.where(pan >= 0, pan, 0)]                  # [N, 4, 3]
        if np.any(quad):
            d = V[quad, 0] + V[quad, 2] - V[quad, 1] - V[quad, 3]
            span = np.linalg.norm(V[quad, 2] - V[quad, 0], axis=1)
            if np.any(np.linalg.norm(d, axis=1) > 1e-9 * span):
                raise ValueError("a rectangular panel is not a parallelogram")
        c3 = (V[:, 0] + V[:, 1] + V[:, 2]) / 3.0
        c4 = (((V[:, 0] + V[:, 1]) + V[:, 2]) + V[:, 3]) / 4.0
        self.c = np.where(quad[:, None], c4, c3)
        subs = []
        sub_of = []
        for k in range(pan.shape[0]):
            a, b, cc, dd = pan[k]
            subs.append((a, b, cc))
            sub_of.append(k)
            if dd >= 0:
                subs.append((a, cc, dd))
                sub_of.append(k)
        self.sub = Geometry(xyz, np.array(subs, np.int64))
        self.sub_of = np.array(sub_of, np.int64)
        self.area = np.bincount(self.sub_of, weights=self.sub.area, minlength=pan.shape[0])
        self.w = self.sub.area / self.area[self.sub_of]
        first = np.searchsorted(self.sub_of, np.arange(pan.shape[0]))
        self.normal = self.sub.normal[first]
        dist = np.linalg.norm(V - self.c[:, None, :], axis=2)
        dist[:, 3] = np.where(quad, dist[:, 3], 0.0)
        self.radius = dist.max(axis=1)

    @property
    def n(self):
        return self.pan.shape[0]

    @property
    def tri(self):
        """[N, 3] vertex ids of a triangle-only mesh."""
        if np.any(self.nv == 4):
            raise AttributeError("hybrid mesh: use pan")
        return self.pan[:, :3]

    @property
    def v(self):
        """[N, 3, 3] vertices of a triangle-only mesh."""
        return self.sub.v if not np.any(self.nv == 4) else None

    def weights(self):
        """W [N, N_sub] sparse, W[k, i] = a_i / A_k for the sub-triangles of k."""
        from scipy import sparse
        return sparse.csr_matrix((self.w, (self.sub_of, np.arange(self.sub_of.shape[0]))),
                                 shape=(self.n, self.sub_of.shape[0]))


def dense_P_panels(H, chunk=200000):
    """Full symmetric P over hybrid panels: W P^tri W^T."""
    W = H.weights()
    Ps = dense_P(H.sub, chunk)
    Pp = np.asarray((W @ (W @ Ps).T).T)
    return np.triu(Pp) + np.triu(Pp, 1).T          # exactly symmetric (upper triangle mirrored)


def rows_P_panels(H, rows, chunk=200000):
    """Selected rows of the hybrid P, shape [len(rows), N]."""
    rows = np.asarray(rows, np.int64)
    W = H.weights()
    sub_rows = np.flatnonzero(np.isin(H.sub_of, rows))
    R = rows_P(H.sub, sub_rows, chunk)                 # [n_sub_rows, N_sub]
    Rp = np.asarray((W @ R.T).T)                       # [n_sub_rows, N]
    out = np.zeros((rows.shape[0], H.n))
    pos = {int(r): i for i, r in enumerate(rows)}
    for t, si in enumerate(sub_rows):
        out[pos[int(H.sub_of[si])]] += H.w[si] * Rp[t]
    return out
