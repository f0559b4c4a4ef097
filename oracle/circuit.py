"""PEEC graph, centroid-midpoint transform, loop analysis and port R, L
(oracle, test infrastructure only).

Follows Sec. II-A (Fig. 1, Algorithm 1, eq. 4-6), Sec. II-B (eq. 7),
Sec. II-C (eq. 8-9) and Sec. III (ports placed as in Q3D, eq. 12).

Readings taken where the paper is silent or garbled:

* Nodes are the centroids of non-terminal panels plus one node per terminal
  (a terminal is a patch of panels collapsed into one equipotential node
  that carries no current).  An edge shared by two non-terminal panels is an
  internal branch oriented from the lower to the higher panel index; an edge
  between a non-terminal panel and a terminal panel is a rim branch from the
  panel to the terminal node; edges inside one terminal are dropped.  Every
  edge must lie in exactly two panels (closed conductor surfaces).
* Algorithm 1 rows are indexed by the global branch (its "k" and "l" are read
  as the global edge), and "same direction" is read as: the panel is the
  branch's tail.  So A_t(b, tail) = +rho_t, A_t(b, head) = -rho_t with
  rho = m_e - c_p, and the panel coefficient I_pt = A_t^T I_edge equals
  J_t * area for a uniform current density J (the identity pinned in tests).
* With that normalisation the Galerkin matrix of eq. 6 becomes
  Z_kl = (Z_s / A_l) delta_kl + (j omega mu0 / 4 pi) P_kl, P_kl as in panels.py.
* Each port adds an ideal external branch from its sink terminal node to its
  source terminal node carrying a 1 V source; the port current is the
  current in that branch; Y = B^T Z_loop^-1 B, Z_port = Y^-1, R = Re Z_port,
  L = Im Z_port / omega.
* The loop matrix M is the fundamental-cycle basis of a breadth-first
  spanning forest (Sec. II-B leaves the loop search to refs [6], [14]).
* The diagonal-of-L preconditioner "Z_s + j omega L_d" (Sec. II-D) is read
  with Z_s the loop-space surface impedance matrix of eq. 8 (kept whole, as
  in the operator) and L_d the diagonal of the branch-branch inductance
  mu0/4pi sum_t A_t P A_t^T, projected by M.
"""
from collections import deque

import numpy as np

from .esi import zs
from .panels import Panels

MU0_4PI = 1e-7


class Circuit:
    """PEEC graph, A_t and M of a mesh.

    sparse=True stores A_t as three scipy CSR matrices (the same entries,
    at most two per branch row) instead of one dense [3, n_cb, n_live]
    array, so that meshes of tens of thousands of panels fit in memory;
    every method accepts either form."""

    def __init__(self, mesh, sparse=False):
        self.mesh = mesh
        tri = np.asarray(mesh.tri, np.int64)
        term = np.asarray(mesh.term, np.int64)
        self.geom = Panels(mesh.xyz, tri)
        npan = tri.shape[0]
        self.panel_node = -np.ones(npan, np.int64)
        live = np.flatnonzero(term < 0)
        self.live = live                                   # current-carrying panels
        self.panel_node[live] = np.arange(live.shape[0])
        self.n_live = live.shape[0]
        self.n_term = int(term.max()) + 1 if term.size and term.max() >= 0 else 0
        self.n_nodes = self.n_live + self.n_term

        # edges: unordered vertex pairs -> the two panels containing them (a
        # triangle has 3 edges, a rectangle 4; its diagonal is not an edge)
        e_all = []
        owner = []
        for k in range(npan):
            vs = [int(x) for x in tri[k] if x >= 0]
            for i in range(len(vs)):
                e_all.append((vs[i], vs[(i + 1) % len(vs)]))
                owner.append(k)
        e_all = np.array(e_all, np.int64)
        owner = np.array(owner, np.int64)
        und = np.sort(e_all, axis=1)
        keys, inv, cnt = np.unique(und, axis=0, return_inverse=True, return_counts=True)
        inv = inv.ravel()
        if np.any(cnt != 2):
            raise ValueError("mesh is not a closed 2-manifold")
        order = np.argsort(inv, kind="stable")
        pan = owner[order].reshape(-1, 2)                  # [n_edges, 2]
        self.edge_vertices = keys

        tails = []
        heads = []
        ridx = []                                          # (edge, tail panel, head panel or -1)
        for e in range(keys.shape[0]):
            p, q = pan[e]
            tp, tq = term[p], term[q]
            if tp < 0 and tq < 0:
                a, b = min(p, q), max(p, q)
                tails.append(self.panel_node[a])
                heads.append(self.panel_node[b])
                ridx.append((e, a, b))
            elif tp >= 0 and tq >= 0:
                if tp != tq:
                    raise ValueError("two terminals touch")
            else:
                a, t = (p, tq) if tp < 0 else (q, tp)
                tails.append(self.panel_node[a])
                heads.append(self.n_live + t)
                ridx.append((e, a, -1))
        self.n_cb = len(ridx)                               # conductor branches
        ports = list(mesh.ports)
        self.n_port = len(ports)
        for s, k in ports:
            tails.append(self.n_live + k)                   # sink -> source
            heads.append(self.n_live + s)
        self.tail = np.array(tails, np.int64)
        self.head = np.array(heads, np.int64)
        self.n_branch = self.tail.shape[0]

        # centroid-midpoint matrices A_t (Algorithm 1): [n_cb, n_live] x 3,
        # A_t(b, tail) = +rho_t, A_t(b, head) = -rho_t, rho = m_e - c_p
        G = self.geom
        xyz = np.asarray(mesh.xyz, float)
        rows, cols, vals = [], [], []
        for b, (e, a, h) in enumerate(ridx):
            mid = 0.5 * (xyz[keys[e, 0]] + xyz[keys[e, 1]])
            rows.append(b)
            cols.append(self.panel_node[a])
            vals.append(mid - G.c[a])
            if h >= 0:
                rows.append(b)
                cols.append(self.panel_node[h])
                vals.append(-(mid - G.c[h]))
        rows = np.array(rows, np.int64)
        cols = np.array(cols, np.int64)
        vals = np.array(vals, float).reshape(-1, 3)
        if sparse:
            from scipy import sparse as sp
            self.A = [sp.csr_matrix((vals[:, t], (rows, cols)), shape=(self.n_cb, self.n_live))
                      for t in range(3)]
        else:
            self.A = np.zeros((3, self.n_cb, self.n_live))
            for t in range(3):
                np.add.at(self.A[t], (rows, cols), vals[:, t])
        self.branch_edge = np.array([r[0] for r in ridx], np.int64)
        self.M = self._loops()

    def incidence(self):
        """Node-branch incidence B [n_nodes, n_branch]: +1 at tail, -1 at head."""
        Bm = np.zeros((self.n_nodes, self.n_branch))
        Bm[self.tail, np.arange(self.n_branch)] = 1.0
        Bm[self.head, np.arange(self.n_branch)] = -1.0
        return Bm

    def _loops(self):
        """Fundamental cycles of a BFS spanning forest over conductor branches."""
        N = self.n_nodes
        adj = [[] for _ in range(N)]
        for b in range(self.n_cb):
            u, v = self.tail[b], self.head[b]
            adj[u].append((v, b))
            adj[v].append((u, b))
        for lst in adj:
            lst.sort()
        parent = -np.ones(N, np.int64)
        pbranch = -np.ones(N, np.int64)
        depth = -np.ones(N, np.int64)
        in_tree = np.zeros(self.n_branch, bool)
        for root in range(N):
            if depth[root] >= 0:
                continue
            depth[root] = 0
            dq = deque([root])
            while dq:
                u = dq.popleft()
                for v, b in adj[u]:
                    if depth[v] < 0:
                        depth[v] = depth[u] + 1
                        parent[v] = u
                        pbranch[v] = b
                        in_tree[b] = True
                        dq.append(v)
        loops = []
        for b in range(self.n_branch):
            if in_tree[b]:
                continue
            row = np.zeros(self.n_branch)
            row[b] = 1.0
            # walk from head back to tail through the tree: the loop goes
            # tail -> head along b, then head -> ... -> tail in the tree
            u = self.head[b]
            v = self.tail[b]
            path_u = []
            path_v = []
            uu, vv = u, v
            while depth[uu] > depth[vv]:
                path_u.append(uu)
                uu = parent[uu]
            while depth[vv] > depth[uu]:
                path_v.append(vv)
                vv = parent[vv]
            while uu != vv:
                if parent[uu] < 0 or parent[vv] < 0:
                    raise ValueError("port joins two disconnected conductors")
                path_u.append(uu)
                uu = parent[uu]
                path_v.append(vv)
                vv = parent[vv]
            # from head up to the common ancestor: traverse node -> parent
            for x in path_u:
                tb = pbranch[x]
                row[tb] += 1.0 if self.tail[tb] == x else -1.0
            # from the common ancestor down to tail: traverse parent -> node
            for x in path_v:
                tb = pbranch[x]
                row[tb] += 1.0 if self.head[tb] == x else -1.0
            loops.append(row)
        return np.array(loops)

    # ---- loop system (eq. 7-8) -------------------------------------------------

    def port_rhs(self):
        """B_port [n_loops, n_port]: column p = M[:, port branch p] (1 V sources)."""
        return self.M[:, self.n_cb:].copy()

    def zs_panels(self, f):
        """Z_s(f) / A_l for the live panels (eq. 3 per panel conductor)."""
        cond = np.asarray(self.mesh.cond)[self.live]
        sig = np.asarray(self.mesh.sigma)[cond]
        thk = np.asarray(self.mesh.thickness)[cond]
        return zs(f, sig, thk) / self.geom.area[self.live]

    def ma(self):
        """M A_t restricted to conductor branches: [3, n_loops, n_live]."""
        Mc = self.M[:, :self.n_cb]
        return np.stack([np.asarray(Mc @ self.A[t]) for t in range(3)])

    def potential_part(self, P_live, MA=None):
        """G = sum_t (M A_t) P (M A_t)^T, real and frequency independent."""
        MA = self.ma() if MA is None else MA
        return sum(MA[t] @ P_live @ MA[t].T for t in range(3))

    def resistive_parts(self, MA=None):
        """The resistive part of eq. 8 grouped by material.

        Z_s of eq. 3 depends only on a conductor's (sigma, thickness), so
        sum_t (M A_t) diag(Z_s/A) (M A_t)^T = sum_m Z_s^m(f) K_m with the
        frequency-independent K_m = sum_t (M A_t) diag(1/A_l [l in m]) (M A_t)^T
        over the distinct materials m.  Returns [(sigma, thickness, K_m)]."""
        MA = self.ma() if MA is None else MA
        cond = np.asarray(self.mesh.cond)[self.live]
        sig = np.asarray(self.mesh.sigma, float)[cond]
        thk = np.asarray(self.mesh.thickness, float)[cond]
        inv_a = 1.0 / self.geom.area[self.live]
        out = []
        for s_, t_ in sorted(set(zip(sig.tolist(), thk.tolist()))):
            w = np.where((sig == s_) & (thk == t_), inv_a, 0.0)
            out.append((s_, t_, sum((MA[t] * w[None, :]) @ MA[t].T for t in range(3))))
        return out

    def loop_matrix(self, f, Gpot, parts=None):
        """Z_loop(f) = sum_t (M A_t) diag(Z_s/A) (M A_t)^T + j omega mu0/4pi G
        (parts: resistive_parts(), the same sum grouped by material)."""
        if parts is None:
            MA = self.ma()
            d = self.zs_panels(f)
            R = sum((MA[t] * d[None, :]) @ MA[t].T for t in range(3))
        else:
            R = sum(complex(zs(f, s_, t_)) * K for s_, t_, K in parts)
        return R + 1j * 2 * np.pi * f * MU0_4PI * Gpot

    def solve(self, freqs, P_full):
        """Port R, L per frequency by dense direct solve; also loop currents."""
        P_live = P_full[np.ix_(self.live, self.live)]
        MA = self.ma()
        Gpot = self.potential_part(P_live, MA)
        del P_live
        parts = self.resistive_parts(MA)
        del MA
        B = self.port_rhs()
        R = []
        L = []
        X = []
        for f in freqs:
            Z = self.loop_matrix(f, Gpot, parts)
            x = np.linalg.solve(Z, B.astype(complex))
            del Z
            Y = B.T @ x
            Zp = np.linalg.inv(Y)
            R.append(Zp.real)
            L.append(Zp.imag / (2 * np.pi * f) if f > 0 else np.full_like(Zp.real, np.nan))
            X.append(x)
        return np.array(R), np.array(L), X

    def panel_currents(self, x):
        """I_pt = A_t^T M^T x for loop currents x [n_loops, k] -> [3, n_live, k]."""
        ie = self.M[:, :self.n_cb].T @ x
        return np.stack([self.A[t].T @ ie for t in range(3)])


def mna_port_admittance(circ, f, P_full):
    """Port admittance Y by nodal (MNA) analysis, no loops (cross-check).

    Unknowns: conductor branch currents, node potentials, port branch
    currents.  Rows: branch equations (Z I)_b - (phi_tail - phi_head) = 0,
    port rows phi_source - phi_sink = E_p, KCL at every node, and one
    grounded node per connected component.
    """
    P_live = P_full[np.ix_(circ.live, circ.live)]
    nb = circ.n_cb
    nn = circ.n_nodes
    npt = circ.n_port
    d = circ.zs_panels(f)
    Zb = sum(circ.A[t] @ (np.diag(d) + 1j * 2 * np.pi * f * MU0_4PI * P_live) @ circ.A[t].T
             for t in range(3))
    n = nb + nn + npt
    K = np.zeros((n + nn, n), complex)
    rows = 0
    K[:nb, :nb] = Zb
    for b in range(nb):
        K[b, nb + circ.tail[b]] -= 1.0
        K[b, nb + circ.head[b]] += 1.0
    rows = nb
    for p in range(npt):
        b = nb + p
        K[rows + p, nb + circ.head[b]] = 1.0    # source node
        K[rows + p, nb + circ.tail[b]] = -1.0   # sink node
    rows += npt
    for b in range(circ.n_branch):
        col = b if b < nb else nb + nn + (b - nb)
        K[rows + circ.tail[b], col] += 1.0
        K[rows + circ.head[b], col] -= 1.0
    rows += nn
    # ground one node per component (over all branches)
    comp = -np.ones(nn, np.int64)
    adj = [[] for _ in range(nn)]
    for b in range(circ.n_branch):
        adj[circ.tail[b]].append(circ.head[b])
        adj[circ.head[b]].append(circ.tail[b])
    grounds = []
    for r in range(nn):
        if comp[r] >= 0:
            continue
        comp[r] = r
        grounds.append(r)
        dq = deque([r])
        while dq:
            u = dq.popleft()
            for v in adj[u]:
                if comp[v] < 0:
                    comp[v] = r
                    dq.append(v)
    Kg = np.zeros((len(grounds), n), complex)
    for i, g in enumerate(grounds):
        Kg[i, nb + g] = 1.0
    Kfull = np.vstack([K[:rows], Kg])
    rhs = np.zeros((Kfull.shape[0], npt), complex)
    for p in range(npt):
        rhs[nb + p, p] = 1.0
    sol, *_ = np.linalg.lstsq(Kfull, rhs, rcond=None)
    return sol[nb + nn:, :]                         # port currents: Y[q, p]


def precond_matrix_L(circ, f, P_full, M=None):
    """Diagonal-of-L preconditioner, the comparison of Sec. II-D and Table IV:
    Z_s + j omega L_d, with Z_s the loop-space surface impedance matrix of
    eq. 8 kept whole and L_d the diagonal of the edge-edge interaction matrix
    mu0/4pi sum_t A_t P A_t^T, taken over conductor branches and projected by
    the loop matrix:
        Q_L(f) = sum_t (M A_t) diag(Z_s/A) (M A_t)^T
                 + j omega mu0/4pi M_c diag(sum_t A_t P A_t^T) M_c^T.
    M: another loop basis over the same branches (default: the oracle's)."""
    P_live = P_full[np.ix_(circ.live, circ.live)]
    Mc = (circ.M if M is None else np.asarray(M))[:, :circ.n_cb]
    MA = np.stack([Mc @ circ.A[t] for t in range(3)])
    d = circ.zs_panels(f)
    R = sum((MA[t] * d[None, :]) @ MA[t].T for t in range(3))
    Ld = np.diag(sum(circ.A[t] @ P_live @ circ.A[t].T for t in range(3)))
    return R + 1j * 2 * np.pi * f * MU0_4PI * ((Mc * Ld[None, :]) @ Mc.T)


def precond_matrix(circ, f, P_full, M=None):
    """Diagonal-of-P preconditioner of eq. 10 (Sec. II-D), dense:
    Q(f) = sum_t (M A_t) diag(Z_s/A + j omega mu0/4pi P_ll) (M A_t)^T.
    M: another loop basis over the same branches (default: the oracle's)."""
    pd = np.diag(P_full)[circ.live]
    d = circ.zs_panels(f) + 1j * 2 * np.pi * f * MU0_4PI * pd
    Mc = (circ.M if M is None else np.asarray(M))[:, :circ.n_cb]
    MA = np.stack([Mc @ circ.A[t] for t in range(3)])
    return sum((MA[t] * d[None, :]) @ MA[t].T for t in range(3))
