// PEEC topology, centroid-midpoint transform, loop basis and the sparse
// diagonal-of-P preconditioner pencil (host C++, setup only).
//
// Sec. II-A (Fig. 1, Algorithm 1): panel centroids are circuit nodes and a
// shared edge is a branch; rho = m_e - c_p enters A_t(branch, panel) with
// sign + on the branch's tail panel and - on its head panel, so that
// I_pt = A_t^T I_edge is the panel current density times the panel area.
// Branch rules (the paper draws them only): an edge between two current-
// carrying panels is oriented from the lower to the higher panel index; an
// edge between a current-carrying panel and a terminal patch runs from the
// panel to the terminal node (a terminal patch is one equipotential node
// with no surface current); edges inside one terminal patch are dropped.
// Branches are numbered in the lexicographic order of their sorted vertex
// pairs, then one external branch per port (sink -> source).
//
// Sec. II-B leaves the loop search to the literature; this library builds a
// sparse basis (not the fundamental cycles of a spanning tree):
//  * a vertex loop for every mesh vertex that keeps a branch, circulating
//    around the vertex (it crosses each incident edge from the panel in
//    which the edge's other end precedes the vertex to the panel in which it
//    follows it, on a consistently oriented copy of the mesh); the vertex
//    loops of one closed component sum to zero, so the lowest vertex of each
//    component is skipped;
//  * 2g global loops per component of genus g from a tree-cotree split
//    (primal BFS forest T over the vertices, dual BFS forest C over the
//    branches not in T; each branch left over closes a cycle through C);
//  * one loop per port: the port branch closed through C.
// The count equals branches - nodes + components (checked), and every loop
// is verified to be a cycle (M B^T = 0).
#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <numeric>
#include <unordered_map>

#include "xrl_internal.hpp"

namespace xrl {

namespace {

struct UF {
  std::vector<int> p;
  explicit UF(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int f(int x) {
    while (p[x] != x) x = p[x] = p[p[x]];
    return x;
  }
  void u(int a, int b) {
    a = f(a);
    b = f(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

}  // namespace

void build_topology(xrl_ctx* c) {
  Topo& T = c->topo;
  const int N = c->N;
  const int nv = (int)(c->xyz.size() / 3);
  const auto& pan = c->pan;
  auto nvert = [&](int p) { return panel_nv(pan, p); };
  // terminals from port panel lists (identical lists share a terminal)
  std::vector<int> term(N, -1);
  std::map<std::vector<int32_t>, int> term_id;
  std::vector<std::pair<int, int>> ports;   // (source terminal, sink terminal)
  auto get_term = [&](std::vector<int32_t> lst) {
    std::sort(lst.begin(), lst.end());
    auto it = term_id.find(lst);
    if (it != term_id.end()) return it->second;
    int id = (int)term_id.size();
    for (int p : lst) {
      XRL_CHECK(p >= 0 && p < N, XRL_EINVAL, "port panel index out of range");
      XRL_CHECK(term[p] < 0, XRL_EINVAL, "a panel belongs to two different terminals");
      term[p] = id;
    }
    term_id[lst] = id;
    return id;
  };
  for (size_t k = 0; k < c->port_src.size(); ++k) {
    int s = get_term(c->port_src[k]);
    int t = get_term(c->port_sink[k]);
    XRL_CHECK(s != t, XRL_EINVAL, "port source and sink are the same terminal");
    ports.push_back({s, t});
  }
  T.n_term = (int)term_id.size();
  T.n_port = (int)ports.size();
  T.live_of_panel.assign(N, -1);
  T.n_live = 0;
  for (int p = 0; p < N; ++p)
    if (term[p] < 0) T.live_of_panel[p] = T.n_live++;
  T.n_nodes = T.n_live + T.n_term;
  auto node_of = [&](int p) { return term[p] < 0 ? T.live_of_panel[p] : T.n_live + term[p]; };

  // edges
  struct HE {
    int a, b, p;
  };
  std::vector<HE> he;
  he.reserve(kPanEdges * (size_t)N);
  for (int p = 0; p < N; ++p) {
    const int nvp = nvert(p);
    for (int e = 0; e < nvp; ++e) {   // a rectangle's diagonal is not an edge
      int a = pan[4 * p + e], b = pan[4 * p + (e + 1) % nvp];
      XRL_CHECK(a != b, XRL_ETOPO, "degenerate panel");
      he.push_back({std::min(a, b), std::max(a, b), p});
    }
  }
  std::sort(he.begin(), he.end(), [](const HE& x, const HE& y) {
    return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.p < y.p);
  });
  const int ne = (int)he.size() / 2;
  for (int e = 0; e < ne; ++e) {
    XRL_CHECK(he[2 * e].a == he[2 * e + 1].a && he[2 * e].b == he[2 * e + 1].b &&
                  (2 * e + 2 >= (int)he.size() || he[2 * e + 2].a != he[2 * e].a ||
                   he[2 * e + 2].b != he[2 * e].b),
              XRL_ETOPO, "mesh is not a closed 2-manifold (an edge is not shared by exactly two panels)");
  }
  std::vector<int> edge_p(2 * ne), edge_v(2 * ne), edge_branch(ne, -1);
  for (int e = 0; e < ne; ++e) {
    edge_p[2 * e] = he[2 * e].p;
    edge_p[2 * e + 1] = he[2 * e + 1].p;
    edge_v[2 * e] = he[2 * e].a;
    edge_v[2 * e + 1] = he[2 * e].b;
  }
  // panel centroids (host copy, for rho)
  auto X = [&](int v, int k) { return c->xyz[3 * (size_t)v + k]; };
  std::vector<double> cen(3 * (size_t)N);
  for (int p = 0; p < N; ++p) panel_centroid_host(c->xyz, pan, p, &cen[3 * (size_t)p]);

  T.br_tail.clear();
  T.br_head.clear();
  for (int s = 0; s < 2; ++s) {
    T.br_pan[s].clear();
    T.br_rho[s].clear();
  }
  std::vector<int> branch_edge;
  for (int e = 0; e < ne; ++e) {
    int p = edge_p[2 * e], q = edge_p[2 * e + 1];
    int tp = term[p], tq = term[q];
    int tail_p, head_p, head_node;
    if (tp < 0 && tq < 0) {
      tail_p = std::min(p, q);
      head_p = std::max(p, q);
      head_node = T.live_of_panel[head_p];
    } else if (tp >= 0 && tq >= 0) {
      XRL_CHECK(tp == tq, XRL_ETOPO, "two different terminals touch");
      continue;
    } else {
      tail_p = tp < 0 ? p : q;
      head_p = -1;
      head_node = T.n_live + (tp < 0 ? tq : tp);
    }
    int b = (int)T.br_tail.size();
    edge_branch[e] = b;
    branch_edge.push_back(e);
    T.br_tail.push_back(T.live_of_panel[tail_p]);
    T.br_head.push_back(head_node);
    T.br_pan[0].push_back(tail_p);
    T.br_pan[1].push_back(head_p);
    double mid[3];
    for (int k = 0; k < 3; ++k) mid[k] = 0.5 * (X(edge_v[2 * e], k) + X(edge_v[2 * e + 1], k));
    for (int k = 0; k < 3; ++k) T.br_rho[0].push_back(mid[k] - cen[3 * tail_p + k]);
    for (int k = 0; k < 3; ++k) T.br_rho[1].push_back(head_p >= 0 ? -(mid[k] - cen[3 * head_p + k]) : 0.0);
  }
  T.n_cb = (int)T.br_tail.size();
  for (auto& pr : ports) {
    T.br_tail.push_back(T.n_live + pr.second);  // sink -> source
    T.br_head.push_back(T.n_live + pr.first);
  }
  T.n_branch = (int)T.br_tail.size();

  // consistent orientation (BFS over all mesh edges)
  std::vector<int> flip(N, -1);
  {
    std::vector<std::vector<std::pair<int, int>>> padj(N);   // (neighbour panel, edge)
    for (int e = 0; e < ne; ++e) {
      padj[edge_p[2 * e]].push_back({edge_p[2 * e + 1], e});
      padj[edge_p[2 * e + 1]].push_back({edge_p[2 * e], e});
    }
    auto dir = [&](int p, int a, int b) {   // +1 if p (as stored, then flipped) traverses a->b
      int s = 0;
      const int nvp = nvert(p);
      for (int k = 0; k < nvp; ++k)
        if (pan[4 * p + k] == a && pan[4 * p + (k + 1) % nvp] == b) s = 1;
        else if (pan[4 * p + k] == b && pan[4 * p + (k + 1) % nvp] == a) s = -1;
      return flip[p] ? -s : s;
    };
    for (int r = 0; r < N; ++r) {
      if (flip[r] >= 0) continue;
      flip[r] = 0;
      std::deque<int> dq{r};
      while (!dq.empty()) {
        int p = dq.front();
        dq.pop_front();
        for (auto& nb : padj[p]) {
          int q = nb.first, e = nb.second;
          int a = edge_v[2 * e], b = edge_v[2 * e + 1];
          if (flip[q] < 0) {
            flip[q] = 0;
            if (dir(q, a, b) == dir(p, a, b)) flip[q] = 1;
            dq.push_back(q);
          } else {
            XRL_CHECK(dir(q, a, b) == -dir(p, a, b), XRL_ETOPO, "surface is not orientable");
          }
        }
      }
    }
  }
  auto follows = [&](int p, int v, int a) {   // in oriented panel p, does a directly follow v?
    const int nvp = nvert(p);
    int o[4] = {pan[4 * p], pan[4 * p + 1], pan[4 * p + 2], pan[4 * p + 3]};
    if (flip[p]) std::swap(o[1], o[nvp - 1]);   // reversed cycle (v0, v_last, ..., v1)
    for (int k = 0; k < nvp; ++k)
      if (o[k] == v) return o[(k + 1) % nvp] == a;
    return false;
  };

  // vertex -> incident non-dropped edges
  std::vector<std::vector<int>> vedges(nv);
  for (int e = 0; e < ne; ++e)
    if (edge_branch[e] >= 0) {
      vedges[edge_v[2 * e]].push_back(e);
      vedges[edge_v[2 * e + 1]].push_back(e);
    }
  // components of the dual graph over conductor branches
  UF uf(T.n_nodes);
  for (int b = 0; b < T.n_cb; ++b) uf.u(T.br_tail[b], T.br_head[b]);

  std::vector<std::vector<std::pair<int, int8_t>>> loops;   // (branch, sign)
  std::vector<char> comp_seen(T.n_nodes, 0);
  int n_vl = 0;
  for (int v = 0; v < nv; ++v) {
    if (vedges[v].empty()) continue;
    int e0 = vedges[v][0];
    int comp = uf.f(T.br_tail[edge_branch[e0]]);
    if (!comp_seen[comp]) {   // lowest surviving vertex of this component: skipped
      comp_seen[comp] = 1;
      continue;
    }
    std::vector<std::pair<int, int8_t>> row;
    for (int e : vedges[v]) {
      int a = edge_v[2 * e] == v ? edge_v[2 * e + 1] : edge_v[2 * e];
      int p = edge_p[2 * e], q = edge_p[2 * e + 1];
      int src = follows(p, v, a) ? q : p;   // the panel in which a precedes v
      int b = edge_branch[e];
      row.push_back({b, (int8_t)(T.br_tail[b] == node_of(src) ? 1 : -1)});
    }
    std::sort(row.begin(), row.end());
    loops.push_back(row);
    ++n_vl;
  }
  T.n_vertex_loops = n_vl;

  // tree-cotree
  std::vector<char> inT(ne, 0);
  {
    std::vector<std::vector<std::pair<int, int>>> vadj(nv);
    for (int e = 0; e < ne; ++e)
      if (edge_branch[e] >= 0) {
        vadj[edge_v[2 * e]].push_back({edge_v[2 * e + 1], e});
        vadj[edge_v[2 * e + 1]].push_back({edge_v[2 * e], e});
      }
    for (auto& l : vadj) std::sort(l.begin(), l.end());
    std::vector<char> seen(nv, 0);
    for (int r = 0; r < nv; ++r) {
      if (seen[r] || vadj[r].empty()) continue;
      seen[r] = 1;
      std::deque<int> dq{r};
      while (!dq.empty()) {
        int u = dq.front();
        dq.pop_front();
        for (auto& nb : vadj[u])
          if (!seen[nb.first]) {
            seen[nb.first] = 1;
            inT[nb.second] = 1;
            dq.push_back(nb.first);
          }
      }
    }
  }
  std::vector<int> par(T.n_nodes, -1), pbr(T.n_nodes, -1), depth(T.n_nodes, -1);
  std::vector<char> inC(T.n_cb, 0);
  {
    std::vector<std::vector<std::pair<int, int>>> nadj(T.n_nodes);
    for (int b = 0; b < T.n_cb; ++b) {
      if (inT[branch_edge[b]]) continue;
      nadj[T.br_tail[b]].push_back({T.br_head[b], b});
      nadj[T.br_head[b]].push_back({T.br_tail[b], b});
    }
    for (auto& l : nadj) std::sort(l.begin(), l.end());
    for (int r = 0; r < T.n_nodes; ++r) {
      if (depth[r] >= 0) continue;
      depth[r] = 0;
      std::deque<int> dq{r};
      while (!dq.empty()) {
        int u = dq.front();
        dq.pop_front();
        for (auto& nb : nadj[u])
          if (depth[nb.first] < 0) {
            depth[nb.first] = depth[u] + 1;
            par[nb.first] = u;
            pbr[nb.first] = nb.second;
            inC[nb.second] = 1;
            dq.push_back(nb.first);
          }
      }
    }
  }
  auto close_through_C = [&](int b) {
    std::map<int, int> acc;
    acc[b] += 1;
    int uu = T.br_head[b], vv = T.br_tail[b];
    std::vector<int> pu, pv;
    while (depth[uu] > depth[vv]) { pu.push_back(uu); uu = par[uu]; }
    while (depth[vv] > depth[uu]) { pv.push_back(vv); vv = par[vv]; }
    while (uu != vv) {
      XRL_CHECK(par[uu] >= 0 && par[vv] >= 0, XRL_ETOPO,
                "a port (or global loop) joins two disconnected conductors");
      pu.push_back(uu); uu = par[uu];
      pv.push_back(vv); vv = par[vv];
    }
    for (int x : pu) acc[pbr[x]] += (T.br_tail[pbr[x]] == x) ? 1 : -1;
    for (int x : pv) acc[pbr[x]] += (T.br_head[pbr[x]] == x) ? 1 : -1;
    std::vector<std::pair<int, int8_t>> row;
    for (auto& kv : acc)
      if (kv.second != 0) row.push_back({kv.first, (int8_t)kv.second});
    return row;
  };
  int n_gl = 0;
  for (int b = 0; b < T.n_cb; ++b)
    if (!inT[branch_edge[b]] && !inC[b]) {
      loops.push_back(close_through_C(b));
      ++n_gl;
    }
  for (int pp = 0; pp < T.n_port; ++pp) {
    loops.push_back(close_through_C(T.n_cb + pp));
    ++n_gl;
  }
  T.n_global_loops = n_gl;
  T.n_loops = (int)loops.size();
  // count check: branches - nodes + components (ports inside components)
  {
    UF u2(T.n_nodes);
    for (int b = 0; b < T.n_branch; ++b) u2.u(T.br_tail[b], T.br_head[b]);
    int comps = 0;
    for (int n = 0; n < T.n_nodes; ++n)
      if (u2.f(n) == n) ++comps;
    XRL_CHECK(T.n_loops == T.n_branch - T.n_nodes + comps, XRL_ETOPO,
              "loop basis size does not match the cycle-space dimension (a terminal patch is not a disk?)");
  }
  // CSR + cycle check
  T.m_ptr.assign(T.n_loops + 1, 0);
  T.m_col.clear();
  T.m_val.clear();
  std::vector<int64_t> nodesum(T.n_nodes, 0);
  for (int l = 0; l < T.n_loops; ++l) {
    for (auto& pr : loops[l]) {
      T.m_col.push_back(pr.first);
      T.m_val.push_back(pr.second);
      nodesum[T.br_tail[pr.first]] += pr.second;
      nodesum[T.br_head[pr.first]] -= pr.second;
    }
    for (auto& pr : loops[l]) {
      XRL_CHECK(nodesum[T.br_tail[pr.first]] == 0 && nodesum[T.br_head[pr.first]] == 0, XRL_ETOPO,
                "internal: a loop is not a cycle");
    }
    T.m_ptr[l + 1] = (int64_t)T.m_col.size();
  }
  // transpose
  T.mt_ptr.assign(T.n_branch + 1, 0);
  for (int32_t b : T.m_col) T.mt_ptr[b + 1]++;
  for (int b = 0; b < T.n_branch; ++b) T.mt_ptr[b + 1] += T.mt_ptr[b];
  T.mt_col.assign(T.m_col.size(), 0);
  T.mt_val.assign(T.m_col.size(), 0);
  {
    std::vector<int64_t> pos(T.mt_ptr.begin(), T.mt_ptr.end() - 1);
    for (int l = 0; l < T.n_loops; ++l)
      for (int64_t k = T.m_ptr[l]; k < T.m_ptr[l + 1]; ++k) {
        int b = T.m_col[k];
        T.mt_col[pos[b]] = l;
        T.mt_val[pos[b]] = T.m_val[k];
        ++pos[b];
      }
  }
  // materials
  T.mat_of_cond.assign(c->sigma.size(), 0);
  T.mat_sigma.clear();
  T.mat_thick.clear();
  for (size_t k = 0; k < c->sigma.size(); ++k) {
    int m = -1;
    for (size_t j = 0; j < T.mat_sigma.size(); ++j)
      if (T.mat_sigma[j] == c->sigma[k] && T.mat_thick[j] == c->thick[k]) m = (int)j;
    if (m < 0) {
      m = (int)T.mat_sigma.size();
      T.mat_sigma.push_back(c->sigma[k]);
      T.mat_thick.push_back(c->thick[k]);
    }
    T.mat_of_cond[k] = m;
  }
  T.n_mat = (int)T.mat_sigma.size();
}

// Pencil of the preconditioner Q(f) over the loops: every stored entry keeps
// n_mat + 1 coefficients, Q_ij(f) = sum_m Z_s,m(f) v_m + j omega mu0/4pi v_nm.
// The surface-impedance part is the loop-space Z_s of eq. 8 in both forms,
// sum_t (M A_t) diag(Z_s/A) (M A_t)^T, assembled panel by panel over the
// pairs of branches that touch the panel.  The potential part is
//  * p12 == NULL, diagonal-of-P (eq. 10): sum_t (M A_t) diag(P_ll) (M A_t)^T;
//  * p12 != NULL, diagonal-of-L (the comparison preconditioner of Sec. II-D,
//    Table IV): M diag(G_b) M^T with G_b = sum_t A_t P A_t^T on the branches.
//    A branch touches at most two panels (tail s = 0, head s = 1), so with the
//    signed rho of A_t, (G_b)_bb = sum_s |rho_s|^2 P_ss + 2 (rho_0 . rho_1) P_01.
// Both have the sparsity of "loops that touch a common panel", so the banded
// factorisation serves both.
void build_precond_pattern(xrl_ctx* c, const std::vector<double>& pdiag, const std::vector<double>* p12) {
  Topo& T = c->topo;
  const int N = c->N;
  const int nm = T.n_mat;
  const int W = nm + 1;
  auto dot3 = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  std::unordered_map<uint64_t, std::vector<double>> acc;
  acc.reserve((size_t)T.n_loops * 24);
  // coefficient w0 (and w1 >= 0) of Q_ij += M_i,bi M_j,bj u0 (u1) for every loop i through bi
  // and j through bj
  auto scatter = [&](int bi, int bj, int w0, double u0, int w1, double u1) {
    for (int64_t ki = T.mt_ptr[bi]; ki < T.mt_ptr[bi + 1]; ++ki)
      for (int64_t kj = T.mt_ptr[bj]; kj < T.mt_ptr[bj + 1]; ++kj) {
        uint64_t key = ((uint64_t)(uint32_t)T.mt_col[ki] << 32) | (uint32_t)T.mt_col[kj];
        const double m = T.mt_val[ki] * T.mt_val[kj];
        auto& v = acc[key];
        if (v.empty()) v.assign(W, 0.0);
        v[w0] += m * u0;
        if (w1 >= 0) v[w1] += m * u1;
      }
  };
  // branches of each live panel with their signed rho
  std::vector<std::vector<std::pair<int, int>>> pb(N);   // (branch, side)
  for (int b = 0; b < T.n_cb; ++b)
    for (int s = 0; s < 2; ++s)
      if (T.br_pan[s][b] >= 0) pb[T.br_pan[s][b]].push_back({b, s});
  for (int p = 0; p < N; ++p) {
    if (T.live_of_panel[p] < 0) continue;
    const double area = panel_area_host(c->xyz, c->pan, p);
    const int mat = T.mat_of_cond[c->cond[p]];
    for (auto& bi : pb[p])
      for (auto& bj : pb[p]) {
        double dot = dot3(&T.br_rho[bi.second][3 * (size_t)bi.first], &T.br_rho[bj.second][3 * (size_t)bj.first]);
        scatter(bi.first, bj.first, mat, dot / area, p12 ? -1 : nm, dot * pdiag[p]);
      }
  }
  if (p12) {
    XRL_CHECK((int)p12->size() == T.n_cb, XRL_EINVAL, "one P entry per conductor branch");
    for (int b = 0; b < T.n_cb; ++b) {
      double g = 0.0;
      for (int s = 0; s < 2; ++s) {
        const int p = T.br_pan[s][b];
        if (p < 0) continue;
        const double* r = &T.br_rho[s][3 * (size_t)b];
        g += dot3(r, r) * pdiag[p];
      }
      if (T.br_pan[0][b] >= 0 && T.br_pan[1][b] >= 0)
        g += 2.0 * dot3(&T.br_rho[0][3 * (size_t)b], &T.br_rho[1][3 * (size_t)b]) * (*p12)[b];
      scatter(b, b, nm, g, -1, 0.0);
    }
  }
  std::vector<std::pair<uint64_t, const std::vector<double>*>> ent;
  ent.reserve(acc.size());
  for (auto& kv : acc) ent.push_back({kv.first, &kv.second});
  std::sort(ent.begin(), ent.end(), [](auto& a, auto& b) { return a.first < b.first; });
  T.q_ptr.assign(T.n_loops + 1, 0);
  T.q_col.resize(ent.size());
  T.q_val.resize(ent.size() * W);
  for (size_t k = 0; k < ent.size(); ++k) {
    int r = (int)(ent[k].first >> 32);
    T.q_ptr[r + 1]++;
    T.q_col[k] = (int32_t)(ent[k].first & 0xffffffffu);
    for (int w = 0; w < W; ++w) T.q_val[k * W + w] = (*ent[k].second)[w];
  }
  for (int r = 0; r < T.n_loops; ++r) T.q_ptr[r + 1] += T.q_ptr[r];
}

}  // namespace xrl

namespace xrl {

// Reverse Cuthill-McKee order of the vertex-loop block of Q (the paper
// applies Q^-1 with a sparse LU, Sec. II-D; a vertex loop couples only to
// the loops of neighbouring vertices, so after RCM the block is banded),
// then the band and border values of every pencil member.
void build_band(xrl_ctx* c) {
  Topo& T = c->topo;
  const int nv = T.n_vertex_loops;
  const int ng = T.n_loops - nv;
  const int W = T.n_mat + 1;
  T.n_band = nv;
  T.n_border = ng;
  // adjacency among vertex loops
  std::vector<std::vector<int>> adj(nv);
  for (int r = 0; r < nv; ++r)
    for (int64_t k = T.q_ptr[r]; k < T.q_ptr[r + 1]; ++k) {
      int cidx = T.q_col[k];
      if (cidx != r && cidx < nv) adj[r].push_back(cidx);
    }
  for (auto& a : adj) std::sort(a.begin(), a.end());
  std::vector<int> order;
  order.reserve(nv);
  std::vector<char> seen(nv, 0);
  std::vector<int> deg(nv);
  for (int i = 0; i < nv; ++i) deg[i] = (int)adj[i].size();
  auto bfs_last = [&](int s, std::vector<int>& lvl) {
    lvl.assign(nv, -1);
    std::deque<int> dq{s};
    lvl[s] = 0;
    int last = s;
    while (!dq.empty()) {
      int u = dq.front();
      dq.pop_front();
      last = u;
      for (int v : adj[u])
        if (lvl[v] < 0) {
          lvl[v] = lvl[u] + 1;
          dq.push_back(v);
        }
    }
    return last;
  };
  std::vector<int> lvl;
  for (int start = 0; start < nv; ++start) {
    if (seen[start]) continue;
    // pseudo-peripheral node of this component: a few BFS sweeps from the minimum degree node
    int s = start;
    {
      std::vector<int> l0;
      bfs_last(start, l0);
      for (int i = 0; i < nv; ++i)
        if (l0[i] >= 0 && deg[i] < deg[s]) s = i;
      for (int it = 0; it < 3; ++it) s = bfs_last(s, lvl);
    }
    std::deque<int> dq{s};
    seen[s] = 1;
    while (!dq.empty()) {
      int u = dq.front();
      dq.pop_front();
      order.push_back(u);
      std::vector<int> nb;
      for (int v : adj[u])
        if (!seen[v]) {
          seen[v] = 1;
          nb.push_back(v);
        }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
      for (int v : nb) dq.push_back(v);
    }
  }
  std::reverse(order.begin(), order.end());
  T.band_perm = order;
  std::vector<int> pos(nv);
  for (int i = 0; i < nv; ++i) pos[order[i]] = i;
  int b = 0;
  for (int r = 0; r < nv; ++r)
    for (int64_t k = T.q_ptr[r]; k < T.q_ptr[r + 1]; ++k) {
      int cidx = T.q_col[k];
      if (cidx < nv) b = std::max(b, std::abs(pos[r] - pos[cidx]));
    }
  T.band = b;
  T.band_val.clear();
  T.border_vg.clear();
  T.border_gg.clear();
  // a band or border too wide for the banded solver is never factorised (the
  // multigrid takes Q instead): its values, W nv (b + 1) + W nv ng doubles,
  // would only take memory (tens of GB on the package stacks)
  if (!band_fits(b, ng)) return;
  T.band_val.assign((size_t)W * nv * (b + 1), 0.0);
  T.border_vg.assign((size_t)W * nv * ng, 0.0);
  T.border_gg.assign((size_t)W * ng * ng, 0.0);
  for (int r = 0; r < T.n_loops; ++r)
    for (int64_t k = T.q_ptr[r]; k < T.q_ptr[r + 1]; ++k) {
      int cidx = T.q_col[k];
      for (int w = 0; w < W; ++w) {
        double v = T.q_val[(size_t)k * W + w];
        if (r < nv && cidx < nv) {
          int i = pos[r], j = pos[cidx];
          if (j <= i) T.band_val[((size_t)w * nv + i) * (b + 1) + (j - i + b)] = v;
        } else if (r < nv && cidx >= nv) {
          T.border_vg[((size_t)w * nv + pos[r]) * ng + (cidx - nv)] = v;
        } else if (r >= nv && cidx >= nv) {
          T.border_gg[((size_t)w * ng + (r - nv)) * ng + (cidx - nv)] = v;
        }
      }
    }
}

}  // namespace xrl
