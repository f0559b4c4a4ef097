// Panel geometry, Morton keys, the near-field rule table, the P2M/L2P moment
// table and the FP64 direct-sum reference product (sm_103a).
//
// P_kl = (1/(A_k A_l)) int_k int_l 1/|r - r'| dS' dS is the panel potential
// kernel of eq. 6 (Sec. II-A) under the centroid-midpoint normalisation.  The
// paper fills the near-field matrix "on panels" (Sec. II-C) without naming
// a quadrature; entries here follow a fixed rule table (class boundaries in
// q = |c_k - c_l| / (r_k + r_l), r = max centroid-vertex distance), always
// evaluated on the ordered pair (lo, hi) of CALLER panel indices so that P is
// exactly symmetric:
//   k == l         closed form (4/3) sum_sides (1/a) ln(s / (s - 2a))
//   shared edge    mean of both one-sided semi-analytic integrals, outer
//                  rule: Duffy map graded (u = 1 - (1-xi)^3) to the shared edge
//   shared vertex  same, Duffy map graded (u = xi^3) to the shared vertex
//   q < 1.5        outer collapsed Gauss 8x8 on lo, analytic potential of hi
//   1.5 <= q < 3   outer collapsed Gauss 5x5 on lo
//   3 <= q < 10    point product rule 4x4 x 4x4
//   q >= 10        point product rule 3x3 x 3x3
// The analytic potential of a uniformly charged flat triangle is the closed
// form of Wilton et al. (1984) / Graglia (1993).
#include <algorithm>
#include <cmath>
#include <vector>

#include "xrl_internal.hpp"

namespace xrl {

// ---- rule tables in constant memory -----------------------------------------------
// Layout: per rule, points as (c0, c1, c2, w): p = c0 v0 + c1 v1 + c2 v2, weights sum to 1.
constexpr int kR3 = 0, kR4 = kR3 + 9, kR5 = kR4 + 16, kR8 = kR5 + 25, kRE = kR8 + 64,
              kRV = kRE + 100, kRtot = kRV + 100;
__constant__ double c_rule[kRtot * 4];

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double nrm(V3 a) { return sqrt(dot(a, a)); }

// int_T 1/|x - r'| dS' for the flat triangle (v0, v1, v2)
__device__ double tri_potential(V3 x, V3 v0, V3 v1, V3 v2) {
  V3 n = cross(sub(v1, v0), sub(v2, v0));
  double nn = nrm(n);
  n = {n.x / nn, n.y / nn, n.z / nn};
  double w0 = dot(sub(x, v0), n);
  double aw = fabs(w0);
  V3 rho = {x.x - w0 * n.x, x.y - w0 * n.y, x.z - w0 * n.z};
  V3 vs[3] = {v0, v1, v2};
  double tot = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    V3 a = vs[i], b = vs[(i + 1) % 3];
    V3 L = sub(b, a);
    double le = nrm(L);
    V3 lh = {L.x / le, L.y / le, L.z / le};
    V3 u = cross(lh, n);
    V3 ar = sub(a, rho), br = sub(b, rho);
    double P0 = dot(ar, u);
    double lm = dot(ar, lh), lp = dot(br, lh);
    double Rm = nrm(sub(a, x)), Rp = nrm(sub(b, x));
    double R0s = P0 * P0 + w0 * w0;
    if (P0 != 0.0) {
      double lnp = lp >= 0.0 ? log(Rp + lp) : log(R0s / (Rp - lp));
      double lnm = lm >= 0.0 ? log(Rm + lm) : log(R0s / (Rm - lm));
      tot += P0 * (lnp - lnm);
    }
    if (aw > 0.0) {
      double beta = atan(P0 * lp / (R0s + aw * Rp)) - atan(P0 * lm / (R0s + aw * Rm));
      tot -= aw * beta;
    }
  }
  return tot;
}

__device__ double self_term(V3 v0, V3 v1, V3 v2) {
  double a = nrm(sub(v1, v2)), b = nrm(sub(v2, v0)), c = nrm(sub(v0, v1));
  double s = a + b + c;
  return (4.0 / 3.0) * (log(s / (s - 2.0 * a)) / a + log(s / (s - 2.0 * b)) / b + log(s / (s - 2.0 * c)) / c);
}

__device__ __forceinline__ V3 ld3(const double* p) { return {p[0], p[1], p[2]}; }

// outer rule on (o0, o1, o2) (already arranged), inner analytic on triangle I; / area_I
__device__ double semi(int r0, int nq, V3 o0, V3 o1, V3 o2, V3 i0, V3 i1, V3 i2, double areaI) {
  double acc = 0.0;
  for (int q = 0; q < nq; ++q) {
    const double* r = &c_rule[(r0 + q) * 4];
    V3 x = {r[0] * o0.x + r[1] * o1.x + r[2] * o2.x, r[0] * o0.y + r[1] * o1.y + r[2] * o2.y,
            r[0] * o0.z + r[1] * o1.z + r[2] * o2.z};
    acc += r[3] * tri_potential(x, i0, i1, i2);
  }
  return acc / areaI;
}

__device__ double product(int r0, int nq, V3 a0, V3 a1, V3 a2, V3 b0, V3 b1, V3 b2) {
  double acc = 0.0;
  for (int i = 0; i < nq; ++i) {
    const double* ri = &c_rule[(r0 + i) * 4];
    V3 x = {ri[0] * a0.x + ri[1] * a1.x + ri[2] * a2.x, ri[0] * a0.y + ri[1] * a1.y + ri[2] * a2.y,
            ri[0] * a0.z + ri[1] * a1.z + ri[2] * a2.z};
    double s = 0.0;
    for (int j = 0; j < nq; ++j) {
      const double* rj = &c_rule[(r0 + j) * 4];
      V3 y = {rj[0] * b0.x + rj[1] * b1.x + rj[2] * b2.x, rj[0] * b0.y + rj[1] * b1.y + rj[2] * b2.y,
              rj[0] * b0.z + rj[1] * b1.z + rj[2] * b2.z};
      s += rj[3] / nrm(sub(x, y));
    }
    acc += ri[3] * s;
  }
  return acc;
}

struct PanelView {
  const double* vtx;     // [N][12] (a triangle's 4th vertex unused)
  const double* cen;     // [N][3]
  const double* area;
  const double* radius;
  const int32_t* tri;    // [N][4], -1 in slot 3 for a triangle
  const int32_t* cidx;   // [N]
};

// One triangle of the rule table: a triangle panel itself, or half s of a
// rectangle (v0, v1, v2) / (v0, v2, v3), with its own area, centroid and radius.
struct SubTri {
  V3 v[3];
  int32_t id[3];
  double area, r;
  V3 c;
};

__device__ __forceinline__ int n_sub(const PanelView& pv, int k) { return pv.tri[4 * (size_t)k + 3] >= 0 ? 2 : 1; }

__device__ SubTri sub_tri(const PanelView& pv, int k, int s) {
  const double* v = pv.vtx + 12 * (size_t)k;
  const int32_t* t = pv.tri + 4 * (size_t)k;
  const int i1 = s == 0 ? 1 : 2, i2 = s == 0 ? 2 : 3;
  SubTri st;
  st.v[0] = ld3(v);
  st.v[1] = ld3(v + 3 * i1);
  st.v[2] = ld3(v + 3 * i2);
  st.id[0] = t[0];
  st.id[1] = t[i1];
  st.id[2] = t[i2];
  if (t[3] < 0) {
    st.area = pv.area[k];
    st.c = ld3(pv.cen + 3 * (size_t)k);
    st.r = pv.radius[k];
  } else {
    st.c = {__ddiv_rn(__dadd_rn(__dadd_rn(st.v[0].x, st.v[1].x), st.v[2].x), 3.0),
            __ddiv_rn(__dadd_rn(__dadd_rn(st.v[0].y, st.v[1].y), st.v[2].y), 3.0),
            __ddiv_rn(__dadd_rn(__dadd_rn(st.v[0].z, st.v[1].z), st.v[2].z), 3.0)};
    st.area = 0.5 * nrm(cross(sub(st.v[1], st.v[0]), sub(st.v[2], st.v[0])));
    st.r = fmax(fmax(nrm(sub(st.v[0], st.c)), nrm(sub(st.v[1], st.c))), nrm(sub(st.v[2], st.c)));
  }
  return st;
}

// rule-table entry of two distinct triangles, A the lower one in the caller order
__device__ double p_tri(const SubTri& A, const SubTri& B) {
  bool sa[3], sb[3];
  int ns = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sa[i] = (A.id[i] == B.id[0]) || (A.id[i] == B.id[1]) || (A.id[i] == B.id[2]);
    sb[i] = (B.id[i] == A.id[0]) || (B.id[i] == A.id[1]) || (B.id[i] == A.id[2]);
    ns += sa[i] ? 1 : 0;
  }
  if (ns >= 1) {
    bool edge = (ns == 2);
    // edge rule: start at the non-shared vertex; vertex rule: at the shared vertex
    int fa = 0, fb = 0;
#pragma unroll
    for (int i = 2; i >= 0; --i) {
      if (edge ? !sa[i] : sa[i]) fa = i;
      if (edge ? !sb[i] : sb[i]) fb = i;
    }
    int r0 = edge ? kRE : kRV;
    double s1 = semi(r0, 100, A.v[fa], A.v[(fa + 1) % 3], A.v[(fa + 2) % 3], B.v[0], B.v[1], B.v[2], B.area);
    double s2 = semi(r0, 100, B.v[fb], B.v[(fb + 1) % 3], B.v[(fb + 2) % 3], A.v[0], A.v[1], A.v[2], A.area);
    return (s1 + s2) * 0.5;
  }
  double dx = __dsub_rn(A.c.x, B.c.x), dy = __dsub_rn(A.c.y, B.c.y), dz = __dsub_rn(A.c.z, B.c.z);
  double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  double q = __ddiv_rn(d, __dadd_rn(A.r, B.r));
  if (q < kQNear) return semi(kR8, 64, A.v[0], A.v[1], A.v[2], B.v[0], B.v[1], B.v[2], B.area);
  if (q < kQSemi) return semi(kR5, 25, A.v[0], A.v[1], A.v[2], B.v[0], B.v[1], B.v[2], B.area);
  if (q < kQFar) return product(kR4, 16, A.v[0], A.v[1], A.v[2], B.v[0], B.v[1], B.v[2]);
  return product(kR3, 9, A.v[0], A.v[1], A.v[2], B.v[0], B.v[1], B.v[2]);
}

// P entry for Morton ranks k, l.  A rectangle's entries are the area-weighted
// sums over its two triangles, P_kl = sum_i sum_j (a_i/A_k)(a_j/A_l) P_ij.
__device__ double p_entry(const PanelView& pv, int k, int l) {
  if (k == l) {
    if (n_sub(pv, k) == 1) {
      const double* v = pv.vtx + 12 * (size_t)k;
      return self_term(ld3(v), ld3(v + 3), ld3(v + 6));
    }
    const SubTri s0 = sub_tri(pv, k, 0), s1 = sub_tri(pv, k, 1);
    const double w0 = s0.area / pv.area[k], w1 = s1.area / pv.area[k];
    return w0 * w0 * self_term(s0.v[0], s0.v[1], s0.v[2]) + 2.0 * w0 * w1 * p_tri(s0, s1) +
           w1 * w1 * self_term(s1.v[0], s1.v[1], s1.v[2]);
  }
  int a = k, b = l;
  if (pv.cidx[k] > pv.cidx[l]) {
    a = l;
    b = k;
  }
  const int na = n_sub(pv, a), nb = n_sub(pv, b);
  if (na == 1 && nb == 1) return p_tri(sub_tri(pv, a, 0), sub_tri(pv, b, 0));
  double acc = 0.0;
  for (int i = 0; i < na; ++i) {
    const SubTri A = sub_tri(pv, a, i);
    const double wa = A.area / pv.area[a];
    for (int j = 0; j < nb; ++j) {
      const SubTri B = sub_tri(pv, b, j);
      acc += wa * (B.area / pv.area[b]) * p_tri(A, B);
    }
  }
  return acc;
}

// ---- kernels -------------------------------------------------------------------------
__global__ void k_geometry(int N, const double* __restrict__ xyz, const int32_t* __restrict__ pan,
                           double* __restrict__ cen, double* __restrict__ area, double* __restrict__ radius) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int32_t* t = pan + 4 * (size_t)p;
  const int nv = t[3] >= 0 ? 4 : 3;
  const double* vs[4];
  for (int i = 0; i < nv; ++i) vs[i] = xyz + 3 * (size_t)t[i];
  // vertex mean, FMA-free: ((v0 + v1) + v2) / 3, or (((v0 + v1) + v2) + v3) / 4
  double c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double s3 = __dadd_rn(__dadd_rn(vs[0][k], vs[1][k]), vs[2][k]);
    c[k] = nv == 4 ? __ddiv_rn(__dadd_rn(s3, vs[3][k]), 4.0) : __ddiv_rn(s3, 3.0);
  }
  V3 e1 = {vs[1][0] - vs[0][0], vs[1][1] - vs[0][1], vs[1][2] - vs[0][2]};
  V3 e2 = {vs[2][0] - vs[0][0], vs[2][1] - vs[0][1], vs[2][2] - vs[0][2]};
  double ar = 0.5 * nrm(cross(e1, e2));
  if (nv == 4) {
    V3 e3 = {vs[3][0] - vs[0][0], vs[3][1] - vs[0][1], vs[3][2] - vs[0][2]};
    ar += 0.5 * nrm(cross(e2, e3));
  }
  area[p] = ar;
  double r = 0.0;
  for (int i = 0; i < nv; ++i) {
    V3 d = {vs[i][0] - c[0], vs[i][1] - c[1], vs[i][2] - c[2]};
    r = fmax(r, nrm(d));
  }
  radius[p] = r;
  for (int k = 0; k < 3; ++k) cen[3 * (size_t)p + k] = c[k];
}

// one block: lo[3], side = max extent * (1 + 2^-20)
__global__ void k_bounds(int N, const double* __restrict__ cen, double* __restrict__ box) {
  __shared__ double smin[3][256], smax[3][256];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int p = threadIdx.x; p < N; p += blockDim.x)
    for (int k = 0; k < 3; ++k) {
      double v = cen[3 * (size_t)p + k];
      mn[k] = fmin(mn[k], v);
      mx[k] = fmax(mx[k], v);
    }
  for (int k = 0; k < 3; ++k) {
    smin[k][threadIdx.x] = mn[k];
    smax[k][threadIdx.x] = mx[k];
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) {
        smin[k][threadIdx.x] = fmin(smin[k][threadIdx.x], smin[k][threadIdx.x + s]);
        smax[k][threadIdx.x] = fmax(smax[k][threadIdx.x], smax[k][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) {
      box[k] = smin[k][0];
      ext = fmax(ext, __dsub_rn(smax[k][0], smin[k][0]));
    }
    box[3] = __dmul_rn(ext, 1.0 + 0x1p-20);
  }
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

__global__ void k_keys(int N, const double* __restrict__ cen, const double* __restrict__ box,
                       uint64_t* __restrict__ keys) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t q[3];
  for (int k = 0; k < 3; ++k) {
    double t = __dmul_rn(__ddiv_rn(__dsub_rn(cen[3 * (size_t)p + k], box[k]), box[3]), 2097152.0);
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    q[k] = (uint32_t)f;
  }
  keys[p] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
}

__global__ void k_gather_panels(int N, const int32_t* __restrict__ perm, const double* __restrict__ xyz,
                                const int32_t* __restrict__ tri_in, const double* __restrict__ cen_in,
                                const double* __restrict__ area_in, const double* __restrict__ rad_in,
                                double* vtx, double* cen, double* area, double* radius, int32_t* tri, int32_t* cidx) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int p = perm[r];
  for (int v = 0; v < 4; ++v) {
    int id = tri_in[4 * (size_t)p + v];
    tri[4 * (size_t)r + v] = id;
    for (int k = 0; k < 3; ++k) vtx[12 * (size_t)r + 3 * v + k] = id >= 0 ? xyz[3 * (size_t)id + k] : 0.0;
  }
  for (int k = 0; k < 3; ++k) cen[3 * (size_t)r + k] = cen_in[3 * (size_t)p + k];
  area[r] = area_in[p];
  radius[r] = rad_in[p];
  cidx[r] = p;
}

// Near-field fill in three passes, so that the threads of a warp evaluate
// entries of one class of the rule table (its classes differ in cost by two
// orders of magnitude; mixed in one warp, every warp paid for the dearest):
//  1. k_near_count: per leaf, the number of its entries in each class;
//  2. k_near_list: the entries (value position, target, source) in lists
//     ordered by class, then leaf (within a leaf in any order);
//  3. k_near_eval: every listed entry by p_entry, the same function as before,
//     so the values do not depend on the grouping.
// Classes: 0 self, 1 triangles sharing a vertex, 2 q < kQNear, 3 q < kQSemi,
// 4 q < kQFar, 5 far, 6 a rectangle involved (general path).
constexpr int kNearClasses = 7;

__device__ int near_class(const PanelView& pv, int k, int j) {
  if (k == j) return 0;
  if (n_sub(pv, k) > 1 || n_sub(pv, j) > 1) return 6;
  const int32_t* tk = pv.tri + 4 * (size_t)k;
  const int32_t* tj = pv.tri + 4 * (size_t)j;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (tk[a] == tj[b]) return 1;
  const double* ck = pv.cen + 3 * (size_t)k;
  const double* cj = pv.cen + 3 * (size_t)j;
  const double dx = __dsub_rn(ck[0], cj[0]), dy = __dsub_rn(ck[1], cj[1]), dz = __dsub_rn(ck[2], cj[2]);
  const double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  const double q = __ddiv_rn(d, __dadd_rn(pv.radius[k], pv.radius[j]));
  return q < kQNear ? 2 : q < kQSemi ? 3 : q < kQFar ? 4 : 5;
}

// one block per leaf: its entries, U-list source by U-list source
__global__ void k_near_count(PanelView pv, const int32_t* __restrict__ leaf_first, const int32_t* __restrict__ leaf_count,
                             const int32_t* __restrict__ u_ptr, const int32_t* __restrict__ u_src,
                             int32_t* __restrict__ cnt) {
  __shared__ int sc[kNearClasses];
  const int B = blockIdx.x;
  if (threadIdx.x < kNearClasses) sc[threadIdx.x] = 0;
  __syncthreads();
  const int nB = leaf_count[B], f0 = leaf_first[B];
  for (int s = u_ptr[B]; s < u_ptr[B + 1]; ++s) {
    const int S = u_src[s], nS = leaf_count[S], fS = leaf_first[S];
    for (int e = threadIdx.x; e < nB * nS; e += blockDim.x)
      atomicAdd(&sc[near_class(pv, f0 + e / nS, fS + e % nS)], 1);
  }
  __syncthreads();
  if (threadIdx.x < kNearClasses) cnt[(size_t)B * kNearClasses + threadIdx.x] = sc[threadIdx.x];
}

__global__ void k_near_list(PanelView pv, const int32_t* __restrict__ leaf_first, const int32_t* __restrict__ leaf_count,
                            const int32_t* __restrict__ u_ptr, const int32_t* __restrict__ u_src,
                            const int64_t* __restrict__ near_off, const int32_t* __restrict__ near_w,
                            const int64_t* __restrict__ base, int64_t* __restrict__ lpos, int32_t* __restrict__ lk,
                            int32_t* __restrict__ lj) {
  __shared__ unsigned long long slot[kNearClasses];
  const int B = blockIdx.x;
  if (threadIdx.x < kNearClasses) slot[threadIdx.x] = (unsigned long long)base[(size_t)B * kNearClasses + threadIdx.x];
  __syncthreads();
  const int nB = leaf_count[B], f0 = leaf_first[B], w = near_w[B];
  const int64_t off = near_off[B];
  int col = 0;
  for (int s = u_ptr[B]; s < u_ptr[B + 1]; ++s) {
    const int S = u_src[s], nS = leaf_count[S], fS = leaf_first[S];
    for (int e = threadIdx.x; e < nB * nS; e += blockDim.x) {
      const int ii = e / nS, jl = e % nS;
      const int k = f0 + ii, j = fS + jl;
      const unsigned long long i = atomicAdd(&slot[near_class(pv, k, j)], 1ull);
      lpos[i] = off + (int64_t)ii * w + col + jl;
      lk[i] = k;
      lj[i] = j;
    }
    col += nS;
  }
}

__global__ void k_near_eval(PanelView pv, int64_t n, const int64_t* __restrict__ lpos, const int32_t* __restrict__ lk,
                            const int32_t* __restrict__ lj, double* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) val[lpos[i]] = p_entry(pv, lk[i], lj[i]);
}

// FP64 direct sum with the rule table: one block per target, Morton rank
// k = rows[blockIdx.x] (rows = NULL: k = blockIdx.x), output row blockIdx.x
__global__ void k_direct(PanelView pv, int N, int nc, const int32_t* __restrict__ rows, const double* __restrict__ X,
                         double* __restrict__ Y) {
  const int k = rows ? rows[blockIdx.x] : (int)blockIdx.x;
  const int ko = blockIdx.x;
  extern __shared__ double red[];
  double acc[8];
  for (int c0 = 0; c0 < nc; c0 += 8) {
    int cn = min(8, nc - c0);
    for (int c = 0; c < 8; ++c) acc[c] = 0.0;
    for (int l = threadIdx.x; l < N; l += blockDim.x) {
      double pkl = p_entry(pv, k, l);
      for (int c = 0; c < cn; ++c) acc[c] += pkl * X[(size_t)l * nc + c0 + c];
    }
    for (int c = 0; c < cn; ++c) {
      red[threadIdx.x] = acc[c];
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
      }
      if (threadIdx.x == 0) Y[(size_t)ko * nc + c0 + c] = red[0];
      __syncthreads();
    }
  }
}

// moments S[i][(n,m,re/im)] = (1/A) int_i conj(Y_n^m((y - c_leaf)/h)) dS (exact with the rule)
// (a rectangle integrates its two triangles, each weighted by its share of the area)
__global__ void k_moments(int N, int p, const double* __restrict__ vtx, const int32_t* __restrict__ tri,
                          const double* __restrict__ area, const int32_t* __restrict__ leaf_of,
                          const double* __restrict__ leaf_ctr, double inv_h, const double* __restrict__ rule,
                          int nq, double* __restrict__ S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nc = (p + 1) * (p + 1);
  double acc[169];
  double yr[13][13], yi[13][13];
  for (int k = 0; k < nc; ++k) acc[k] = 0.0;
  const double* pv = vtx + 12 * (size_t)i;
  const double* c = leaf_ctr + 3 * (size_t)leaf_of[i];
  const int nsub = tri[4 * (size_t)i + 3] >= 0 ? 2 : 1;
  for (int q = 0; q < nq * nsub; ++q) {
    const int s = q / nq;
    const double* r = rule + 4 * (q - s * nq);
    const double* v0 = pv;
    const double* v1 = pv + 3 * (1 + s);
    const double* v2 = pv + 3 * (2 + s);
    double ws = 1.0;
    if (nsub == 2) {
      V3 e1 = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]}, e2 = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
      ws = 0.5 * nrm(cross(e1, e2)) / area[i];
    }
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = ((r[0] * v0[k] + r[1] * v1[k] + r[2] * v2[k]) - c[k]) * inv_h;
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    // regular harmonics, m >= 0 (Condon-Shortley phase): Y_m^m = -(x+iy)/(2m) Y_{m-1}^{m-1}
    yr[0][0] = 1.0;
    yi[0][0] = 0.0;
    for (int m = 0; m <= p; ++m) {
      if (m > 0) {
        double a = yr[m - 1][m - 1], b = yi[m - 1][m - 1];
        yr[m][m] = -(x[0] * a - x[1] * b) / (2.0 * m);
        yi[m][m] = -(x[0] * b + x[1] * a) / (2.0 * m);
      }
      for (int n = m + 1; n <= p; ++n) {
        double p2r = (n - 2 >= m) ? yr[n - 2][m] : 0.0, p2i = (n - 2 >= m) ? yi[n - 2][m] : 0.0;
        double den = (double)((n + m) * (n - m));
        yr[n][m] = ((2.0 * n - 1.0) * x[2] * yr[n - 1][m] - r2 * p2r) / den;
        yi[n][m] = ((2.0 * n - 1.0) * x[2] * yi[n - 1][m] - r2 * p2i) / den;
      }
    }
    double w = r[3] * ws;
    for (int n = 0; n <= p; ++n) {
      acc[n * n] += w * yr[n][0];
      for (int m = 1; m <= n; ++m) {
        acc[n * n + 2 * m - 1] += w * yr[n][m];
        acc[n * n + 2 * m] -= w * yi[n][m];   // conjugate
      }
    }
  }
  for (int k = 0; k < nc; ++k) S[(size_t)i * nc + k] = acc[k];
}

// ---- host wrappers -------------------------------------------------------------------

static void collapsed_rule(int q, std::vector<double>& out) {
  std::vector<double> x, w;
  gauss_legendre01(q, x, w);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double s = x[i], t = x[j];
      double c1 = s, c2 = t * (1.0 - s), c0 = 1.0 - c1 - c2;
      out.insert(out.end(), {c0, c1, c2, 2.0 * w[i] * w[j] * (1.0 - s)});
    }
}

static void graded_rule(int n, int k, bool edge, std::vector<double>& out) {
  std::vector<double> x, w;
  gauss_legendre01(n, x, w);
  for (int i = 0; i < n; ++i) {
    double u, du;
    if (edge) {
      u = 1.0 - std::pow(1.0 - x[i], k);
      du = k * std::pow(1.0 - x[i], k - 1) * w[i];
    } else {
      u = std::pow(x[i], k);
      du = k * std::pow(x[i], k - 1) * w[i];
    }
    for (int j = 0; j < n; ++j) {
      double t = x[j];
      out.insert(out.end(), {1.0 - u, u * (1.0 - t), u * t, 2.0 * u * du * w[j]});
    }
  }
}

void upload_rule_tables(xrl_ctx* c) {
  std::vector<double> r;
  collapsed_rule(kFarQ, r);
  collapsed_rule(kMidQ, r);
  collapsed_rule(kSemiQ, r);
  collapsed_rule(kNearQ, r);
  graded_rule(kEdgeN, kEdgeK, true, r);
  graded_rule(kVertN, kVertK, false, r);
  XRL_CHECK((int)r.size() == kRtot * 4, XRL_EINVAL, "rule table size");
  XRL_CUDA(cudaMemcpyToSymbol(c_rule, r.data(), r.size() * sizeof(double)));
  c->gl_nodes = r;
}

static PanelView view(const xrl_ctx* c) {
  return {c->d.vtx.p, c->d.cen.p, c->d.area.p, c->d.radius.p, c->d.tri.p, c->d.cidx.p};
}

void launch_geometry(xrl_ctx* c) {
  const int N = c->N;
  DBuf<double> xyz;
  xyz.upload(c->alloc, c->xyz);
  DBuf<int32_t> tri;
  tri.upload(c->alloc, c->pan);
  DBuf<double> cen0, area0, rad0, box;
  cen0.alloc(c->alloc, 3 * (size_t)N);
  area0.alloc(c->alloc, N);
  rad0.alloc(c->alloc, N);
  box.alloc(c->alloc, 4);
  c->d.keys.alloc(c->alloc, N);
  int nb = (N + 255) / 256;
  k_geometry<<<nb, 256, 0, c->stream>>>(N, xyz.p, tri.p, cen0.p, area0.p, rad0.p);
  k_bounds<<<1, 256, 0, c->stream>>>(N, cen0.p, box.p);
  k_keys<<<nb, 256, 0, c->stream>>>(N, cen0.p, box.p, c->d.keys.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<uint64_t> keys = c->d.keys.download();
  std::vector<double> hbox = box.download();
  for (int k = 0; k < 3; ++k) c->tree.lo[k] = hbox[k];
  c->tree.side = hbox[3];
  build_tree(c, keys);
  c->d.perm.upload(c->alloc, c->tree.perm);
  c->d.vtx.alloc(c->alloc, 12 * (size_t)N);
  c->d.cen.alloc(c->alloc, 3 * (size_t)N);
  c->d.area.alloc(c->alloc, N);
  c->d.radius.alloc(c->alloc, N);
  c->d.tri.alloc(c->alloc, 4 * (size_t)N);
  c->d.cidx.alloc(c->alloc, N);
  k_gather_panels<<<nb, 256, 0, c->stream>>>(N, c->d.perm.p, xyz.p, tri.p, cen0.p, area0.p, rad0.p, c->d.vtx.p,
                                             c->d.cen.p, c->d.area.p, c->d.radius.p, c->d.tri.p, c->d.cidx.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(c->stream));
}

void launch_near_fill(xrl_ctx* c) {
  const Tree& t = c->tree;
  const int nl = t.n_leaves();
  std::vector<int64_t> off(nl + 1, 0);
  std::vector<int32_t> w(nl, 0);
  for (int i = 0; i < nl; ++i) {
    int width = 0;
    for (int64_t s = t.u_ptr[i]; s < t.u_ptr[i + 1]; ++s) width += t.leaf_count[t.u_src[s]];
    w[i] = width;
    off[i + 1] = off[i] + (int64_t)width * t.leaf_count[i];
  }
  c->stats.near_nnz = off[nl];
  // Morton index of every near column of every leaf (for the tiled P2P)
  std::vector<int64_t> coff(nl + 1, 0);
  std::vector<int32_t> nsrc;
  for (int i = 0; i < nl; ++i) {
    for (int64_t s = t.u_ptr[i]; s < t.u_ptr[i + 1]; ++s) {
      int S = t.u_src[s];
      for (int q = 0; q < t.leaf_count[S]; ++q) nsrc.push_back(t.leaf_first[S] + q);
    }
    coff[i + 1] = (int64_t)nsrc.size();
  }
  c->d.near_col_off.upload(c->alloc, coff);
  c->max_leaf = 0;
  for (int i = 0; i < nl; ++i) c->max_leaf = std::max(c->max_leaf, t.leaf_count[i]);
  c->d.near_src.upload(c->alloc, nsrc);
  std::vector<int32_t> uptr32(t.u_ptr.begin(), t.u_ptr.end());
  c->d.leaf_first.upload(c->alloc, t.leaf_first);
  c->d.leaf_count.upload(c->alloc, t.leaf_count);
  c->d.u_ptr32.upload(c->alloc, uptr32);
  c->d.u_src.upload(c->alloc, t.u_src);
  off.pop_back();
  c->d.near_off.upload(c->alloc, off);
  c->d.near_w.upload(c->alloc, w);
  const int64_t nnz = c->stats.near_nnz;
  c->d.near_val.alloc(c->alloc, (size_t)nnz);
  if (nnz == 0) return;
  DBuf<int32_t> cnt;
  cnt.alloc(c->alloc, (size_t)nl * kNearClasses);
  k_near_count<<<nl, 256, 0, c->stream>>>(view(c), c->d.leaf_first.p, c->d.leaf_count.p, c->d.u_ptr32.p,
                                           c->d.u_src.p, cnt.p);
  XRL_CUDA(cudaGetLastError());
  const std::vector<int32_t> hc = cnt.download();
  // list start of (leaf, class): classes in order, leaves in order within a class
  std::vector<int64_t> base((size_t)nl * kNearClasses);
  int64_t run = 0;
  for (int k = 0; k < kNearClasses; ++k)
    for (int i = 0; i < nl; ++i) {
      base[(size_t)i * kNearClasses + k] = run;
      run += hc[(size_t)i * kNearClasses + k];
    }
  XRL_CHECK(run == nnz, XRL_EINVAL, "internal: near-field class counts do not add up");
  DBuf<int64_t> dbase, lpos;
  DBuf<int32_t> lk, lj;
  dbase.upload(c->alloc, base);
  lpos.alloc(c->alloc, (size_t)nnz);
  lk.alloc(c->alloc, (size_t)nnz);
  lj.alloc(c->alloc, (size_t)nnz);
  k_near_list<<<nl, 256, 0, c->stream>>>(view(c), c->d.leaf_first.p, c->d.leaf_count.p, c->d.u_ptr32.p,
                                          c->d.u_src.p, c->d.near_off.p, c->d.near_w.p, dbase.p, lpos.p, lk.p, lj.p);
  k_near_eval<<<(unsigned)((nnz + 255) / 256), 256, 0, c->stream>>>(view(c), nnz, lpos.p, lk.p, lj.p,
                                                                      c->d.near_val.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(c->stream));
}

void launch_moments(xrl_ctx* c) {
  const Tree& t = c->tree;
  const int N = c->N;
  const int p = c->p;
  const int nl = t.n_leaves();
  const double h = t.side / (double)(1 << t.L);
  std::vector<double> ctr(3 * (size_t)nl);
  for (int i = 0; i < nl; ++i) {
    uint32_t x, y, z;
    morton_decode(t.box_key[t.level_off[t.L] + i], &x, &y, &z);
    ctr[3 * i + 0] = t.lo[0] + (x + 0.5) * h;
    ctr[3 * i + 1] = t.lo[1] + (y + 0.5) * h;
    ctr[3 * i + 2] = t.lo[2] + (z + 0.5) * h;
  }
  std::vector<double> rule;
  int qm = (p + 3) / 2;
  collapsed_rule(qm, rule);
  DBuf<double> dctr, drule;
  dctr.upload(c->alloc, ctr);
  drule.upload(c->alloc, rule);
  DBuf<int32_t> leaf_of;
  leaf_of.upload(c->alloc, t.leaf_of);
  c->d.mom.alloc(c->alloc, (size_t)N * c->ncoef);
  k_moments<<<(N + 127) / 128, 128, 0, c->stream>>>(N, p, c->d.vtx.p, c->d.tri.p, c->d.area.p, leaf_of.p, dctr.p,
                                                     1.0 / h, drule.p, qm * qm, c->d.mom.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(c->stream));
}

// P entries of a list of panel pairs (Morton ranks), with the rule table
__global__ void k_pair_entries(PanelView pv, int n, const int32_t* __restrict__ pk, const int32_t* __restrict__ pl,
                               double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = p_entry(pv, pk[i], pl[i]);
}

std::vector<double> pair_entries(xrl_ctx* c, const std::vector<int32_t>& k, const std::vector<int32_t>& l) {
  XRL_CHECK(k.size() == l.size(), XRL_EINVAL, "pair list sizes differ");
  const int n = (int)k.size();
  if (n == 0) return {};
  std::vector<int32_t> rk(n), rl(n);
  for (int i = 0; i < n; ++i) {
    XRL_CHECK(k[i] >= 0 && k[i] < c->N && l[i] >= 0 && l[i] < c->N, XRL_EINVAL, "pair panel out of range");
    rk[i] = c->tree.rank[k[i]];
    rl[i] = c->tree.rank[l[i]];
  }
  DBuf<int32_t> dk, dl;
  DBuf<double> dv;
  dk.upload(c->alloc, rk);
  dl.upload(c->alloc, rl);
  dv.alloc(c->alloc, n);
  k_pair_entries<<<(n + 255) / 256, 256, 0, c->stream>>>(view(c), n, dk.p, dl.p, dv.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(c->stream));
  return dv.download();
}

void launch_direct(xrl_ctx* c, int nc, const double* X, double* Y, cudaStream_t s) {
  k_direct<<<c->N, 256, 256 * sizeof(double), s>>>(view(c), c->N, nc, nullptr, X, Y);
  XRL_CUDA(cudaGetLastError());
}

void launch_direct_rows(xrl_ctx* c, int nrows, const int32_t* rows, int nc, const double* X, double* Y,
                        cudaStream_t s) {
  if (nrows <= 0) return;
  k_direct<<<nrows, 256, 256 * sizeof(double), s>>>(view(c), c->N, nc, rows, X, Y);
  XRL_CUDA(cudaGetLastError());
}

}  // namespace xrl
