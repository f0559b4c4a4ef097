// Multigrid application of the diagonal-of-P preconditioner Q(f) (eq. 10)
// for meshes whose loop matrix has no narrow band (planes with many holes).
//
// The paper factors Q with a sparse LU (MKL Pardiso, Sec. II-D).  For vertex
// loops Q is a surface Laplacian with complex panel weights (Z_s/A + j omega
// mu0/4pi P_ll), so a smoothed-aggregation algebraic multigrid V-cycle
// (Vanek, Mandel and Brezina, 1996) approximates Q^-1 well; FGMRES, being
// flexible, takes it as its preconditioner.
//
// Setup (host, once per mesh, frequency independent).  Q(f) = sum_m
// Z_s^m(f) QA_m + j omega mu0/4pi QP is a pencil of W = n_mat + 1 real
// matrices with one sparsity pattern, so every level keeps a pencil too:
//  * strength: a_ij of the real sum of the pencil's components, each scaled
//    by the mean magnitude of its diagonal; j is a strong neighbour of i when
//    |a_ij| >= eps sqrt(|a_ii a_jj|), eps = 0.08 / 2^level;
//  * aggregation (greedy, in row order): a node whose strong neighbours are
//    all free starts an aggregate with them; free nodes then join the
//    aggregate of their strongest aggregated neighbour; the rest start their
//    own aggregates;
//  * prolongation P = (I - w D^-1 A) P_t (P_t the aggregate indicator,
//    w = 4 / (3 lambda), lambda ~ the largest eigenvalue of D^-1 A by 20 power
//    iterations), restriction R = P^T, coarse pencil C_k = R A_k P for every
//    component k (Galerkin);
//  * levels until at most kCoarse unknowns (or coarsening stalls).
// Apply (device, FP32 complex): per frequency the level matrices' values and
// Jacobi diagonals are combined from the pencils once per solve, and the
// coarsest matrix is inverted (Gauss-Jordan with partial pivoting, one CTA per
// frequency); per preconditioner application opt.mg_cycles V-cycles, each
// with kSweeps damped Jacobi sweeps before and after the coarse correction.
// The global (homology and port) loops have long rows that spoil
// aggregation; up to kCoarse of them are eliminated instead: the hierarchy is
// built on the vertex-loop block A_vv only, and per frequency the Schur
// complement S = A_gg - A_gv A_vv^-1 A_vg (dense, ng x ng, A_vv^-1 by V-cycles
// on the columns of A_vg) is inverted, so that an application is two
// multigrid solves around an exact solve of the global loops.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "cplx.cuh"
#include "xrl_internal.hpp"

namespace xrl {

namespace {

constexpr int kCoarse = 2560;     // coarsest level size for the dense inverse
constexpr int kMaxLevels = 12;
constexpr int kSweeps = 2;        // Jacobi sweeps before and after the coarse correction
constexpr float kOmegaJ = 0.6f;   // Jacobi damping

struct Csr {
  int n = 0, m = 0;                // rows, columns
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;         // [nnz][W]
};

// real strength matrix values: pencil components scaled by their mean |diagonal|
std::vector<double> strength_values(const Csr& A, int W) {
  std::vector<double> sc(W, 0.0);
  std::vector<int> cnt(W, 0);
  for (int i = 0; i < A.n; ++i)
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (A.col[q] == i)
        for (int k = 0; k < W; ++k) {
          sc[k] += std::fabs(A.val[q * W + k]);
          cnt[k]++;
        }
  for (int k = 0; k < W; ++k) sc[k] = (cnt[k] && sc[k] > 0) ? cnt[k] / sc[k] : 0.0;
  std::vector<double> s(A.col.size());
  for (size_t q = 0; q < A.col.size(); ++q) {
    double v = 0.0;
    for (int k = 0; k < W; ++k) v += A.val[q * W + k] * sc[k];
    s[q] = v;
  }
  return s;
}

// Galerkin product R A P for all W components (R = P^T given as CSR over coarse rows)
Csr galerkin(const Csr& A, int W, const Csr& P, const Csr& R) {
  const int nc = P.m;
  // AP = A P (n x nc)
  Csr AP;
  AP.n = A.n;
  AP.m = nc;
  AP.ptr.assign(A.n + 1, 0);
  std::vector<int32_t> mark(nc, -1);
  std::vector<double> acc((size_t)nc * W, 0.0);
  std::vector<int32_t> cols;
  for (int i = 0; i < A.n; ++i) {
    cols.clear();
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      const int j = A.col[q];
      for (int64_t t = P.ptr[j]; t < P.ptr[j + 1]; ++t) {
        const int cc = P.col[t];
        const double pv = P.val[t];
        if (mark[cc] != i) {
          mark[cc] = i;
          cols.push_back(cc);
          for (int k = 0; k < W; ++k) acc[(size_t)cc * W + k] = 0.0;
        }
        for (int k = 0; k < W; ++k) acc[(size_t)cc * W + k] += A.val[q * W + k] * pv;
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int cc : cols) {
      AP.col.push_back(cc);
      for (int k = 0; k < W; ++k) AP.val.push_back(acc[(size_t)cc * W + k]);
    }
    AP.ptr[i + 1] = (int64_t)AP.col.size();
  }
  // C = R AP (nc x nc)
  Csr C;
  C.n = nc;
  C.m = nc;
  C.ptr.assign(nc + 1, 0);
  std::fill(mark.begin(), mark.end(), -1);
  for (int r = 0; r < nc; ++r) {
    cols.clear();
    for (int64_t t = R.ptr[r]; t < R.ptr[r + 1]; ++t) {
      const int i = R.col[t];
      const double rv = R.val[t];
      for (int64_t q = AP.ptr[i]; q < AP.ptr[i + 1]; ++q) {
        const int cc = AP.col[q];
        if (mark[cc] != r) {
          mark[cc] = r;
          cols.push_back(cc);
          for (int k = 0; k < W; ++k) acc[(size_t)cc * W + k] = 0.0;
        }
        for (int k = 0; k < W; ++k) acc[(size_t)cc * W + k] += rv * AP.val[q * W + k];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int cc : cols) {
      C.col.push_back(cc);
      for (int k = 0; k < W; ++k) C.val.push_back(acc[(size_t)cc * W + k]);
    }
    C.ptr[r + 1] = (int64_t)C.col.size();
  }
  return C;
}

// transpose of a real CSR (values one per entry)
Csr transpose1(const Csr& P) {
  Csr R;
  R.n = P.m;
  R.m = P.n;
  R.ptr.assign(P.m + 1, 0);
  for (int32_t cc : P.col) R.ptr[cc + 1]++;
  for (int r = 0; r < P.m; ++r) R.ptr[r + 1] += R.ptr[r];
  R.col.resize(P.col.size());
  R.val.resize(P.col.size());
  std::vector<int64_t> pos(R.ptr.begin(), R.ptr.end() - 1);
  for (int i = 0; i < P.n; ++i)
    for (int64_t t = P.ptr[i]; t < P.ptr[i + 1]; ++t) {
      const int64_t d = pos[P.col[t]]++;
      R.col[d] = i;
      R.val[d] = P.val[t];
    }
  return R;
}

// smoothed-aggregation prolongator of one level; returns false when no
// coarsening happened.  `special` marks the global (homology and port) loops:
// each stays a singleton aggregate, so that it reaches the coarsest level and
// its dense solve unchanged, and the local aggregation ignores its long rows
// (a global loop taken into a local aggregate would drag that aggregate along
// its whole path).  On return `special` marks the coarse singletons.
bool prolongator(const Csr& A, int W, int level, Csr& P, std::vector<char>& special) {
  const int n = A.n;
  const std::vector<double> s = strength_values(A, W);
  std::vector<double> diag(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (A.col[q] == i) diag[i] = s[q];
  const double eps = 0.08 / (double)(1 << level);
  auto strong = [&](int i, int64_t q) {
    const int j = A.col[q];
    return j != i && !special[j] && std::fabs(s[q]) >= eps * std::sqrt(std::fabs(diag[i] * diag[j]));
  };
  std::vector<int32_t> agg(n, -1);
  int na = 0;
  std::vector<char> cspecial;
  for (int i = 0; i < n; ++i)
    if (special[i]) {
      agg[i] = na++;
      cspecial.push_back(1);
    }
  // pass 1: nodes whose strong neighbourhood is entirely free
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free = true, any = false;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1] && free; ++q)
      if (strong(i, q)) {
        any = true;
        if (agg[A.col[q]] >= 0) free = false;
      }
    if (!free || !any) continue;
    agg[i] = na;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (strong(i, q)) agg[A.col[q]] = na;
    ++na;
    cspecial.push_back(0);
  }
  // pass 2: join the strongest aggregated neighbour
  std::vector<int32_t> agg2(agg);
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    double best = -1.0;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (strong(i, q) && agg[A.col[q]] >= 0 && std::fabs(s[q]) > best) {
        best = std::fabs(s[q]);
        agg2[i] = agg[A.col[q]];
      }
  }
  agg.swap(agg2);
  // pass 3: what is left forms aggregates with its free strong neighbours
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (strong(i, q) && agg[A.col[q]] < 0) agg[A.col[q]] = na;
    ++na;
    cspecial.push_back(0);
  }
  if (na >= n || na == 0) return false;
  // lambda_max(D^-1 A) by power iteration on the strength matrix
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.001 * (double)(i % 97);
  double lam = 1.0;
  for (int it = 0; it < 20; ++it) {
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      double v = 0.0;
      for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) v += s[q] * x[A.col[q]];
      y[i] = diag[i] != 0.0 ? v / diag[i] : 0.0;
      nrm += y[i] * y[i];
    }
    nrm = std::sqrt(nrm);
    double xn = 0.0;
    for (int i = 0; i < n; ++i) xn += x[i] * x[i];
    lam = nrm / std::sqrt(xn);
    if (nrm == 0.0) break;
    for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
  }
  const double w = 4.0 / (3.0 * std::max(lam, 1e-30));
  // P = (I - w D^-1 S) P_t, one row per fine node
  P.n = n;
  P.m = na;
  P.ptr.assign(n + 1, 0);
  P.col.clear();
  P.val.clear();
  std::vector<int32_t> mark(na, -1), cols;
  std::vector<double> acc(na, 0.0);
  for (int i = 0; i < n; ++i) {
    cols.clear();
    auto add = [&](int a, double v) {
      if (mark[a] != i) {
        mark[a] = i;
        cols.push_back(a);
        acc[a] = 0.0;
      }
      acc[a] += v;
    };
    add(agg[i], 1.0);
    if (diag[i] != 0.0)
      for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) add(agg[A.col[q]], -w * s[q] / diag[i]);
    std::sort(cols.begin(), cols.end());
    for (int a : cols)
      if (acc[a] != 0.0) {
        P.col.push_back(a);
        P.val.push_back(acc[a]);
      }
    P.ptr[i + 1] = (int64_t)P.col.size();
  }
  special.swap(cspecial);
  return true;
}

// ---- device kernels (FP32 complex) ----------------------------------------------------------
__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fscl(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// values of one level for frequency f: a = sum_m zs_m(f) v_m + j wp(f) v_P
__global__ void k_amg_vals(int64_t nnz, int W, int nf, const double* __restrict__ pen, const cplx* __restrict__ zsf,
                           const double* __restrict__ wpf, float2* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  const int f = blockIdx.y;
  const int nm = W - 1;
  const double* v = pen + q * W;
  double re = 0.0, im = wpf[f] * v[nm];
  for (int m = 0; m < nm; ++m) {
    const cplx z = zsf[(size_t)f * nm + m];
    re += z.x * v[m];
    im += z.y * v[m];
  }
  out[(size_t)f * nnz + q] = make_float2((float)re, (float)im);
}

__global__ void k_amg_dinv(int n, int64_t nnz, const int64_t* __restrict__ dpos, const float2* __restrict__ vals,
                           float2* __restrict__ dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int f = blockIdx.y;
  const int64_t q = dpos[i];
  float2 d = q >= 0 ? vals[(size_t)f * nnz + q] : make_float2(0.f, 0.f);
  const float m2 = d.x * d.x + d.y * d.y;
  dinv[(size_t)f * n + i] = m2 > 0.f ? make_float2(d.x / m2, -d.y / m2) : make_float2(0.f, 0.f);
}

// r = b - A_f x (x = NULL: r = b) for all systems; system s has frequency s / nport
__global__ void k_amg_resid(int n, int nsys, int nport, int64_t nnz, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ col, const float2* __restrict__ vals,
                            const float2* __restrict__ b, const float2* __restrict__ x, float2* __restrict__ r) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), i = (int)(idx % n);
  float2 acc = b[idx];
  if (x) {
    const float2* va = vals + (size_t)(s / nport) * nnz;
    const float2* xs = x + (size_t)s * n;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) acc = fsub(acc, fmul(va[q], xs[col[q]]));
  }
  r[idx] = acc;
}

// x = (x or 0) + omega D^-1 r
__global__ void k_amg_jacobi(int n, int nsys, int nport, const float2* __restrict__ dinv, const float2* __restrict__ r,
                             float2* __restrict__ x, float omega, int init) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), i = (int)(idx % n);
  const float2 d = fscl(fmul(dinv[(size_t)(s / nport) * n + i], r[idx]), omega);
  x[idx] = init ? d : fadd(x[idx], d);
}

// y[s][i] (=, or +=) sum_t M[i][t] x[s][t] for a real CSR M (restriction, prolongation)
__global__ void k_amg_transfer(int n, int m, int nsys, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                               const float* __restrict__ val, const float2* __restrict__ x, float2* __restrict__ y,
                               int add) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), i = (int)(idx % n);
  const float2* xs = x + (size_t)s * m;
  float2 acc = make_float2(0.f, 0.f);
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) acc = fadd(acc, fscl(xs[col[q]], val[q]));
  y[idx] = add ? fadd(y[idx], acc) : acc;
}

// dense coarsest matrix of frequency f: [A | I] row-major n x 2n
__global__ void k_amg_dense(int n, int64_t nnz, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const float2* __restrict__ vals, float2* __restrict__ aug) {
  const int f = blockIdx.y;
  float2* a = aug + (size_t)f * n * 2 * n;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    float2* row = a + (size_t)i * 2 * n;
    for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) row[j] = make_float2(j == n + i ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int q = ptr[i] + threadIdx.x; q < ptr[i + 1]; q += blockDim.x) row[col[q]] = vals[(size_t)f * nnz + q];
    __syncthreads();
  }
}

// Gauss-Jordan with partial pivoting on [A | I] (one CTA per frequency, n <=
// kCoarse); the right half becomes A^-1.  Per pivot step the pivot column is
// copied to shared memory first, then every row is updated by the whole
// block (consecutive threads on consecutive columns).  *bad is set when a
// pivot vanishes.
__global__ void __launch_bounds__(1024) k_amg_gauss_jordan(int n, float2* __restrict__ aug, int32_t* __restrict__ bad) {
  const int f = blockIdx.x;
  float2* a = aug + (size_t)f * n * 2 * n;
  const int ld = 2 * n;
  __shared__ float sv[1024];
  __shared__ int si[1024];
  __shared__ float2 fcol[kCoarse];
  __shared__ float2 inv_s;
  for (int k = 0; k < n; ++k) {
    float best = -1.f;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const float2 v = a[(size_t)i * ld + k];
      const float m = v.x * v.x + v.y * v.y;
      if (m > best) {
        best = m;
        bi = i;
      }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st && sv[threadIdx.x + st] > sv[threadIdx.x]) {
        sv[threadIdx.x] = sv[threadIdx.x + st];
        si[threadIdx.x] = si[threadIdx.x + st];
      }
      __syncthreads();
    }
    const int p = si[0];
    const bool zero = !(sv[0] > 0.f);
    __syncthreads();
    if (zero) {
      if (threadIdx.x == 0) atomicExch(bad, 1);
      return;
    }
    if (p != k)
      for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        const float2 t = a[(size_t)k * ld + j];
        a[(size_t)k * ld + j] = a[(size_t)p * ld + j];
        a[(size_t)p * ld + j] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      const float2 d = a[(size_t)k * ld + k];
      const float m2 = d.x * d.x + d.y * d.y;
      inv_s = make_float2(d.x / m2, -d.y / m2);
    }
    __syncthreads();
    const float2 inv = inv_s;
    for (int j = threadIdx.x; j < ld; j += blockDim.x) a[(size_t)k * ld + j] = fmul(a[(size_t)k * ld + j], inv);
    for (int i = threadIdx.x; i < n; i += blockDim.x) fcol[i] = a[(size_t)i * ld + k];
    __syncthreads();
    const float2* rk = a + (size_t)k * ld;
    for (int i = 0; i < n; ++i) {
      const float2 fct = fcol[i];
      if (i == k || (fct.x == 0.f && fct.y == 0.f)) continue;
      float2* ri = a + (size_t)i * ld;
      for (int j = k + threadIdx.x; j < ld; j += blockDim.x) ri[j] = fsub(ri[j], fmul(fct, rk[j]));
    }
    __syncthreads();
  }
}

// x[s] = A_f^-1 b[s] with the right half of the Gauss-Jordan array
__global__ void k_amg_dense_apply(int n, int nsys, int nport, const float2* __restrict__ aug,
                                  const float2* __restrict__ b, float2* __restrict__ x) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), i = (int)(idx % n);
  const float2* row = aug + ((size_t)(s / nport) * n + i) * 2 * n + n;
  const float2* bs = b + (size_t)s * n;
  float2 acc = make_float2(0.f, 0.f);
  for (int j = 0; j < n; ++j) acc = fadd(acc, fmul(row[j], bs[j]));
  x[idx] = acc;
}

__global__ void k_amg_to32(size_t n, const cplx* __restrict__ a, float2* __restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k_amg_to64(size_t n, const float2* __restrict__ a, cplx* __restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

unsigned nb256(size_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// ---- host side -----------------------------------------------------------------------------
void amg_prepare(xrl_ctx* c) {
  const Topo& T = c->topo;
  AmgHier& H = c->amg;
  H = AmgHier();
  const int W = T.n_mat + 1;
  H.W = W;
  // split Q = [A_vv A_vg; A_gv A_gg]: vertex loops first, then the global
  // loops (their long rows are eliminated by the Schur complement, or, when
  // there are more than kCoarse of them, kept as singleton aggregates)
  const int n = T.n_loops, nv = T.n_vertex_loops, ng = n - nv;
  const bool schur = ng > 0 && ng <= kCoarse && nv > 0;
  Csr A, Avg, Agv, Agg;
  auto block = [&](Csr& B, int r0, int r1, int c0, int c1) {
    B.n = r1 - r0;
    B.m = c1 - c0;
    B.ptr.assign(B.n + 1, 0);
    for (int i = r0; i < r1; ++i) {
      for (int64_t q = T.q_ptr[i]; q < T.q_ptr[i + 1]; ++q) {
        const int j = T.q_col[q];
        if (j < c0 || j >= c1) continue;
        B.col.push_back(j - c0);
        for (int k = 0; k < W; ++k) B.val.push_back(T.q_val[(size_t)q * W + k]);
      }
      B.ptr[i - r0 + 1] = (int64_t)B.col.size();
    }
  };
  std::vector<char> special;
  if (schur) {
    block(A, 0, nv, 0, nv);
    block(Avg, 0, nv, nv, n);
    block(Agv, nv, n, 0, nv);
    block(Agg, nv, n, nv, n);
    special.assign(nv, 0);
    auto up = [&](const Csr& B, AmgBlock& D) {
      D.n = B.n;
      D.nnz = (int64_t)B.col.size();
      XRL_CHECK(B.col.size() < (size_t)INT32_MAX, XRL_ENOMEM, "global-loop block too large for 32-bit indices");
      D.ptr.upload(c->alloc, std::vector<int32_t>(B.ptr.begin(), B.ptr.end()));
      D.col.upload(c->alloc, B.col);
      D.pen.upload(c->alloc, B.val);
    };
    up(Avg, H.vg);
    up(Agv, H.gv);
    up(Agg, H.gg);
    H.nv = nv;
    H.ng = ng;
  } else {
    A.n = A.m = n;
    A.ptr = T.q_ptr;
    A.col = T.q_col;
    A.val = T.q_val;
    special.assign(n, 0);
    for (int i = nv; i < n; ++i) special[i] = 1;
    H.nv = n;
    H.ng = 0;
  }
  for (int lev = 0; lev < kMaxLevels; ++lev) {
    AmgLevel L;
    L.n = A.n;
    L.nnz = (int64_t)A.col.size();
    std::vector<int32_t> p32(A.ptr.begin(), A.ptr.end());
    std::vector<int64_t> dpos(A.n, -1);
    for (int i = 0; i < A.n; ++i)
      for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
        if (A.col[q] == i) dpos[i] = q;
    XRL_CHECK(A.col.size() < (size_t)INT32_MAX, XRL_ENOMEM, "multigrid level too large for 32-bit indices");
    L.ptr.upload(c->alloc, p32);
    L.col.upload(c->alloc, A.col);
    L.pen.upload(c->alloc, A.val);
    L.dpos.upload(c->alloc, dpos);
    Csr P;
    const bool last = A.n <= kCoarse || lev == kMaxLevels - 1 || !prolongator(A, W, lev, P, special) ||
                      P.m > (int)(0.85 * A.n);
    if (last) {
      L.coarsest = true;
      H.lv.push_back(std::move(L));
      break;
    }
    const Csr R = transpose1(P);
    std::vector<int32_t> pp(P.ptr.begin(), P.ptr.end()), rp(R.ptr.begin(), R.ptr.end());
    std::vector<float> pv(P.val.begin(), P.val.end()), rv(R.val.begin(), R.val.end());
    L.nc = P.m;
    L.p_ptr.upload(c->alloc, pp);
    L.p_col.upload(c->alloc, P.col);
    L.p_val.upload(c->alloc, pv);
    L.r_ptr.upload(c->alloc, rp);
    L.r_col.upload(c->alloc, R.col);
    L.r_val.upload(c->alloc, rv);
    H.lv.push_back(std::move(L));
    A = galerkin(A, W, P, R);
  }
  H.ready = true;
}

// y[s][i] = (b ? b[s][i] : 0) - sum_q B_f(s)[i][col q] x[s][col q] for a CSR
// block B of `rows` rows over vectors x of length m (system s at frequency s / nport)
__global__ void k_amg_bmv(int rows, int m, int nsys, int nport, int64_t nnz, const int32_t* __restrict__ ptr,
                          const int32_t* __restrict__ col, const float2* __restrict__ vals,
                          const float2* __restrict__ b, const float2* __restrict__ x, float2* __restrict__ y) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * nsys) return;
  const int s = (int)(idx / rows), i = (int)(idx % rows);
  const float2* va = vals + (size_t)(s / nport) * nnz;
  const float2* xs = x + (size_t)s * m;
  float2 acc = b ? b[idx] : make_float2(0.f, 0.f);
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) acc = fsub(acc, fmul(va[q], xs[col[q]]));
  y[idx] = acc;
}

// columns j0 .. j0 + ch - 1 of A_vg(f) as right-hand sides B[f ch + jj][i] (B zeroed before)
__global__ void k_amg_gather_cols(int nv, int nf, int j0, int ch, int64_t nnz, const int32_t* __restrict__ ptr,
                                  const int32_t* __restrict__ col, const float2* __restrict__ vals,
                                  float2* __restrict__ B) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nv * nf) return;
  const int f = (int)(idx / nv), i = (int)(idx % nv);
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int j = col[q] - j0;
    if (j >= 0 && j < ch) B[((size_t)f * ch + j) * nv + i] = vals[(size_t)f * nnz + q];
  }
}

// out[i][s] = in[s][i]  (S systems of length n)
__global__ void k_amg_transpose(int S, int n, const float2* __restrict__ in, float2* __restrict__ out) {
  __shared__ float2 t[32][33];
  const int i0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int sv = s0 + r, iv = i0 + threadIdx.x;
    if (sv < S && iv < n) t[r][threadIdx.x] = in[(size_t)sv * n + iv];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int iv = i0 + r, sv = s0 + threadIdx.x;
    if (sv < S && iv < n) out[(size_t)iv * S + sv] = t[threadIdx.x][r];
  }
}

// Schur columns: aug[f][i][j0 + jj] -= sum_k A_gv(f)[i][k] Y[k][f ch + jj]  (Y transposed, [nv][nf ch])
__global__ void k_amg_schur(int ng, int nf, int j0, int ch, int64_t nnz, const int32_t* __restrict__ ptr,
                            const int32_t* __restrict__ col, const float2* __restrict__ vals,
                            const float2* __restrict__ Yt, float2* __restrict__ aug) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nf * ng * ch) return;
  const int jj = (int)(idx % ch);
  const size_t r = idx / ch;
  const int i = (int)(r % ng), f = (int)(r / ng);
  const float2* va = vals + (size_t)f * nnz;
  const size_t S = (size_t)nf * ch;
  float2 acc = make_float2(0.f, 0.f);
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) acc = fadd(acc, fmul(va[q], Yt[(size_t)col[q] * S + (size_t)f * ch + jj]));
  float2* e = aug + ((size_t)f * ng + i) * 2 * ng + j0 + jj;
  *e = fsub(*e, acc);
}

__global__ void k_amg_split(int n, int nv, int nsys, const cplx* __restrict__ v, float2* __restrict__ bv,
                            float2* __restrict__ bg) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), i = (int)(idx % n);
  const float2 x = make_float2((float)v[idx].x, (float)v[idx].y);
  if (i < nv)
    bv[(size_t)s * nv + i] = x;
  else
    bg[(size_t)s * (n - nv) + i - nv] = x;
}

__global__ void k_amg_join(int n, int nv, int nsys, const float2* __restrict__ zv, const float2* __restrict__ zg,
                           cplx* __restrict__ z) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), i = (int)(idx % n);
  const float2 x = i < nv ? zv[(size_t)s * nv + i] : zg[(size_t)s * (n - nv) + i - nv];
  z[idx] = make_double2((double)x.x, (double)x.y);
}

__global__ void k_amg_axpy(size_t n, const float2* __restrict__ a, float2* __restrict__ b, int init);
static const float2* mg_solve(xrl_ctx* c, AmgWork& w, int nsys, int nport, int ncyc, cudaStream_t s);

// per-solve values: level matrices for nf frequencies, Jacobi diagonals, the
// coarsest inverse, and with global loops the inverted Schur complement
// S(f) = A_gg - A_gv A_vv^-1 A_vg (A_vv^-1 by max(2, mg_cycles) V-cycles on the
// columns of A_vg, ch of them per pass)
void amg_factor(xrl_ctx* c, AmgWork& w, int nf, int nsys, const cplx* zsf, const double* wpf, cudaStream_t s) {
  AmgHier& H = c->amg;
  XRL_CHECK(H.ready, XRL_ESTATE, "multigrid hierarchy not built");
  const int nl = (int)H.lv.size();
  const int ng = H.ng, nv = H.nv;
  const int ch = ng > 0 ? std::min(ng, std::max(1, (int)(((int64_t)1 << 29) / ((int64_t)nf * nv * 8)))) : 0;
  w.nf = nf;
  w.cap = std::max(nsys, nf * ch);
  w.lv.resize(nl);
  w.err.alloc(c->alloc, 1);
  XRL_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int32_t), s));
  const int ncyc = std::max(1, c->opt.mg_cycles);
  for (int l = 0; l < nl; ++l) {
    AmgLevel& L = H.lv[l];
    AmgLevelWork& K = w.lv[l];
    K.vals.alloc(c->alloc, (size_t)nf * L.nnz);
    K.dinv.alloc(c->alloc, (size_t)nf * L.n);
    K.x.alloc(c->alloc, (size_t)w.cap * L.n);
    K.b.alloc(c->alloc, (size_t)w.cap * L.n);
    K.r.alloc(c->alloc, (size_t)w.cap * L.n);
    k_amg_vals<<<dim3(nb256(L.nnz), nf), 256, 0, s>>>(L.nnz, H.W, nf, L.pen.p, zsf, wpf, K.vals.p);
    k_amg_dinv<<<dim3(nb256(L.n), nf), 256, 0, s>>>(L.n, L.nnz, L.dpos.p, K.vals.p, K.dinv.p);
    count_launch(c, 2);
    if (l == 0 && (ncyc > 1 || ng > 0)) {
      w.bsave.alloc(c->alloc, (size_t)w.cap * L.n);
      w.xacc.alloc(c->alloc, (size_t)w.cap * L.n);
    }
    if (L.coarsest && L.n <= kCoarse) {
      K.aug.alloc(c->alloc, (size_t)nf * L.n * 2 * L.n);
      k_amg_dense<<<dim3(std::min(L.n, 1024), nf), 256, 0, s>>>(L.n, L.nnz, L.ptr.p, L.col.p, K.vals.p, K.aug.p);
      k_amg_gauss_jordan<<<nf, 1024, 0, s>>>(L.n, K.aug.p, w.err.p);
      count_launch(c, 2);
    }
  }
  if (ng > 0) {
    auto vals = [&](const AmgBlock& B, DBuf<float2>& out) {
      out.alloc(c->alloc, (size_t)nf * B.nnz);
      if (B.nnz) k_amg_vals<<<dim3(nb256(B.nnz), nf), 256, 0, s>>>(B.nnz, H.W, nf, B.pen.p, zsf, wpf, out.p);
      count_launch(c);
    };
    vals(H.vg, w.vg_vals);
    vals(H.gv, w.gv_vals);
    vals(H.gg, w.gg_vals);
    w.saug.alloc(c->alloc, (size_t)nf * ng * 2 * ng);
    k_amg_dense<<<dim3(std::min(ng, 1024), nf), 256, 0, s>>>(ng, H.gg.nnz, H.gg.ptr.p, H.gg.col.p, w.gg_vals.p,
                                                             w.saug.p);
    count_launch(c);
    DBuf<float2> Yt;
    Yt.alloc(c->alloc, (size_t)nf * ch * nv);
    AmgLevelWork& K0 = w.lv[0];
    for (int j0 = 0; j0 < ng; j0 += ch) {
      const int cj = std::min(ch, ng - j0);
      const int S = nf * cj;
      XRL_CUDA(cudaMemsetAsync(K0.b.p, 0, sizeof(float2) * (size_t)S * nv, s));
      k_amg_gather_cols<<<nb256((size_t)nv * nf), 256, 0, s>>>(nv, nf, j0, cj, H.vg.nnz, H.vg.ptr.p, H.vg.col.p,
                                                               w.vg_vals.p, K0.b.p);
      const float2* Y = mg_solve(c, w, S, cj, std::max(2, ncyc), s);
      k_amg_transpose<<<dim3((nv + 31) / 32, (S + 31) / 32), dim3(32, 8), 0, s>>>(S, nv, Y, Yt.p);
      k_amg_schur<<<nb256((size_t)nf * ng * cj), 256, 0, s>>>(ng, nf, j0, cj, H.gv.nnz, H.gv.ptr.p, H.gv.col.p,
                                                              w.gv_vals.p, Yt.p, w.saug.p);
      count_launch(c, 3);
    }
    k_amg_gauss_jordan<<<nf, 1024, 0, s>>>(ng, w.saug.p, w.err.p);
    w.u.alloc(c->alloc, (size_t)nsys * nv);
    w.tg.alloc(c->alloc, (size_t)nsys * ng);
    w.zg.alloc(c->alloc, (size_t)nsys * ng);
    count_launch(c);
  }
  XRL_CUDA(cudaGetLastError());
}

__global__ void k_amg_axpy(size_t n, const float2* __restrict__ a, float2* __restrict__ b, int init) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = init ? a[i] : fadd(b[i], a[i]);
}

// one V-cycle: w.lv[0].x = V(w.lv[0].b)
static void vcycle(xrl_ctx* c, AmgWork& w, int nsys, int nport, cudaStream_t s) {
  AmgHier& H = c->amg;
  const int nl = (int)H.lv.size();
  // downward: pre-smooth, restrict the residual
  for (int l = 0; l < nl; ++l) {
    AmgLevel& L = H.lv[l];
    AmgLevelWork& K = w.lv[l];
    const size_t tot = (size_t)L.n * nsys;
    if (L.coarsest) {
      if (K.aug.n) {
        k_amg_dense_apply<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, K.aug.p, K.b.p, K.x.p);
        count_launch(c);
      } else {   // coarsening stalled above the dense size: Jacobi sweeps
        k_amg_jacobi<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, K.dinv.p, K.b.p, K.x.p, kOmegaJ, 1);
        for (int it = 1; it < 20; ++it) {
          k_amg_resid<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, L.nnz, L.ptr.p, L.col.p, K.vals.p, K.b.p,
                                                 K.x.p, K.r.p);
          k_amg_jacobi<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, K.dinv.p, K.r.p, K.x.p, kOmegaJ, 0);
        }
        count_launch(c, 39);
      }
      break;
    }
    k_amg_jacobi<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, K.dinv.p, K.b.p, K.x.p, kOmegaJ, 1);
    for (int it = 1; it < kSweeps; ++it) {
      k_amg_resid<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, L.nnz, L.ptr.p, L.col.p, K.vals.p, K.b.p, K.x.p,
                                             K.r.p);
      k_amg_jacobi<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, K.dinv.p, K.r.p, K.x.p, kOmegaJ, 0);
    }
    k_amg_resid<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, L.nnz, L.ptr.p, L.col.p, K.vals.p, K.b.p, K.x.p, K.r.p);
    const size_t totc = (size_t)L.nc * nsys;
    k_amg_transfer<<<nb256(totc), 256, 0, s>>>(L.nc, L.n, nsys, L.r_ptr.p, L.r_col.p, L.r_val.p, K.r.p,
                                               w.lv[l + 1].b.p, 0);
    count_launch(c, 2 * kSweeps + 1);
  }
  // upward: prolongate the correction, post-smooth
  for (int l = nl - 2; l >= 0; --l) {
    AmgLevel& L = H.lv[l];
    AmgLevelWork& K = w.lv[l];
    const size_t tot = (size_t)L.n * nsys;
    k_amg_transfer<<<nb256(tot), 256, 0, s>>>(L.n, L.nc, nsys, L.p_ptr.p, L.p_col.p, L.p_val.p, w.lv[l + 1].x.p,
                                              K.x.p, 1);
    for (int it = 0; it < kSweeps; ++it) {
      k_amg_resid<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, L.nnz, L.ptr.p, L.col.p, K.vals.p, K.b.p, K.x.p,
                                             K.r.p);
      k_amg_jacobi<<<nb256(tot), 256, 0, s>>>(L.n, nsys, nport, K.dinv.p, K.r.p, K.x.p, kOmegaJ, 0);
    }
    count_launch(c, 1 + 2 * kSweeps);
  }
  XRL_CUDA(cudaGetLastError());
}

// ncyc V-cycles on w.lv[0].b (the later ones on the level-0 residual); returns
// the buffer holding the solution
static const float2* mg_solve(xrl_ctx* c, AmgWork& w, int nsys, int nport, int ncyc, cudaStream_t s) {
  AmgHier& H = c->amg;
  AmgLevel& L0 = H.lv[0];
  AmgLevelWork& K0 = w.lv[0];
  const size_t n0 = (size_t)L0.n * nsys;
  if (ncyc > 1) {
    k_amg_axpy<<<nb256(n0), 256, 0, s>>>(n0, K0.b.p, w.bsave.p, 1);
    count_launch(c);
  }
  vcycle(c, w, nsys, nport, s);
  if (ncyc == 1) return K0.x.p;
  for (int cy = 1; cy < ncyc; ++cy) {
    k_amg_axpy<<<nb256(n0), 256, 0, s>>>(n0, K0.x.p, w.xacc.p, cy == 1);
    k_amg_resid<<<nb256(n0), 256, 0, s>>>(L0.n, nsys, nport, L0.nnz, L0.ptr.p, L0.col.p, K0.vals.p, w.bsave.p,
                                          w.xacc.p, K0.b.p);
    count_launch(c, 2);
    vcycle(c, w, nsys, nport, s);
  }
  k_amg_axpy<<<nb256(n0), 256, 0, s>>>(n0, K0.x.p, w.xacc.p, 0);
  count_launch(c);
  return w.xacc.p;
}

// z ~= Q^-1 v; v, z [nsys][n_loops] FP64 complex.  Without global loops:
// opt.mg_cycles V-cycles.  With them, block elimination with the Schur
// complement of amg_factor:
//   u = A_vv^-1 v_v,  z_g = S^-1 (v_g - A_gv u),  z_v = A_vv^-1 (v_v - A_vg z_g)
void amg_apply(xrl_ctx* c, AmgWork& w, int nsys, int nport, const cplx* v, cplx* z, cudaStream_t s) {
  AmgHier& H = c->amg;
  AmgLevelWork& K0 = w.lv[0];
  const int nv = H.nv, ng = H.ng, n = nv + ng;
  const int ncyc = std::max(1, c->opt.mg_cycles);
  const size_t nvs = (size_t)nv * nsys, tot = (size_t)n * nsys;
  if (ng == 0) {
    k_amg_to32<<<nb256(nvs), 256, 0, s>>>(nvs, v, K0.b.p);
    const float2* x = mg_solve(c, w, nsys, nport, ncyc, s);
    k_amg_to64<<<nb256(nvs), 256, 0, s>>>(nvs, x, z);
    count_launch(c, 2);
    XRL_CUDA(cudaGetLastError());
    return;
  }
  k_amg_split<<<nb256(tot), 256, 0, s>>>(n, nv, nsys, v, w.bsave.p, w.tg.p);
  k_amg_axpy<<<nb256(nvs), 256, 0, s>>>(nvs, w.bsave.p, K0.b.p, 1);
  count_launch(c, 2);
  const float2* u = mg_solve(c, w, nsys, nport, ncyc, s);
  k_amg_axpy<<<nb256(nvs), 256, 0, s>>>(nvs, u, w.u.p, 1);
  const size_t ngs = (size_t)ng * nsys;
  k_amg_bmv<<<nb256(ngs), 256, 0, s>>>(ng, nv, nsys, nport, H.gv.nnz, H.gv.ptr.p, H.gv.col.p, w.gv_vals.p, w.tg.p,
                                       w.u.p, w.tg.p);
  k_amg_dense_apply<<<nb256(ngs), 256, 0, s>>>(ng, nsys, nport, w.saug.p, w.tg.p, w.zg.p);
  // bsave still holds v_v: mg_solve only reads its saved right-hand side
  count_launch(c, 3);
  k_amg_bmv<<<nb256(nvs), 256, 0, s>>>(nv, ng, nsys, nport, H.vg.nnz, H.vg.ptr.p, H.vg.col.p, w.vg_vals.p,
                                       w.bsave.p, w.zg.p, K0.b.p);
  count_launch(c);
  const float2* zv = mg_solve(c, w, nsys, nport, ncyc, s);
  k_amg_join<<<nb256(tot), 256, 0, s>>>(n, nv, nsys, zv, w.zg.p, z);
  count_launch(c);
  XRL_CUDA(cudaGetLastError());
}

// the coarsest inverse's pivot status (after the stream reached the factorisation)
void amg_check(xrl_ctx* c, AmgWork& w, cudaStream_t s) {
  if (!w.err.n) return;
  int32_t e = 0;
  XRL_CUDA(cudaMemcpyAsync(&e, w.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaStreamSynchronize(s));
  XRL_CHECK(e == 0, XRL_ENOCONV, "multigrid: the coarsest matrix is singular");
}

}  // namespace xrl
