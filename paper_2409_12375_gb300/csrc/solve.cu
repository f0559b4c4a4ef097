// Loop-space operator, diagonal-of-P preconditioner and batched flexible
// GMRES for the broadband sweep (sm_103a).
//
// Sec. II-C splits the loop system (eq. 7) as eq. 8-9:
//   Z(f) I_l = M [ sum_t A_t (diag(Z_s(f)/A) + j omega mu0/4pi P) A_t^T ] M^T I_l = V_l.
// One product therefore gathers panel currents I_pt = A_t^T M^T I_l (three
// Cartesian components, real and imaginary part: 6 real FMM columns per
// complex system), applies the frequency-independent P once to all columns
// of all (frequency, port) systems with the FMM, and scatters back with the
// per-system factors j omega mu0/4pi and Z_s(f)/A (Sec. II-D: "the potential
// part is computed once and scaled by j omega mu0/4pi").
//
// Preconditioner (Sec. II-D, eq. 10): Q(f) = M [sum_t A_t diag(Z_s/A +
// j omega mu0/4pi P_ll) A_t^T] M^T.  With one surface impedance per material,
// Q(f) = sum_m Z_s^m(f) QA_m + j omega mu0/4pi QP: a pencil of real sparse
// matrices built once (topology.cpp); the paper factors Q with a sparse LU
// (MKL Pardiso); here Q^-1 v is approximated on the GPU by Jacobi-
// preconditioned COCG (conjugate orthogonal CG for complex symmetric
// matrices) with a fixed iteration budget, which makes the preconditioner
// vary between applications, so the outer solver is right-preconditioned
// FLEXIBLE GMRES (the paper: mRHS-GMRES, restart 50, Sec. III).
//
// All systems of a sweep form one block: vectors are [n_sys][n_loops]
// complex (interleaved double2), every kernel loops over all systems, and
// converged systems are frozen by a device-side mask.
#include <cmath>
#include <vector>

#include "cplx.cuh"
#include "xrl_internal.hpp"

namespace xrl {

constexpr double kMu0Over4Pi = 1e-7;

// ---- per-system constants ------------------------------------------------------------------
// Z_s(f) of eq. 3: R_DC x / (1 - exp(-x)), x = (1+j) R_RF sqrt(f) / R_DC,
// series 1 + x/2 + x^2/12 - x^4/720 for |x| < 1e-3.
__global__ void k_sys_consts(int nsys, int nport, int nmat, const double* __restrict__ freq,
                             const double* __restrict__ sig, const double* __restrict__ thk,
                             cplx* __restrict__ zs, double* __restrict__ wp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys * nmat) return;
  int s = i / nmat, m = i % nmat;
  double f = freq[s / nport];
  double rdc = 2.0 / (sig[m] * thk[m]);
  double rrf = sqrt(3.14159265358979323846 * (4e-7 * 3.14159265358979323846) / sig[m]);
  double a = rrf * sqrt(f) / rdc;   // x = a (1 + j)
  cplx x = make_double2(a, a);
  cplx q;
  if (sqrt(2.0) * a < 1e-3) {
    cplx x2 = cm(x, x), x4 = cm(x2, x2);
    q = make_double2(1.0 + x.x / 2.0 + x2.x / 12.0 - x4.x / 720.0, x.y / 2.0 + x2.y / 12.0 - x4.y / 720.0);
  } else {
    // 1 - exp(-x) = -expm1(-a - j a) = -(expm1(-a) cos a - 2 sin^2(a/2)) + j e^{-a} sin a
    double sh = sin(0.5 * a);
    cplx den = make_double2(-(expm1(-a) * cos(a) - 2.0 * sh * sh), exp(-a) * sin(a));
    q = cdiv(x, den);
  }
  zs[i] = cscale(q, rdc);
  if (m == 0) wp[s] = 2.0 * 3.14159265358979323846 * f * kMu0Over4Pi;
}

// ---- operator pieces -------------------------------------------------------------------------
// complex arithmetic in the precision of the product (FP32 for the inner
// iterations, FP64 for the residuals)
template <class T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };
template <class C, class R>
__device__ __forceinline__ C cmk(R a, R b) { C r; r.x = a; r.y = b; return r; }
template <class C>
__device__ __forceinline__ C cadd_t(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <class C>
__device__ __forceinline__ C csub_t(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <class C>
__device__ __forceinline__ C cmul_t(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <class C, class R>
__device__ __forceinline__ C cscale_t(C a, R s) { a.x *= s; a.y *= s; return a; }

// X[r][6s + 2t + ri] = (A_t^T M^T v_s)(r); v is [nsys][nloop], or [nloop][nsys]
// with loop_major (then the threads of one panel read one contiguous row)
template <class T>
__global__ void k_gather(int N, int nsys, int nloop, const int32_t* __restrict__ pan_br,
                         const double* __restrict__ pan_rho, const int32_t* __restrict__ mt_ptr,
                         const int32_t* __restrict__ mt_col, const int8_t* __restrict__ mt_val,
                         const cplx* __restrict__ v, T* __restrict__ X, int loop_major) {
  typedef typename CT<T>::type C;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * nsys) return;
  int r = (int)(idx / nsys), s = (int)(idx % nsys);
  const cplx* vs = v + (size_t)s * nloop;
  C ip[3] = {cmk<C>((T)0, (T)0), cmk<C>((T)0, (T)0), cmk<C>((T)0, (T)0)};
  for (int k = 0; k < kPanEdges; ++k) {
    int b = pan_br[kPanEdges * r + k];
    if (b < 0) continue;
    C ie = cmk<C>((T)0, (T)0);
    for (int q = mt_ptr[b]; q < mt_ptr[b + 1]; ++q) {
      const cplx x = loop_major ? v[(size_t)mt_col[q] * nsys + s] : vs[mt_col[q]];
      const C xc = cmk<C>((T)x.x, (T)x.y);
      ie = mt_val[q] > 0 ? cadd_t(ie, xc) : csub_t(ie, xc);
    }
    const double* rho = pan_rho + 3 * kPanEdges * (size_t)r + 3 * k;
    for (int t = 0; t < 3; ++t) ip[t] = cadd_t(ip[t], cscale_t(ie, (T)rho[t]));
  }
  T* out = X + (size_t)r * 6 * nsys + 6 * s;
  for (int t = 0; t < 3; ++t) {
    out[2 * t] = ip[t].x;
    out[2 * t + 1] = ip[t].y;
  }
}

// out[l][s] = in[s][l] (systems fastest), 32 x 32 tiles through shared memory
__global__ void k_to_loop_major(int n, int nsys, const cplx* __restrict__ in, cplx* __restrict__ out) {
  __shared__ cplx tile[32][33];
  const int l0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int sy = s0 + k, lx = l0 + threadIdx.x;
    if (sy < nsys && lx < n) tile[k][threadIdx.x] = in[(size_t)sy * n + lx];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int ly = l0 + k, sx = s0 + threadIdx.x;
    if (ly < n && sx < nsys) out[(size_t)ly * nsys + sx] = tile[threadIdx.x][k];
  }
}

// Vb[b][s] = sum_side rho . (j w' Y + Z_s/A X) at the branch's panels
// (branch-major, systems fastest: coalesced X, Y reads and Vb writes)
template <class T>
__global__ void k_scatter(int B, int nsys, int nmat, const int32_t* __restrict__ br_pan,
                          const double* __restrict__ br_rho, const int32_t* __restrict__ pan_mat,
                          const double* __restrict__ area, const cplx* __restrict__ zs,
                          const double* __restrict__ wp, const T* __restrict__ X,
                          const T* __restrict__ Y, cplx* __restrict__ Vb) {
  typedef typename CT<T>::type C;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)B * nsys) return;
  int b = (int)(idx / nsys), s = (int)(idx % nsys);
  C acc = cmk<C>((T)0, (T)0);
  const T w = (T)wp[s];
  for (int side = 0; side < 2; ++side) {
    int r = br_pan[2 * b + side];
    if (r < 0) continue;
    const double* rho = br_rho + 6 * (size_t)b + 3 * side;
    const cplx zd = zs[s * nmat + pan_mat[r]];
    const T ia = (T)1 / (T)area[r];   // in the product's precision: no FP64 divide in the FP32 pass
    const C z = cmk<C>((T)zd.x * ia, (T)zd.y * ia);
    const T* xr = X + (size_t)r * 6 * nsys + 6 * s;
    const T* yr = Y + (size_t)r * 6 * nsys + 6 * s;
    for (int t = 0; t < 3; ++t) {
      const C xv = cmk<C>(xr[2 * t], xr[2 * t + 1]);
      const C val = cadd_t(cmul_t(z, xv), cmk<C>(-w * yr[2 * t + 1], w * yr[2 * t]));
      acc = cadd_t(acc, cscale_t(val, (T)rho[t]));
    }
  }
  Vb[idx] = make_double2((double)acc.x, (double)acc.y);
}

// w[s][l] = sum_b M(l, b) Vb[b][s]   (port branches carry no impedance: their Vb is zero)
// One warp per (loop, 32 systems): the row walk is warp-uniform and the Vb
// reads are contiguous over the systems.  Rows longer than kLongRow (the
// homology and port loops) are left to k_loop_reduce_long.
constexpr int kLongRow = 256;
__global__ void k_loop_reduce(int nloop, int nsys, int ncb, const int32_t* __restrict__ m_ptr,
                              const int32_t* __restrict__ m_col, const int8_t* __restrict__ m_val,
                              const cplx* __restrict__ Vb, cplx* __restrict__ w) {
  const size_t wid = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int sg = (nsys + 31) >> 5;
  if (wid >= (size_t)nloop * sg) return;
  const int l = (int)(wid / sg);
  const int s = (int)(wid % sg) * 32 + lane;
  const int q0 = m_ptr[l], q1 = m_ptr[l + 1];
  if (s >= nsys || q1 - q0 > kLongRow) return;
  cplx acc = make_double2(0, 0);
  for (int q = q0; q < q1; ++q) {
    const int b = m_col[q];
    if (b >= ncb) continue;
    const cplx v = Vb[(size_t)b * nsys + s];
    acc = m_val[q] > 0 ? cadd(acc, v) : csub(acc, v);
  }
  w[(size_t)s * nloop + l] = acc;
}

// The long rows: kLongSeg CTAs of 8 warps per (long row, 32 systems), each
// summing one segment of the row into part[row][seg][s]; k_loop_reduce_fin
// adds the segments in a fixed order.
constexpr int kLongSeg = 32;
__global__ void __launch_bounds__(256) k_loop_reduce_long(int nsys, int ncb, const int32_t* __restrict__ rows,
                                                          const int32_t* __restrict__ m_ptr,
                                                          const int32_t* __restrict__ m_col,
                                                          const int8_t* __restrict__ m_val,
                                                          const cplx* __restrict__ Vb, cplx* __restrict__ part) {
  __shared__ cplx red[8][32];
  const int l = rows[blockIdx.x], seg = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.z * 32 + lane;
  const int q0 = m_ptr[l], q1 = m_ptr[l + 1];
  const int len = (q1 - q0 + kLongSeg - 1) / kLongSeg;
  const int a = q0 + seg * len, b = min(q1, a + len);
  cplx acc = make_double2(0, 0);
  if (s < nsys)
    for (int q = a + warp; q < b; q += 8) {
      const int br = m_col[q];
      if (br >= ncb) continue;
      const cplx v = Vb[(size_t)br * nsys + s];
      acc = m_val[q] > 0 ? cadd(acc, v) : csub(acc, v);
    }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && s < nsys) {
    cplx t = red[0][lane];
    for (int k = 1; k < 8; ++k) t = cadd(t, red[k][lane]);
    part[((size_t)blockIdx.x * kLongSeg + seg) * nsys + s] = t;
  }
}

__global__ void k_loop_reduce_fin(int nloop, int nsys, int nlong, const int32_t* __restrict__ rows,
                                  const cplx* __restrict__ part, cplx* __restrict__ w) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nlong * nsys) return;
  const int r = e / nsys, s = e % nsys;
  cplx t = make_double2(0, 0);
  for (int k = 0; k < kLongSeg; ++k) t = cadd(t, part[((size_t)r * kLongSeg + k) * nsys + s]);
  w[(size_t)s * nloop + rows[r]] = t;
}

// w = Q(f_s) v (mode 0) or diag(Q(f_s)) (mode 1, v unused)
__global__ void k_qspmv(int nloop, int nsys, int nmat, const int32_t* __restrict__ q_ptr,
                        const int32_t* __restrict__ q_col, const double* __restrict__ q_val,
                        const cplx* __restrict__ zs, const double* __restrict__ wp,
                        const cplx* __restrict__ v, cplx* __restrict__ w, int mode) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nloop * nsys) return;
  int s = (int)(idx / nloop), l = (int)(idx % nloop);
  const int W = nmat + 1;
  cplx acc = make_double2(0, 0);
  const cplx* vs = v ? v + (size_t)s * nloop : nullptr;
  for (int q = q_ptr[l]; q < q_ptr[l + 1]; ++q) {
    int col = q_col[q];
    if (mode == 1 && col != l) continue;
    const double* qv = q_val + (size_t)q * W;
    cplx a = make_double2(0.0, wp[s] * qv[nmat]);
    for (int m = 0; m < nmat; ++m) a = cadd(a, cscale(zs[s * nmat + m], qv[m]));
    acc = cadd(acc, mode == 1 ? a : cm(a, vs[col]));
  }
  w[idx] = acc;
}

// ---- block reductions per system --------------------------------------------------------------
__device__ cplx block_sum(cplx v, cplx* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  cplx r = sh[0];
  __syncthreads();
  return r;
}

// out[s] = sum_i op(a_s[i]) b_s[i], op = conj (herm = 1) or identity; one block per system
__global__ void k_dot(int n, int nsys, const cplx* __restrict__ a, const cplx* __restrict__ b, int herm,
                      cplx* __restrict__ out) {
  __shared__ cplx sh[256];
  int s = blockIdx.x;
  const cplx* as = a + (size_t)s * n;
  const cplx* bs = b + (size_t)s * n;
  cplx acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cadd(acc, cm(herm ? cconj(as[i]) : as[i], bs[i]));
  cplx r = block_sum(acc, sh);
  if (threadIdx.x == 0) out[s] = r;
}

// ---- COCG (inner solve of Q z = v) ------------------------------------------------------------
// state per system: rho, alpha, flags
__global__ void k_cocg_init(int n, int nsys, const cplx* __restrict__ v, const cplx* __restrict__ dinv,
                            cplx* __restrict__ z, cplx* __restrict__ r, cplx* __restrict__ p,
                            cplx* __restrict__ rho, double* __restrict__ vnorm2, int* __restrict__ live) {
  __shared__ cplx sh[256];
  int s = blockIdx.x;
  size_t o = (size_t)s * n;
  cplx acc = make_double2(0, 0), nn = make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cplx vi = v[o + i];
    z[o + i] = make_double2(0, 0);
    r[o + i] = vi;
    cplx u = cm(dinv[o + i], vi);
    p[o + i] = u;
    acc = cadd(acc, cm(vi, u));
    nn.x += cabs2(vi);
  }
  cplx a = block_sum(acc, sh);
  cplx b = block_sum(nn, sh);
  if (threadIdx.x == 0) {
    rho[s] = a;
    vnorm2[s] = b.x;
    live[s] = b.x > 0.0 ? 1 : 0;
  }
}

// alpha = rho / p^T q; z += alpha p; r -= alpha q; then rho' = r^T D^-1 r, beta, p = D^-1 r + beta p
__global__ void k_cocg_step(int n, int nsys, const cplx* __restrict__ q, const cplx* __restrict__ dinv,
                            cplx* __restrict__ z, cplx* __restrict__ r, cplx* __restrict__ p,
                            cplx* __restrict__ rho, const double* __restrict__ vnorm2, int* __restrict__ live,
                            double tol2) {
  __shared__ cplx sh[256];
  int s = blockIdx.x;
  if (!live[s]) return;
  size_t o = (size_t)s * n;
  cplx acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cadd(acc, cm(p[o + i], q[o + i]));
  cplx ptq = block_sum(acc, sh);
  if (cabs2(ptq) == 0.0) {
    if (threadIdx.x == 0) live[s] = 0;
    return;
  }
  cplx alpha = cdiv(rho[s], ptq);
  cplx rr = make_double2(0, 0), nn = make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    z[o + i] = cadd(z[o + i], cm(alpha, p[o + i]));
    cplx ri = csub(r[o + i], cm(alpha, q[o + i]));
    r[o + i] = ri;
    rr = cadd(rr, cm(ri, cm(dinv[o + i], ri)));
    nn.x += cabs2(ri);
  }
  cplx rho_new = block_sum(rr, sh);
  cplx rn = block_sum(nn, sh);
  if (rn.x <= tol2 * vnorm2[s] || cabs2(rho[s]) == 0.0) {
    if (threadIdx.x == 0) live[s] = 0;
    return;
  }
  cplx beta = cdiv(rho_new, rho[s]);
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[o + i] = cadd(cm(dinv[o + i], r[o + i]), cm(beta, p[o + i]));
  __syncthreads();
  if (threadIdx.x == 0) rho[s] = rho_new;
}

__global__ void k_inv(size_t n, const cplx* __restrict__ d, cplx* __restrict__ di) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) di[i] = cdiv(make_double2(1.0, 0.0), d[i]);
}

// ---- FGMRES pieces ------------------------------------------------------------------------------
// h[s][i] = v_i^H w for i <= j (block per (i, s)), accumulated into H column j (add = 1) or set
__global__ void k_arnoldi_dots(int n, int nsys, int j, int ldh, const cplx* __restrict__ V,
                               const cplx* __restrict__ w, cplx* __restrict__ h, const int* __restrict__ active) {
  __shared__ cplx sh[256];
  int i = blockIdx.x, s = blockIdx.y;
  if (!active[s]) return;
  const cplx* vi = V + ((size_t)i * nsys + s) * n;
  const cplx* ws = w + (size_t)s * n;
  cplx acc = make_double2(0, 0);
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc = cadd(acc, cm(cconj(vi[e]), ws[e]));
  cplx r = block_sum(acc, sh);
  if (threadIdx.x == 0) h[(size_t)s * ldh + i] = r;
}

// w -= sum_{i<=j} h_i v_i ; also Hcol += h (Hcol = H[s][:, j])
__global__ void k_arnoldi_sub(int n, int nsys, int j, int ldh, const cplx* __restrict__ V,
                              const cplx* __restrict__ h, cplx* __restrict__ w, const int* __restrict__ active) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  int s = (int)(idx / n), e = (int)(idx % n);
  if (!active[s]) return;
  cplx acc = w[idx];
  for (int i = 0; i <= j; ++i) acc = csub(acc, cm(h[(size_t)s * ldh + i], V[((size_t)i * nsys + s) * n + e]));
  w[idx] = acc;
}

// H[s][i][j] += h[s][i] (i <= j), then ||w|| -> H[s][j+1][j]; v_{j+1} = w / ||w||;
// Givens update of the residual estimate; mark converged systems.
// H layout: [s][(m+1)][m] row-major.
__global__ void k_arnoldi_norm(int n, int nsys, int j, int m, cplx* __restrict__ H, const cplx* __restrict__ h1,
                               const cplx* __restrict__ h2, cplx* __restrict__ w, cplx* __restrict__ Vnext,
                               cplx* __restrict__ cs, cplx* __restrict__ sn, cplx* __restrict__ g,
                               int* __restrict__ active, const double* __restrict__ bnorm,
                               const double* __restrict__ thr, double* __restrict__ resid,
                               int* __restrict__ iters) {
  __shared__ cplx sh[256];
  int s = blockIdx.x;
  if (!active[s]) return;
  const int ldh = m + 1;
  cplx* ws = w + (size_t)s * n;
  // eight independent loads in flight per thread: one CTA per system streams
  // the vector, so memory-level parallelism, not bandwidth, sets the time
  constexpr int U = 8;
  double part[U];
#pragma unroll
  for (int u = 0; u < U; ++u) part[u] = 0.0;
  for (int e0 = threadIdx.x; e0 < n; e0 += U * blockDim.x) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n) part[u] += cabs2(ws[e]);
    }
  }
  cplx acc = make_double2(0, 0);
#pragma unroll
  for (int u = 0; u < U; ++u) acc.x += part[u];
  double nw = sqrt(block_sum(acc, sh).x);
  const double inv = nw > 0 ? 1.0 / nw : 0.0;
  cplx* vn = Vnext + (size_t)s * n;
  for (int e0 = threadIdx.x; e0 < n; e0 += U * blockDim.x) {
    cplx v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      v[u] = e < n ? ws[e] : make_double2(0, 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n) vn[e] = cscale(v[u], inv);
    }
  }
  if (threadIdx.x == 0) {
    cplx* Hs = H + (size_t)s * (m + 1) * m;
    for (int i = 0; i <= j; ++i) Hs[i * m + j] = cadd(h1[(size_t)s * ldh + i], h2[(size_t)s * ldh + i]);
    Hs[(j + 1) * m + j] = make_double2(nw, 0.0);
    // apply previous rotations
    for (int i = 0; i < j; ++i) {
      cplx a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
      cplx c = cs[s * m + i], sv = sn[s * m + i];
      Hs[i * m + j] = cadd(cm(cconj(c), a), cm(cconj(sv), b));
      Hs[(i + 1) * m + j] = csub(cm(c, b), cm(sv, a));
    }
    cplx a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
    double na = sqrt(cabs2(a)), nb = sqrt(cabs2(b));
    double den = sqrt(na * na + nb * nb);
    cplx c, sv;
    if (den == 0.0) {
      c = make_double2(1, 0);
      sv = make_double2(0, 0);
    } else {
      c = cscale(a, 1.0 / den);
      sv = cscale(b, 1.0 / den);
    }
    cs[s * m + j] = c;
    sn[s * m + j] = sv;
    Hs[j * m + j] = make_double2(den, 0.0);
    Hs[(j + 1) * m + j] = make_double2(0, 0);
    cplx gj = g[s * (m + 1) + j];
    g[s * (m + 1) + j] = cm(cconj(c), gj);
    g[s * (m + 1) + j + 1] = cscale(cm(sv, gj), -1.0);
    double res = sqrt(cabs2(g[s * (m + 1) + j + 1]));
    resid[s] = res / bnorm[s];
    iters[s] += 1;
    if (res <= thr[s] || nw == 0.0) active[s] = 0;
  }
}

// y = H^-1 g (upper triangular, k x k per system); x += Z y
__global__ void k_trisolve(int nsys, int m, const int* __restrict__ kcols, const cplx* __restrict__ H,
                           const cplx* __restrict__ g, cplx* __restrict__ y) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  int k = kcols[s];
  const cplx* Hs = H + (size_t)s * (m + 1) * m;
  for (int i = k - 1; i >= 0; --i) {
    cplx acc = g[s * (m + 1) + i];
    for (int j = i + 1; j < k; ++j) acc = csub(acc, cm(Hs[i * m + j], y[s * m + j]));
    y[s * m + i] = cdiv(acc, Hs[i * m + i]);
  }
}

__global__ void k_update_x(int n, int nsys, int m, const int* __restrict__ kcols, const cplx* __restrict__ Z,
                           const cplx* __restrict__ y, cplx* __restrict__ x) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  int s = (int)(idx / n), e = (int)(idx % n);
  cplx acc = x[idx];
  for (int i = 0; i < kcols[s]; ++i) acc = cadd(acc, cm(y[s * m + i], Z[((size_t)i * nsys + s) * n + e]));
  x[idx] = acc;
}

__global__ void k_cadd(size_t n, const cplx* __restrict__ z, cplx* __restrict__ x) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) x[idx] = cadd(x[idx], z[idx]);
}

// r = b - Ax ; beta = ||r||; v0 = r / beta; g = (beta, 0, ...)
// thr[s] = max(tol ||b||, tau ||r||): the inner cycle's stopping level (tau > 0 in
// the mixed-precision mode, where the cycle's operator is only FP32-accurate)
__global__ void k_restart(int n, int nsys, int m, const cplx* __restrict__ b, const cplx* __restrict__ Ax,
                          cplx* __restrict__ V0, cplx* __restrict__ g, const double* __restrict__ bnorm,
                          double tol, double tau, int* __restrict__ active, double* __restrict__ resid,
                          double* __restrict__ thr) {
  __shared__ cplx sh[256];
  int s = blockIdx.x;
  size_t o = (size_t)s * n;
  cplx acc = make_double2(0, 0);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    cplx r = Ax ? csub(b[o + e], Ax[o + e]) : b[o + e];
    V0[o + e] = r;
    acc.x += cabs2(r);
  }
  double beta = sqrt(block_sum(acc, sh).x);
  for (int e = threadIdx.x; e < n; e += blockDim.x) V0[o + e] = beta > 0 ? cscale(V0[o + e], 1.0 / beta) : make_double2(0, 0);
  if (threadIdx.x == 0) {
    for (int i = 0; i <= m; ++i) g[s * (m + 1) + i] = make_double2(0, 0);
    g[s * (m + 1)] = make_double2(beta, 0);
    resid[s] = bnorm[s] > 0 ? beta / bnorm[s] : 0.0;
    active[s] = (beta > tol * bnorm[s]) ? 1 : 0;
    thr[s] = fmax(tol * bnorm[s], tau * beta);
  }
}

__global__ void k_bnorm(int n, int nsys, const cplx* __restrict__ b, double* __restrict__ out) {
  __shared__ cplx sh[256];
  int s = blockIdx.x;
  cplx acc = make_double2(0, 0);
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc.x += cabs2(b[(size_t)s * n + e]);
  double v = sqrt(block_sum(acc, sh).x);
  if (threadIdx.x == 0) out[s] = v;
}

// RHS: b_s = column of M for the port branch of system s (sign +1 on its loop)
__global__ void k_rhs(int nloop, int nsys, int nport, const int32_t* __restrict__ port_loop,
                      const int8_t* __restrict__ port_sign, cplx* __restrict__ b) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nloop * nsys) return;
  int s = (int)(idx / nloop), l = (int)(idx % nloop);
  int p = s % nport;
  b[idx] = make_double2(l == port_loop[p] ? (double)port_sign[p] : 0.0, 0.0);
}

// initial-guess shapes [nsys][N caller][6] (FP32) -> FMM columns X[r][6 s + c]
__global__ void k_shape_to_X(int N, int nsys, const int32_t* __restrict__ perm, const float* __restrict__ shape,
                             double* __restrict__ X) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * nsys * 6) return;
  int c = (int)(idx % 6);
  size_t rs = idx / 6;
  int s = (int)(rs % nsys), r = (int)(rs / nsys);
  X[(size_t)r * 6 * nsys + 6 * s + c] = (double)shape[((size_t)s * N + perm[r]) * 6 + c];
}

// alpha_s = (w^H b) / (w^H w) fitted per system; x = alpha x_s and Ax = alpha w
// when that lowers ||b - A x|| by more than 1 %, else x = Ax = 0
__global__ void k_guess_scale(int n, int nsys, const cplx* __restrict__ b, cplx* __restrict__ xs,
                              cplx* __restrict__ w, int* __restrict__ accepted, double* __restrict__ gain) {
  __shared__ cplx sh[256];
  const int s = blockIdx.x;
  const size_t o = (size_t)s * n;
  cplx wb = make_double2(0, 0), ww = make_double2(0, 0), bb = make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cplx wi = w[o + i], bi = b[o + i];
    wb = cadd(wb, cm(cconj(wi), bi));
    ww.x += cabs2(wi);
    bb.x += cabs2(bi);
  }
  wb = block_sum(wb, sh);
  ww = block_sum(ww, sh);
  bb = block_sum(bb, sh);
  const double red = (ww.x > 0.0 && bb.x > 0.0) ? cabs2(wb) / (ww.x * bb.x) : 0.0;   // 1 - |r|^2/|b|^2
  const bool ok = red > 0.01;
  const cplx alpha = ok ? cscale(wb, 1.0 / ww.x) : make_double2(0, 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xs[o + i] = cm(alpha, xs[o + i]);
    w[o + i] = cm(alpha, w[o + i]);
  }
  if (threadIdx.x == 0) {
    accepted[s] = ok ? 1 : 0;
    gain[s] = ok ? sqrt(fmax(0.0, 1.0 - red)) : 1.0;   // ||b - A x0|| / ||b||
  }
}

// Port reduction per frequency: Y[q][p] = b_q^T x_{f,p}; Z = Y^-1; R, L
__global__ void k_ports(int nf, int nport, int nloop, const double* __restrict__ freq,
                        const int32_t* __restrict__ port_loop, const int8_t* __restrict__ port_sign,
                        const cplx* __restrict__ x, double* __restrict__ R, double* __restrict__ L) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  cplx A[16][32];
  const int n = nport;
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) {
      int s = f * nport + p;
      A[q][p] = cscale(x[(size_t)s * nloop + port_loop[q]], (double)port_sign[q]);
      A[q][n + p] = make_double2(q == p ? 1.0 : 0.0, 0.0);
    }
  // Gauss-Jordan with partial pivoting
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (cabs2(A[r][c]) > cabs2(A[piv][c])) piv = r;
    if (piv != c)
      for (int k = 0; k < 2 * n; ++k) {
        cplx t = A[c][k];
        A[c][k] = A[piv][k];
        A[piv][k] = t;
      }
    cplx d = A[c][c];
    for (int k = 0; k < 2 * n; ++k) A[c][k] = cdiv(A[c][k], d);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      cplx fct = A[r][c];
      for (int k = 0; k < 2 * n; ++k) A[r][k] = csub(A[r][k], cm(fct, A[c][k]));
    }
  }
  double w = 2.0 * 3.14159265358979323846 * freq[f];
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) {
      cplx z = A[q][n + p];
      R[((size_t)f * n + q) * n + p] = z.x;
      L[((size_t)f * n + q) * n + p] = z.y / w;
    }
}

// ---- host side ---------------------------------------------------------------------------
struct SolverState {
  int nsys = 0, nloop = 0, m = 0;
  DBuf<double> freq, wp;
  DBuf<cplx> zs;
};

void solver_prepare(xrl_ctx* c) {
  Topo& T = c->topo;
  Tree& tr = c->tree;
  const int N = c->N;
  std::vector<int32_t> pan_br(kPanEdges * (size_t)N, -1), pan_mat(N, -1), br_pan(2 * (size_t)T.n_cb, -1);
  std::vector<double> pan_rho(3 * kPanEdges * (size_t)N, 0.0), br_rho(6 * (size_t)T.n_cb, 0.0);
  std::vector<int> slot(N, 0);
  for (int b = 0; b < T.n_cb; ++b)
    for (int side = 0; side < 2; ++side) {
      int p = T.br_pan[side][b];
      if (p < 0) continue;
      int r = tr.rank[p];
      int k = slot[p]++;
      XRL_CHECK(k < kPanEdges, XRL_ETOPO, "internal: a panel has more branches than edges");
      pan_br[kPanEdges * (size_t)r + k] = b;
      br_pan[2 * (size_t)b + side] = r;
      for (int t = 0; t < 3; ++t) {
        double v = T.br_rho[side][3 * (size_t)b + t];
        pan_rho[3 * kPanEdges * (size_t)r + 3 * k + t] = v;
        br_rho[6 * (size_t)b + 3 * side + t] = v;
      }
    }
  for (int p = 0; p < N; ++p)
    if (T.live_of_panel[p] >= 0) pan_mat[tr.rank[p]] = T.mat_of_cond[c->cond[p]];
  c->d.pan_br.upload(c->alloc, pan_br);
  c->d.pan_rho.upload(c->alloc, pan_rho);
  c->d.pan_mat.upload(c->alloc, pan_mat);
  c->d.br_pan.upload(c->alloc, br_pan);
  c->d.br_rho.upload(c->alloc, br_rho);
  auto to32 = [](const std::vector<int64_t>& a) { return std::vector<int32_t>(a.begin(), a.end()); };
  XRL_CHECK(T.m_col.size() < (size_t)INT32_MAX && T.q_col.size() < (size_t)INT32_MAX, XRL_ENOMEM,
            "loop or preconditioner matrix too large for 32-bit indices");
  c->d.m_ptr.upload(c->alloc, to32(T.m_ptr));
  {
    std::vector<int32_t> longr;
    for (int l = 0; l < T.n_loops; ++l)
      if (T.m_ptr[l + 1] - T.m_ptr[l] > kLongRow) longr.push_back(l);
    c->d.m_long.upload(c->alloc, longr);
  }
  c->d.m_col.upload(c->alloc, T.m_col);
  c->d.m_val.upload(c->alloc, T.m_val);
  c->d.mt_ptr.upload(c->alloc, to32(T.mt_ptr));
  c->d.mt_col.upload(c->alloc, T.mt_col);
  c->d.mt_val.upload(c->alloc, T.mt_val);
  c->d.q_ptr.upload(c->alloc, to32(T.q_ptr));
  c->d.q_col.upload(c->alloc, T.q_col);
  c->d.q_val.upload(c->alloc, T.q_val);
  c->d.mat_sigma.upload(c->alloc, T.mat_sigma);
  c->d.mat_thick.upload(c->alloc, T.mat_thick);
}

static unsigned nblk(size_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

// w = M Vb for nsys systems (loop rows short and long); returns the launches
static int loop_reduce(xrl_ctx* c, int nsys, const cplx* Vb, cplx* w, cudaStream_t s) {
  const Topo& T = c->topo;
  const int sg = (nsys + 31) / 32;
  k_loop_reduce<<<nblk((size_t)T.n_loops * sg * 32), 256, 0, s>>>(T.n_loops, nsys, T.n_cb, c->d.m_ptr.p,
                                                                  c->d.m_col.p, c->d.m_val.p, Vb, w);
  const int nlong = (int)c->d.m_long.n;
  if (nlong == 0) return 1;
  c->d.m_long_part.ensure(c->alloc, (size_t)nlong * kLongSeg * nsys);
  k_loop_reduce_long<<<dim3(nlong, kLongSeg, sg), 256, 0, s>>>(nsys, T.n_cb, c->d.m_long.p, c->d.m_ptr.p,
                                                               c->d.m_col.p, c->d.m_val.p, Vb, c->d.m_long_part.p);
  k_loop_reduce_fin<<<nblk((size_t)nlong * nsys), 256, 0, s>>>(T.n_loops, nsys, nlong, c->d.m_long.p,
                                                              c->d.m_long_part.p, w);
  return 3;
}

// Work arrays of one solve (device)
struct Work {
  DBuf<double> freq, wp, wpf;
  DBuf<cplx> zs, zsf;
  BandWork bw;
  AmgWork aw;
  int nport = 1;
  bool banded = false, use_amg = false;
  DBuf<cplx> b, x, w, tmp, V, Z, H, h1, h2, cs, sn, g, y, Vb, dinv, zst;
  DBuf<cplx> cz, cr, cp, cq, crho;
  DBuf<double> X, Y, bnorm, resid, cvn, thr;
  DBuf<float> X32, Y32;
  DBuf<int> active, iters, kcols, clive;
};

static void sys_consts(xrl_ctx* c, Work& wk, int nsys, int nport, int nf, const double* freq) {
  const Topo& T = c->topo;
  wk.nport = nport;
  wk.freq.upload(c->alloc, std::vector<double>(freq, freq + nf));
  wk.zs.alloc(c->alloc, (size_t)nsys * T.n_mat);
  wk.wp.alloc(c->alloc, nsys);
  k_sys_consts<<<nblk((size_t)nsys * T.n_mat), 256, 0, c->stream>>>(nsys, nport, T.n_mat, wk.freq.p,
                                                                    c->d.mat_sigma.p, c->d.mat_thick.p, wk.zs.p,
                                                                    wk.wp.p);
  // per-frequency copies (one "system" per frequency) for the preconditioner factors
  wk.zsf.alloc(c->alloc, (size_t)nf * T.n_mat);
  wk.wpf.alloc(c->alloc, nf);
  k_sys_consts<<<nblk((size_t)nf * T.n_mat), 256, 0, c->stream>>>(nf, 1, T.n_mat, wk.freq.p, c->d.mat_sigma.p,
                                                                  c->d.mat_thick.p, wk.zsf.p, wk.wpf.p);
  count_launch(c, 2);
}

// w = Z(f_s) v_s for all systems (eq. 8); the FMM runs in FP64, or in FP32
// for the inner iterations of the mixed-precision mode (low = true)
template <class T>
static void apply_A_t(xrl_ctx* c, Work& wk, int nsys, const cplx* v, cplx* w, T* X, T* Y, bool loop_major) {
  const Topo& T_ = c->topo;
  const int N = c->N;
  const int nc = 6 * nsys;
  cudaStream_t s = c->stream;
  wk.Vb.ensure(c->alloc, (size_t)nsys * T_.n_cb);
  cudaEvent_t ev = prof_begin(c, s);
  k_gather<T><<<nblk((size_t)N * nsys), 256, 0, s>>>(N, nsys, T_.n_loops, c->d.pan_br.p, c->d.pan_rho.p,
                                                     c->d.mt_ptr.p, c->d.mt_col.p, c->d.mt_val.p, v, X,
                                                     loop_major ? 1 : 0);
  const double nnzm = (double)T_.m_col.size();
  prof_end(c, s, ev, PH_OPER, 1, 8.0 * nnzm * nsys + 18.0 * N * nsys, nsys * (16.0 * nnzm + 6.0 * sizeof(T) * N));
  if (sizeof(T) == 8)
    fmm_apply(c, nc, (const double*)X, (double*)Y, s);
  else
    fmm_apply32(c, nc, (const float*)X, (float*)Y, s);
  ev = prof_begin(c, s);
  // conductor branches only; the external port branches carry no impedance
  k_scatter<T><<<nblk((size_t)T_.n_cb * nsys), 256, 0, s>>>(T_.n_cb, nsys, T_.n_mat, c->d.br_pan.p, c->d.br_rho.p,
                                                            c->d.pan_mat.p, c->d.area.p, wk.zs.p, wk.wp.p, X, Y,
                                                            wk.Vb.p);
  const int nlr = loop_reduce(c, nsys, wk.Vb.p, w, s);
  prof_end(c, s, ev, PH_OPER, 1 + nlr, nsys * (2.0 * T_.n_cb * 30.0 + 2.0 * nnzm),
           nsys * (T_.n_cb * (2.0 * 12.0 * sizeof(T) + 16.0) + 16.0 * nnzm + 16.0 * T_.n_loops));
  XRL_CUDA(cudaGetLastError());
  c->stats.n_mvm++;
}

// v is [nsys][n_loops], or [n_loops][nsys] with loop_major; w always [nsys][n_loops]
static void apply_A(xrl_ctx* c, Work& wk, int nsys, const cplx* v, cplx* w, bool low = false,
                    bool loop_major = false) {
  const size_t n = (size_t)c->N * 6 * nsys;
  if (low) {
    wk.X32.ensure(c->alloc, n);
    wk.Y32.ensure(c->alloc, n);
    apply_A_t<float>(c, wk, nsys, v, w, wk.X32.p, wk.Y32.p, loop_major);
  } else {
    wk.X.ensure(c->alloc, n);
    wk.Y.ensure(c->alloc, n);
    apply_A_t<double>(c, wk, nsys, v, w, wk.X.p, wk.Y.p, loop_major);
  }
}

static void apply_Qmat(xrl_ctx* c, Work& wk, int nsys, const cplx* v, cplx* w, int mode) {
  const Topo& T = c->topo;
  cudaEvent_t ev = prof_begin(c, c->stream);
  k_qspmv<<<nblk((size_t)T.n_loops * nsys), 256, 0, c->stream>>>(T.n_loops, nsys, T.n_mat, c->d.q_ptr.p,
                                                                  c->d.q_col.p, c->d.q_val.p, wk.zs.p, wk.wp.p, v,
                                                                  w, mode);
  const double nnzq = (double)T.q_col.size();
  prof_end(c, c->stream, ev, PH_PREC, 1, nsys * nnzq * (8.0 + 4.0 * T.n_mat),
           nnzq * (4.0 + 8.0 * (T.n_mat + 1)) + nsys * 32.0 * T.n_loops);
  XRL_CUDA(cudaGetLastError());
}

// z ~= Q^-1 v by Jacobi-COCG with a fixed budget (or z = v without preconditioner)
static void apply_Qinv(xrl_ctx* c, Work& wk, int nsys, const cplx* v, cplx* z, bool all = false) {
  const int n = c->topo.n_loops;
  cudaStream_t s = c->stream;
  if (c->opt.precond == 0) {
    XRL_CUDA(cudaMemcpyAsync(z, v, sizeof(cplx) * (size_t)n * nsys, cudaMemcpyDeviceToDevice, s));
    return;
  }
  if (wk.banded) {
    band_apply(c, wk.bw, nsys, wk.nport, wk.zsf.p, wk.wpf.p, v, z, all ? nullptr : wk.active.p, s);
    return;
  }
  if (wk.use_amg) {
    cudaEvent_t ev = prof_begin(c, s);
    amg_apply(c, wk.aw, nsys, wk.nport, v, z, s);
    prof_end(c, s, ev, PH_PREC, 0, 0.0, 0.0);
    return;
  }
  const size_t tot = (size_t)n * nsys;
  wk.cr.ensure(c->alloc, tot);
  wk.cp.ensure(c->alloc, tot);
  wk.cq.ensure(c->alloc, tot);
  wk.crho.ensure(c->alloc, nsys);
  wk.cvn.ensure(c->alloc, nsys);
  wk.clive.ensure(c->alloc, nsys);
  cudaEvent_t ev = prof_begin(c, s);
  k_cocg_init<<<nsys, 256, 0, s>>>(n, nsys, v, wk.dinv.p, z, wk.cr.p, wk.cp.p, wk.crho.p, wk.cvn.p, wk.clive.p);
  prof_end(c, s, ev, PH_PREC, 1, 16.0 * tot, 80.0 * tot);
  const double tol2 = c->opt.inner_tol * c->opt.inner_tol;
  for (int it = 0; it < c->opt.inner_iters; ++it) {
    apply_Qmat(c, wk, nsys, wk.cp.p, wk.cq.p, 0);
    ev = prof_begin(c, s);
    k_cocg_step<<<nsys, 256, 0, s>>>(n, nsys, wk.cq.p, wk.dinv.p, z, wk.cr.p, wk.cp.p, wk.crho.p, wk.cvn.p,
                                     wk.clive.p, tol2);
    prof_end(c, s, ev, PH_PREC, 1, 40.0 * tot, 16.0 * 9.0 * tot);
  }
  XRL_CUDA(cudaGetLastError());
  c->stats.total_inner += c->opt.inner_iters;
}

// x0[f * nport + p] = prev[(nf_prev - 1) * nport + p]: every frequency of a chunk
// starts from the last frequency of the previous chunk (same port)
__global__ void k_seed_from_prev(int n, int nsys, int nport, int last0, const cplx* __restrict__ prev,
                                 cplx* __restrict__ x) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nsys) return;
  const int s = (int)(idx / n), e = (int)(idx % n);
  x[idx] = prev[(size_t)(last0 + s % nport) * n + e];
}

void run_solve(xrl_ctx* c, int nf, const double* freq, double* R, double* L, const float* shape, int* accepted,
               double* guess_res, bool from_prev) {
  const Topo& T = c->topo;
  const int np = T.n_port;
  XRL_CHECK(np > 0, XRL_ESTATE, "no ports defined");
  XRL_CHECK(np <= 16, XRL_EINVAL, "at most 16 ports per context");
  const int nsys = nf * np;
  const int n = T.n_loops;
  const int m = std::max(1, std::min(c->opt.restart, 200));
  const size_t tot = (size_t)n * nsys;
  cudaStream_t s = c->stream;
  Work wk;
  sys_consts(c, wk, nsys, np, nf, freq);
  // port loops: the loop containing each port branch (global loops are listed last)
  std::vector<int32_t> port_loop(np, -1);
  std::vector<int8_t> port_sign(np, 0);
  for (int p = 0; p < np; ++p) {
    int b = T.n_cb + p;
    XRL_CHECK(T.mt_ptr[b + 1] - T.mt_ptr[b] == 1, XRL_ETOPO, "internal: a port branch must lie in one loop");
    port_loop[p] = T.mt_col[T.mt_ptr[b]];
    port_sign[p] = T.mt_val[T.mt_ptr[b]];
  }
  DBuf<int32_t> dpl;
  DBuf<int8_t> dps;
  dpl.upload(c->alloc, port_loop);
  dps.upload(c->alloc, port_sign);
  wk.b.alloc(c->alloc, tot);
  wk.x.alloc(c->alloc, tot);
  wk.w.alloc(c->alloc, tot);
  wk.V.alloc(c->alloc, tot * (m + 1));
  // With a fixed preconditioner (all but the inner COCG iteration) the
  // flexible variant's Z_j = M^-1 v_j need not be kept: the cycle ends with
  // x += M^-1 (V y), one more preconditioner application, and Z is one
  // scratch vector instead of m (half the Krylov memory).
  const bool zfree = c->opt.precond != 2;
  wk.Z.alloc(c->alloc, zfree ? tot : tot * m);
  wk.H.alloc(c->alloc, (size_t)nsys * (m + 1) * m);
  wk.h1.alloc(c->alloc, (size_t)nsys * (m + 1));
  wk.h2.alloc(c->alloc, (size_t)nsys * (m + 1));
  wk.cs.alloc(c->alloc, (size_t)nsys * m);
  wk.sn.alloc(c->alloc, (size_t)nsys * m);
  wk.g.alloc(c->alloc, (size_t)nsys * (m + 1));
  wk.y.alloc(c->alloc, (size_t)nsys * m);
  wk.bnorm.alloc(c->alloc, nsys);
  wk.thr.alloc(c->alloc, nsys);
  const bool mixed = c->opt.precision == 1;
  const double tau = mixed ? 1e-5 : 0.0;
  // FP64-accurate products on the tensor cores (integer slices) and FP32 pipes
  // (double-float): the refinement residuals of the mixed mode, and every
  // product of precision 2
  struct Df64Guard {
    xrl_ctx* c;
    bool old;
    ~Df64Guard() { c->df64_m2l = old; }
  } df64_guard{c, c->df64_m2l};
  c->df64_m2l = c->opt.precision >= 1;
  wk.resid.alloc(c->alloc, nsys);
  wk.active.alloc(c->alloc, nsys);
  wk.iters.alloc(c->alloc, nsys);
  wk.kcols.alloc(c->alloc, nsys);
  wk.banded = (c->opt.precond == 1 || c->opt.precond == 3) && band_usable(c);
  wk.use_amg = !wk.banded && c->opt.precond != 0 && c->opt.precond != 2 && c->amg.ready;
  if (wk.banded) {
    band_alloc(c, wk.bw, nf, nsys, mixed);
    band_factor(c, wk.bw, wk.zsf.p, wk.wpf.p, s);
  } else if (wk.use_amg) {
    amg_factor(c, wk.aw, nf, nsys, wk.zsf.p, wk.wpf.p, s);
    amg_check(c, wk.aw, s);
  } else if (c->opt.precond) {
    wk.dinv.alloc(c->alloc, tot);
    apply_Qmat(c, wk, nsys, nullptr, wk.w.p, 1);
    k_inv<<<nblk(tot), 256, 0, s>>>(tot, wk.w.p, wk.dinv.p);
    count_launch(c);
  }
  k_rhs<<<nblk(tot), 256, 0, s>>>(n, nsys, np, dpl.p, dps.p, wk.b.p);
  count_launch(c, 2);
  XRL_CUDA(cudaMemsetAsync(wk.x.p, 0, sizeof(cplx) * tot, s));
  XRL_CUDA(cudaMemsetAsync(wk.iters.p, 0, sizeof(int) * nsys, s));
  k_bnorm<<<nsys, 256, 0, s>>>(n, nsys, wk.b.p, wk.bnorm.p);
  c->stats.n_mvm = 0;
  c->stats.total_inner = 0;
  bool have_guess = false;
  if (shape) {
    // learned initial guess: project the predicted panel currents onto loop space
    // by weighted least squares, min sum_l |I_p(l) - I^(l)|^2 / A_l, i.e.
    // (sum_m QA_m) x = M A diag(1/A) I^ -- the pencil at Z_s = 1, no P part --
    // then fit one complex scale per system against the FP64 residual
    XRL_CHECK(wk.banded, XRL_EINVAL, "the learned initial guess needs the banded preconditioner");
    const Topo& TT = c->topo;
    const int N = c->N;
    wk.X.ensure(c->alloc, (size_t)N * 6 * nsys);
    k_shape_to_X<<<nblk((size_t)N * nsys * 6), 256, 0, s>>>(N, nsys, c->d.perm.p, shape, wk.X.p);
    std::vector<cplx> ones((size_t)nsys * TT.n_mat, make_double2(1.0, 0.0));
    DBuf<cplx> zs1;
    DBuf<double> wp0;
    zs1.upload(c->alloc, ones);
    wp0.upload(c->alloc, std::vector<double>(nsys, 0.0));
    wk.Vb.ensure(c->alloc, (size_t)nsys * TT.n_cb);
    k_scatter<double><<<nblk((size_t)TT.n_cb * nsys), 256, 0, s>>>(TT.n_cb, nsys, TT.n_mat, c->d.br_pan.p,
                                                                   c->d.br_rho.p, c->d.pan_mat.p, c->d.area.p, zs1.p,
                                                                   wp0.p, wk.X.p, wk.X.p, wk.Vb.p);
    count_launch(c, loop_reduce(c, nsys, wk.Vb.p, wk.w.p, s) - 1);
    BandWork pw;
    band_alloc(c, pw, 1, nsys, false);
    band_factor(c, pw, zs1.p, wp0.p, s);
    band_apply(c, pw, nsys, nsys, zs1.p, wp0.p, wk.w.p, wk.x.p, nullptr, s);
    count_launch(c, 3);
    apply_A(c, wk, nsys, wk.x.p, wk.w.p);
    DBuf<int> dacc;
    DBuf<double> dgain;
    dacc.alloc(c->alloc, nsys);
    dgain.alloc(c->alloc, nsys);
    k_guess_scale<<<nsys, 256, 0, s>>>(n, nsys, wk.b.p, wk.x.p, wk.w.p, dacc.p, dgain.p);
    count_launch(c);
    if (accepted) XRL_CUDA(cudaMemcpyAsync(accepted, dacc.p, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s));
    if (guess_res) XRL_CUDA(cudaMemcpyAsync(guess_res, dgain.p, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s));
    XRL_CUDA(cudaStreamSynchronize(s));
    have_guess = true;
  } else if (from_prev && c->last_nsys > 0 && c->last_nport == np && c->d.last_x.n >= (size_t)c->last_nsys * n) {
    // previous-frequency start: the last frequency's solutions of the previous
    // block, scaled per system by the complex factor that minimises the FP64
    // residual, kept only where that lowers ||b - A x0|| by more than 1 %
    k_seed_from_prev<<<nblk(tot), 256, 0, s>>>(n, nsys, np, c->last_nsys - np, c->d.last_x.p, wk.x.p);
    count_launch(c);
    apply_A(c, wk, nsys, wk.x.p, wk.w.p);
    DBuf<int> dacc;
    DBuf<double> dgain;
    dacc.alloc(c->alloc, nsys);
    dgain.alloc(c->alloc, nsys);
    k_guess_scale<<<nsys, 256, 0, s>>>(n, nsys, wk.b.p, wk.x.p, wk.w.p, dacc.p, dgain.p);
    count_launch(c);
    have_guess = true;
  }
  // The inner operator (gather -> FMM -> scatter -> loop reduce, ~14 kernels)
  // is captured once into a CUDA graph and replayed for every later Arnoldi
  // step; its input is staged through a fixed buffer.  The first application
  // runs eagerly so that every buffer exists before the capture.
  const bool use_graph = c->opt.use_graphs != 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_state = 0;
  struct GraphGuard {
    xrl_ctx* c;
    cudaStream_t s;
    cudaGraph_t* g;
    cudaGraphExec_t* e;
    ~GraphGuard() {
      if (c->prof.capturing) {   // an error inside the capture: close it
        cudaGraph_t partial = nullptr;
        cudaStreamEndCapture(s, &partial);
        if (partial) cudaGraphDestroy(partial);
        cudaGetLastError();
        c->prof.capturing = false;
      }
      if (*e) cudaGraphExecDestroy(*e);
      if (*g) cudaGraphDestroy(*g);
      prof_graph_release(c);
    }
  } graph_guard{c, s, &graph, &gexec};
  if (use_graph) wk.zst.alloc(c->alloc, tot);
  std::vector<int> hact(nsys), hiters(nsys);
  const double tol = c->opt.tol;
  int total = 0;
  bool first = true;
  bool done = false;
  while (!done) {
    // restart: true residual with the FP64 operator
    if (!first) apply_A(c, wk, nsys, wk.x.p, wk.w.p);
    k_restart<<<nsys, 256, 0, s>>>(n, nsys, m, wk.b.p, (first && !have_guess) ? nullptr : wk.w.p, wk.V.p, wk.g.p,
                                   wk.bnorm.p, tol, tau, wk.active.p, wk.resid.p, wk.thr.p);
    count_launch(c);
    first = false;
    XRL_CUDA(cudaMemcpyAsync(hact.data(), wk.active.p, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s));
    XRL_CUDA(cudaStreamSynchronize(s));
    int nact = 0;
    for (int v : hact) nact += v;
    if (nact == 0 || total >= c->opt.max_iters) break;
    // kcols counts the Arnoldi columns each system has built in this cycle
    XRL_CUDA(cudaMemsetAsync(wk.kcols.p, 0, sizeof(int) * nsys, s));
    std::vector<int> hk(nsys, 0);
    int j = 0;
    for (; j < m && total < c->opt.max_iters; ++j, ++total) {
      cplx* vj = wk.V.p + (size_t)j * tot;
      cplx* zj = wk.Z.p + (zfree ? (size_t)0 : (size_t)j * tot);
      apply_Qinv(c, wk, nsys, vj, zj);
      bool replayed = false;
      if (!use_graph) {
        apply_A(c, wk, nsys, zj, wk.w.p, mixed);
      } else {
        // staged loop-major, so that the gather reads one contiguous row per loop
        k_to_loop_major<<<dim3((n + 31) / 32, (nsys + 31) / 32), dim3(32, 8), 0, s>>>(n, nsys, zj, wk.zst.p);
        count_launch(c);
        if (graph_state == 0) {
          apply_A(c, wk, nsys, wk.zst.p, wk.w.p, mixed, true);
          XRL_CUDA(cudaGetLastError());   // a bad launch shows here, not as an invalidated capture
          graph_state = 1;
        } else {
          if (graph_state == 1) {
            c->prof.capturing = true;
            XRL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            apply_A(c, wk, nsys, wk.zst.p, wk.w.p, mixed, true);
            XRL_CUDA(cudaStreamEndCapture(s, &graph));
            c->prof.capturing = false;
            XRL_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
            graph_state = 2;
          } else {
            c->stats.n_mvm++;
          }
          XRL_CUDA(cudaGraphLaunch(gexec, s));
          replayed = true;
        }
      }
      // CGS2
      cudaEvent_t evk = prof_begin(c, s);
      k_arnoldi_dots<<<dim3(j + 1, nsys), 256, 0, s>>>(n, nsys, j, m + 1, wk.V.p, wk.w.p, wk.h1.p, wk.active.p);
      k_arnoldi_sub<<<nblk(tot), 256, 0, s>>>(n, nsys, j, m + 1, wk.V.p, wk.h1.p, wk.w.p, wk.active.p);
      k_arnoldi_dots<<<dim3(j + 1, nsys), 256, 0, s>>>(n, nsys, j, m + 1, wk.V.p, wk.w.p, wk.h2.p, wk.active.p);
      k_arnoldi_sub<<<nblk(tot), 256, 0, s>>>(n, nsys, j, m + 1, wk.V.p, wk.h2.p, wk.w.p, wk.active.p);
      // record which systems take this column before they may deactivate
      for (int q = 0; q < nsys; ++q)
        if (hact[q]) hk[q] = j + 1;
      k_arnoldi_norm<<<nsys, 256, 0, s>>>(n, nsys, j, m, wk.H.p, wk.h1.p, wk.h2.p, wk.w.p,
                                          wk.V.p + (size_t)(j + 1) * tot, wk.cs.p, wk.sn.p, wk.g.p, wk.active.p,
                                          wk.bnorm.p, wk.thr.p, wk.resid.p, wk.iters.p);
      prof_end(c, s, evk, PH_KRYLOV, 5, 4.0 * 8.0 * (j + 1) * tot + 10.0 * tot,
               16.0 * (4.0 * (j + 1) * tot + 4.0 * tot));
      XRL_CUDA(cudaGetLastError());
      XRL_CUDA(cudaMemcpyAsync(hact.data(), wk.active.p, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s));
      XRL_CUDA(cudaStreamSynchronize(s));
      if (replayed) prof_graph_replayed(c);
      nact = 0;
      for (int v : hact) nact += v;
      if (nact == 0) {
        ++total;
        ++j;
        break;
      }
    }
    XRL_CUDA(cudaMemcpyAsync(wk.kcols.p, hk.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
    cudaEvent_t evu = prof_begin(c, s);
    k_trisolve<<<nblk(nsys, 64), 64, 0, s>>>(nsys, m, wk.kcols.p, wk.H.p, wk.g.p, wk.y.p);
    if (zfree) {
      // w = V y (w is free at the end of a cycle), z = M^-1 w, x += z
      XRL_CUDA(cudaMemsetAsync(wk.w.p, 0, sizeof(cplx) * tot, s));
      k_update_x<<<nblk(tot), 256, 0, s>>>(n, nsys, m, wk.kcols.p, wk.V.p, wk.y.p, wk.w.p);
      prof_end(c, s, evu, PH_KRYLOV, 2, 8.0 * j * tot, 16.0 * (j + 2) * tot);
      apply_Qinv(c, wk, nsys, wk.w.p, wk.Z.p, true);
      cudaEvent_t eva = prof_begin(c, s);
      k_cadd<<<nblk(tot), 256, 0, s>>>(tot, wk.Z.p, wk.x.p);
      prof_end(c, s, eva, PH_KRYLOV, 1, 2.0 * tot, 48.0 * tot);
    } else {
      k_update_x<<<nblk(tot), 256, 0, s>>>(n, nsys, m, wk.kcols.p, wk.Z.p, wk.y.p, wk.x.p);
      prof_end(c, s, evu, PH_KRYLOV, 2, 8.0 * j * tot, 16.0 * (j + 2) * tot);
    }
    XRL_CUDA(cudaGetLastError());
    if (total >= c->opt.max_iters) {
      // final true residual for the stats
      apply_A(c, wk, nsys, wk.x.p, wk.w.p);
      k_restart<<<nsys, 256, 0, s>>>(n, nsys, m, wk.b.p, wk.w.p, wk.V.p, wk.g.p, wk.bnorm.p, tol, tau,
                                     wk.active.p, wk.resid.p, wk.thr.p);
      done = true;
    }
  }
  // keep the solution for xrl_get_panel_currents
  c->d.last_x.ensure(c->alloc, tot);
  XRL_CUDA(cudaMemcpyAsync(c->d.last_x.p, wk.x.p, sizeof(cplx) * tot, cudaMemcpyDeviceToDevice, s));
  c->last_nsys = nsys;
  c->last_nport = np;
  c->last_port_loop = port_loop;
  // outputs
  DBuf<double> dR, dL;
  dR.alloc(c->alloc, (size_t)nf * np * np);
  dL.alloc(c->alloc, (size_t)nf * np * np);
  k_ports<<<nblk(nf, 64), 64, 0, s>>>(nf, np, n, wk.freq.p, dpl.p, dps.p, wk.x.p, dR.p, dL.p);
  count_launch(c);
  XRL_CUDA(cudaGetLastError());
  std::vector<double> hres(nsys);
  XRL_CUDA(cudaMemcpyAsync(hres.data(), wk.resid.p, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaMemcpyAsync(hiters.data(), wk.iters.p, sizeof(int) * nsys, cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaMemcpyAsync(R, dR.p, sizeof(double) * nf * np * np, cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaMemcpyAsync(L, dL.p, sizeof(double) * nf * np * np, cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaStreamSynchronize(s));
  tc_check(c, s);
  double mr = 0;
  int mi = 0;
  for (int q = 0; q < nsys; ++q) {
    mr = std::max(mr, hres[q]);
    mi = std::max(mi, hiters[q]);
  }
  c->stats.max_rel_res = mr;
  c->stats.total_iters = mi;
  XRL_CHECK(mr <= tol * 1.0000001, XRL_ENOCONV, "FGMRES did not reach the tolerance in max_iters");
}

// mode 0: w = Z(f) v (eq. 8); 1: w = Q(f) v (eq. 10); 2: w = Q(f)^-1 v (banded factors)
void apply_operator_host(xrl_ctx* c, int nsys, const double* freq, const double* v, double* w, int mode) {
  const Topo& T = c->topo;
  const size_t tot = (size_t)T.n_loops * nsys;
  // the operator of the solver's FP64 residuals: double-float on the FP32
  // pipes in the mixed mode, as inside run_solve
  struct Df64Guard {
    xrl_ctx* c;
    bool old;
    ~Df64Guard() { c->df64_m2l = old; }
  } df64_guard{c, c->df64_m2l};
  c->df64_m2l = c->opt.precision >= 1;
  Work wk;
  // one port per "system": each system is its own frequency here
  sys_consts(c, wk, nsys, 1, nsys, freq);
  DBuf<cplx> dv, dw;
  dv.alloc(c->alloc, tot);
  dw.alloc(c->alloc, tot);
  XRL_CUDA(cudaMemcpyAsync(dv.p, v, sizeof(cplx) * tot, cudaMemcpyHostToDevice, c->stream));
  if (mode == 1) {
    apply_Qmat(c, wk, nsys, dv.p, dw.p, 0);
  } else if (mode == 2) {
    band_alloc(c, wk.bw, nsys, nsys, false);
    band_factor(c, wk.bw, wk.zsf.p, wk.wpf.p, c->stream);
    band_apply(c, wk.bw, nsys, 1, wk.zsf.p, wk.wpf.p, dv.p, dw.p, nullptr, c->stream);
  } else {
    apply_A(c, wk, nsys, dv.p, dw.p);
  }
  XRL_CUDA(cudaMemcpyAsync(w, dw.p, sizeof(cplx) * tot, cudaMemcpyDeviceToHost, c->stream));
  XRL_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace xrl
