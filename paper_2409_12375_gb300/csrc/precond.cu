// Exact application of the diagonal-of-P preconditioner Q(f) (eq. 10) by a
// banded complex-symmetric LDL^T factorisation with a dense Schur border.
//
// The paper applies Q^-1 through a sparse LU (MKL Pardiso, Sec. II-D).  Here
// the vertex loops, put in reverse Cuthill-McKee order at setup, make Q_vv a
// band matrix of half-width b (a vertex loop couples only to the loops of the
// neighbouring vertices); the few global loops (homology and ports) border it:
//   Q = [Q_vv  Q_vg; Q_vg^T  Q_gg],  S = Q_gg - Q_vg^T Q_vv^-1 Q_vg.
// Q(f) = sum_m Z_s^m(f) QA_m + j omega mu0/4pi QP is complex symmetric with
// positive definite real and imaginary parts, so LDL^T (transpose, not
// conjugate transpose) without pivoting is stable (Higham, 1998).
//  * factor: one CTA per frequency, right-looking over the band with the
//    active (b+1) x (b+1) window in shared memory as a ring of rows;
//  * apply: one warp per system, forward and backward substitution with the
//    warp's lanes spanning the band, then the border correction.
#include <vector>

#include "cplx.cuh"
#include "xrl_internal.hpp"

namespace xrl {

constexpr int kMaxBand = 63;     // window (b+1)^2 complex in shared memory
constexpr int kMaxBorder = 16;

// fac[f][i][k]: k < b strictly lower L (column i - b + k), k = b the diagonal D
__global__ void k_band_factor(int n, int b, int nmat, const double* __restrict__ band_val,
                              const cplx* __restrict__ zs, const double* __restrict__ wp_f, cplx* __restrict__ fac) {
  extern __shared__ cplx win[];    // [(b+1)][(b+1)]
  const int f = blockIdx.x;
  const int nb1 = b + 1;
  const size_t stride = (size_t)n * nb1;
  const cplx* z = zs + (size_t)f * nmat;
  const double wp = wp_f[f];
  cplx* out = fac + (size_t)f * stride;
  // load rows 0..b
  for (int e = threadIdx.x; e < nb1 * nb1; e += blockDim.x) {
    int r = e / nb1, k = e % nb1;
    win[r * nb1 + k] = r < n ? pencil(band_val + (size_t)r * nb1 + k, stride, nmat, z, wp) : make_double2(0, 0);
  }
  __syncthreads();
  const int npair = b * (b + 1) / 2;
  for (int k = 0; k < n; ++k) {
    const int sk = k % nb1;
    const cplx Dk = win[sk * nb1 + b];
    for (int t = threadIdx.x; t < b; t += blockDim.x) {
      int i = k + 1 + t;
      if (i < n) {
        int si = i % nb1;
        win[si * nb1 + (b - 1 - t)] = cdiv(win[si * nb1 + (b - 1 - t)], Dk);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < npair; q += blockDim.x) {
      // pair (ti, tj), 0 <= tj <= ti < b
      int ti = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
      while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
      while (ti * (ti + 1) / 2 > q) --ti;
      int tj = q - ti * (ti + 1) / 2;
      int i = k + 1 + ti, j = k + 1 + tj;
      if (i < n) {
        int si = i % nb1, sj = j % nb1;
        cplx lik = win[si * nb1 + (b - 1 - ti)];
        cplx ljk = win[sj * nb1 + (b - 1 - tj)];
        int idx = j - i + b;
        win[si * nb1 + idx] = csub(win[si * nb1 + idx], cm(cm(lik, Dk), ljk));
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb1; e += blockDim.x) out[(size_t)k * nb1 + e] = win[sk * nb1 + e];
    __syncthreads();
    const int r = k + nb1;
    for (int e = threadIdx.x; e < nb1; e += blockDim.x)
      win[sk * nb1 + e] = r < n ? pencil(band_val + (size_t)r * nb1 + e, stride, nmat, z, wp) : make_double2(0, 0);
    __syncthreads();
  }
}

// One warp solves Q_vv x = r for one right-hand side (band order).  rhs and
// x may alias.  Lanes hold band positions; y values of the last b rows are
// kept in a shared ring.
__device__ void band_solve_warp(int n, int b, const cplx* __restrict__ fac, const cplx* rhs, cplx* x, cplx* ring) {
  const int lane = threadIdx.x & 31;
  const int nb1 = b + 1;
  // forward: y_i = r_i - sum_{k<i} L_ik y_k ; store w_i = y_i / D_i
  for (int i = 0; i < n; ++i) {
    cplx acc = make_double2(0, 0);
    for (int t = lane; t < b; t += 32) {
      int k = i - b + t;            // column of entry t of row i
      if (k >= 0) acc = cadd(acc, cm(fac[(size_t)i * nb1 + t], ring[k % nb1]));
    }
    acc = warp_sum(acc);
    cplx y = csub(rhs[i], acc);
    __syncwarp();
    if (lane == 0) {
      ring[i % nb1] = y;
      x[i] = cdiv(y, fac[(size_t)i * nb1 + b]);
    }
    __syncwarp();
  }
  // backward: z_i = w_i - sum_{k>i} L_ki z_k
  for (int i = n - 1; i >= 0; --i) {
    cplx acc = make_double2(0, 0);
    for (int t = lane; t < b; t += 32) {
      int k = i + 1 + t;
      if (k < n) acc = cadd(acc, cm(fac[(size_t)k * nb1 + (i - k + b)], ring[k % nb1]));
    }
    acc = warp_sum(acc);
    cplx zi = csub(x[i], acc);
    __syncwarp();
    if (lane == 0) {
      ring[i % nb1] = zi;
      x[i] = zi;
    }
    __syncwarp();
  }
}

// W[f][g][:] = Q_vv(f)^-1 Q_vg(f)[:, g]: one warp per (f, g)
__global__ void k_border_solve(int n, int b, int ng, int nmat, const double* __restrict__ border_vg,
                               const cplx* __restrict__ zs, const double* __restrict__ wp_f,
                               const cplx* __restrict__ fac, cplx* __restrict__ Wb) {
  __shared__ cplx ring[kMaxBand + 1];
  const int f = blockIdx.x / ng, g = blockIdx.x % ng;
  const size_t vstride = (size_t)n * ng;
  cplx* x = Wb + ((size_t)f * ng + g) * n;
  for (int i = threadIdx.x; i < n; i += 32)
    x[i] = pencil(border_vg + (size_t)i * ng + g, vstride, nmat, zs + (size_t)f * nmat, wp_f[f]);
  __syncwarp();
  band_solve_warp(n, b, fac + (size_t)f * n * (b + 1), x, x, ring);
}

// S = Q_gg - Q_vg^T W, then S^-1 in place (Gauss-Jordan, partial pivoting); one warp per f
__global__ void k_schur(int n, int ng, int nmat, const double* __restrict__ border_vg,
                        const double* __restrict__ border_gg, const cplx* __restrict__ zs,
                        const double* __restrict__ wp_f, const cplx* __restrict__ Wb, cplx* __restrict__ Sinv) {
  const int f = blockIdx.x;
  const int lane = threadIdx.x & 31;
  __shared__ cplx A[kMaxBorder][2 * kMaxBorder];
  const cplx* z = zs + (size_t)f * nmat;
  const double wp = wp_f[f];
  const size_t vstride = (size_t)n * ng;
  for (int g1 = 0; g1 < ng; ++g1)
    for (int g2 = 0; g2 < ng; ++g2) {
      cplx acc = make_double2(0, 0);
      const cplx* w = Wb + ((size_t)f * ng + g2) * n;
      for (int i = lane; i < n; i += 32)
        acc = cadd(acc, cm(pencil(border_vg + (size_t)i * ng + g1, vstride, nmat, z, wp), w[i]));
      acc = warp_sum(acc);
      if (lane == 0) {
        cplx q = pencil(border_gg + (size_t)g1 * ng + g2, (size_t)ng * ng, nmat, z, wp);
        A[g1][g2] = csub(q, acc);
        A[g1][ng + g2] = make_double2(g1 == g2 ? 1.0 : 0.0, 0.0);
      }
    }
  __syncwarp();
  if (lane == 0) {
    for (int cc = 0; cc < ng; ++cc) {
      int piv = cc;
      for (int r = cc + 1; r < ng; ++r)
        if (cabs2(A[r][cc]) > cabs2(A[piv][cc])) piv = r;
      for (int k = 0; k < 2 * ng; ++k) {
        cplx t = A[cc][k];
        A[cc][k] = A[piv][k];
        A[piv][k] = t;
      }
      cplx d = A[cc][cc];
      for (int k = 0; k < 2 * ng; ++k) A[cc][k] = cdiv(A[cc][k], d);
      for (int r = 0; r < ng; ++r) {
        if (r == cc) continue;
        cplx fct = A[r][cc];
        for (int k = 0; k < 2 * ng; ++k) A[r][k] = csub(A[r][k], cm(fct, A[cc][k]));
      }
    }
    for (int g1 = 0; g1 < ng; ++g1)
      for (int g2 = 0; g2 < ng; ++g2) Sinv[((size_t)f * ng + g1) * ng + g2] = A[g1][ng + g2];
  }
}

// z = Q(f_s)^-1 v for every system; one warp per system.  scratch: [nsys][n] complex
__global__ void k_band_apply(int nloop, int n, int b, int ng, int nport, int nmat, const int32_t* __restrict__ perm,
                             const double* __restrict__ border_vg, const cplx* __restrict__ zs,
                             const double* __restrict__ wp_f, const cplx* __restrict__ fac,
                             const cplx* __restrict__ Wb, const cplx* __restrict__ Sinv, const cplx* __restrict__ v,
                             cplx* __restrict__ z, cplx* __restrict__ scratch, const int* __restrict__ active) {
  __shared__ cplx ring[kMaxBand + 1];
  __shared__ cplx tg[kMaxBorder], zg[kMaxBorder];
  const int s = blockIdx.x;
  if (active && !active[s]) return;
  const int f = s / nport;
  const int lane = threadIdx.x & 31;
  const cplx* vs = v + (size_t)s * nloop;
  cplx* zs_out = z + (size_t)s * nloop;
  cplx* x = scratch + (size_t)s * n;
  for (int i = lane; i < n; i += 32) x[i] = vs[perm[i]];
  __syncwarp();
  band_solve_warp(n, b, fac + (size_t)f * n * (b + 1), x, x, ring);
  if (ng > 0) {
    const cplx* zf = zs + (size_t)f * nmat;
    const double wp = wp_f[f];
    const size_t vstride = (size_t)n * ng;
    for (int g = 0; g < ng; ++g) {
      cplx acc = make_double2(0, 0);
      for (int i = lane; i < n; i += 32) acc = cadd(acc, cm(pencil(border_vg + (size_t)i * ng + g, vstride, nmat, zf, wp), x[i]));
      acc = warp_sum(acc);
      if (lane == 0) tg[g] = csub(vs[n + g], acc);
    }
    __syncwarp();
    if (lane < ng) {
      cplx acc = make_double2(0, 0);
      for (int g2 = 0; g2 < ng; ++g2) acc = cadd(acc, cm(Sinv[((size_t)f * ng + lane) * ng + g2], tg[g2]));
      zg[lane] = acc;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      cplx acc = x[i];
      for (int g = 0; g < ng; ++g) acc = csub(acc, cm(Wb[((size_t)f * ng + g) * n + i], zg[g]));
      x[i] = acc;
    }
    __syncwarp();
    if (lane < ng) zs_out[n + lane] = zg[lane];
  }
  for (int i = lane; i < n; i += 32) zs_out[perm[i]] = x[i];
}

// ---- host ---------------------------------------------------------------------------------
bool band_usable(const xrl_ctx* c) {
  return c->topo.band <= kMaxBand && c->topo.n_border <= kMaxBorder && c->topo.n_band > 0;
}

void band_prepare(xrl_ctx* c) {
  const Topo& T = c->topo;
  c->d.band_perm.upload(c->alloc, T.band_perm);
  c->d.band_val.upload(c->alloc, T.band_val);
  c->d.border_vg.upload(c->alloc, T.border_vg);
  c->d.border_gg.upload(c->alloc, T.border_gg);
}

// factor Q(f) for nf frequencies (zs [nf][nmat], wp [nf]) into fac, W, Sinv
void band_factor(xrl_ctx* c, int nf, const cplx* zs, const double* wp, cplx* fac, cplx* Wb, cplx* Sinv,
                 cudaStream_t s) {
  const Topo& T = c->topo;
  const int n = T.n_band, b = T.band, ng = T.n_border;
  size_t smem = sizeof(cplx) * (b + 1) * (b + 1);
  if (smem > 48 * 1024) XRL_CUDA(cudaFuncSetAttribute(k_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaEvent_t ev = prof_begin(c, s);
  k_band_factor<<<nf, 256, smem, s>>>(n, b, T.n_mat, c->d.band_val.p, zs, wp, fac);
  int launches = 1;
  if (ng > 0) {
    k_border_solve<<<nf * ng, 32, 0, s>>>(n, b, ng, T.n_mat, c->d.border_vg.p, zs, wp, fac, Wb);
    k_schur<<<nf, 32, 0, s>>>(n, ng, T.n_mat, c->d.border_vg.p, c->d.border_gg.p, zs, wp, Wb, Sinv);
    launches += 2;
  }
  prof_end(c, s, ev, PH_PREC, launches, 8.0 * nf * (double)n * b * b / 2.0, 16.0 * nf * (double)n * (b + 1) * 2.0);
  XRL_CUDA(cudaGetLastError());
}

void band_apply(xrl_ctx* c, int nsys, int nport, const cplx* zs, const double* wp, const cplx* fac, const cplx* Wb,
                const cplx* Sinv, const cplx* v, cplx* z, cplx* scratch, const int* active, cudaStream_t s) {
  const Topo& T = c->topo;
  cudaEvent_t ev = prof_begin(c, s);
  k_band_apply<<<nsys, 32, 0, s>>>(T.n_loops, T.n_band, T.band, T.n_border, nport, T.n_mat, c->d.band_perm.p,
                                   c->d.border_vg.p, zs, wp, fac, Wb, Sinv, v, z, scratch, active);
  prof_end(c, s, ev, PH_PREC, 1, 16.0 * nsys * (double)T.n_band * T.band,
           16.0 * nsys * (double)T.n_band * (2.0 * T.band + 4.0));
  XRL_CUDA(cudaGetLastError());
}

}  // namespace xrl
