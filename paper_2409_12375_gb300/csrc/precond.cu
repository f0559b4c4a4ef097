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

// ---- asynchronous global -> shared copies (16 bytes each) ----------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// rows per streamed chunk: >= b so that the backward pass needs at most two chunks
__host__ __device__ inline int band_chunk(int b) { return b <= 32 ? 32 : 64; }
constexpr int kRing = 64;   // power of two > kMaxBand
// row stride of a stored factor: b + 1, rounded up to even for 8-byte elements
template <class C>
__host__ __device__ inline int band_rs(int b) { return sizeof(C) == 8 ? ((b + 2) & ~1) : b + 1; }
template <class C>
__host__ __device__ inline size_t band_smem_bytes(int b) {
  const int ch = band_chunk(b);
  return sizeof(C) * ((size_t)2 * ch * band_rs<C>(b) + 2 * (size_t)ch);
}

// complex helpers for both precisions
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return cm(a, b); }
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 wsum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double2 wsum(double2 v) { return warp_sum(v); }
__device__ __forceinline__ float2 csubT(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 caddT(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 caddT(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ double2 csubT(double2 a, double2 b) { return csub(a, b); }

// copy rows [r0, r1) of the factor (row stride rs) and entries [r0, r1) of vec
// into shared buffers with 16-byte asynchronous copies.  For 8-byte elements
// rs and r0 are even and vec has a readable element past its end.
template <class C>
__device__ __forceinline__ void band_issue(const C* fac, const C* vec, int r0, int r1, int rs, C* fb, C* vb) {
  constexpr int per = 16 / sizeof(C);
  const int lane = threadIdx.x & 31;
  const int nf = (r1 - r0) * rs;
  const C* src = fac + (size_t)r0 * rs;
  for (int e = per * lane; e < nf; e += 32 * per) cp_async16(fb + e, src + e);
  for (int e = per * lane; e < r1 - r0; e += 32 * per) cp_async16(vb + e, vec + r0 + e);
  cp_commit();
}

// One warp solves Q_vv x = r (band order) in place: rhs in x on entry.  The
// factor holds L below the diagonal and 1/D on it.  Factor rows and the
// right-hand side stream through shared memory in chunks of `ch` rows
// (cp.async, one chunk ahead), so the sequential substitution waits on
// shared memory only.  smem: 3 factor chunks, 2 vector chunks, a ring of the
// last kRing solution values.  C = float2 (mixed precision) or double2.
// One warp solves Q_vv x = r (band order) in place: rhs in x on entry.
// facT holds the factor by columns (facT[i][t] = L[i+1+t][i], facT[i][b] =
// 1/D_i) and fac by rows (fac[i][t] = L[i][i-b+t]); both stream through
// shared memory in chunks (cp.async, one chunk ahead).  The substitution is
// column oriented: row k's pending sum lives in lane k % 32 (slot (k/32)%2),
// (the sum of L_ki times the unknowns already found), so a step is one
// broadcast of the new unknown and at most two complex FMAs per lane.  smem: 2 factor chunks + 2 vector chunks.
template <class C>
__device__ __forceinline__ C csel(bool s, C a, C b) { return s ? a : b; }

template <class C>
__device__ void band_solve_warp(int n, int b, int rs, const C* __restrict__ facT, const C* __restrict__ fac, C* x,
                                C* smem) {
  const int lane = threadIdx.x & 31;
  const int ch = band_chunk(b);
  const size_t fstride = (size_t)ch * rs;
  C* fbuf = smem;                       // [2][ch * rs]
  C* vbuf = smem + 2 * fstride;         // [2][ch]
  const int nchunk = (n + ch - 1) / ch;
  __threadfence();   // x was written by this warp's plain stores; cp.async reads L2
  __syncwarp();
  C acc0 = czero<C>(), acc1 = czero<C>();
  // forward: y_i = r_i - sum_{k<i} L_ik y_k ; x_i <- w_i = y_i / D_i
  band_issue<C>(facT, x, 0, min(n, ch), rs, fbuf, vbuf);
  for (int c = 0; c < nchunk; ++c) {
    const int r0 = c * ch, r1 = min(n, r0 + ch);
    const bool more = c + 1 < nchunk;
    if (more) band_issue<C>(facT, x, r1, min(n, r1 + ch), rs, fbuf + ((c + 1) & 1) * fstride, vbuf + ((c + 1) & 1) * ch);
    if (more) cp_wait_all_but_one(); else cp_wait_all();
    __syncwarp();
    const C* fr = fbuf + (c & 1) * fstride;
    const C* vr = vbuf + (c & 1) * ch;
    for (int i = r0; i < r1; ++i) {
      const C* col = fr + (size_t)(i - r0) * rs;
      const int own = i & 31;
      const bool s1 = (i >> 5) & 1;
      C y = czero<C>();
      if (lane == own) {
        y = csubT(vr[i - r0], csel(s1, acc1, acc0));
        if (s1) acc1 = czero<C>(); else acc0 = czero<C>();
      }
      y.x = __shfl_sync(0xffffffffu, y.x, own);
      y.y = __shfl_sync(0xffffffffu, y.y, own);
      if (lane == own) x[i] = cmul(y, col[b]);
      const int t = (lane - i - 1) & 31;
      int k = i + 1 + t;
      if (t < b && k < n) {
        C d = cmul(col[t], y);
        if ((k >> 5) & 1) acc1 = caddT(acc1, d); else acc0 = caddT(acc0, d);
      }
      k += 32;
      if (t + 32 < b && k < n) {
        C d = cmul(col[t + 32], y);
        if ((k >> 5) & 1) acc1 = caddT(acc1, d); else acc0 = caddT(acc0, d);
      }
    }
    __syncwarp();
  }
  __syncwarp();
  __threadfence();
  __syncwarp();
  // backward: z_i = w_i - sum_{k>i} L_ki z_k, rows of fac in descending chunks
  acc0 = czero<C>();
  acc1 = czero<C>();
  {
    const int c = nchunk - 1;
    band_issue<C>(fac, x, c * ch, n, rs, fbuf + (c & 1) * fstride, vbuf + (c & 1) * ch);
  }
  for (int c = nchunk - 1; c >= 0; --c) {
    const int r0 = c * ch, r1 = min(n, r0 + ch);
    const bool more = c > 0;
    if (more) band_issue<C>(fac, x, r0 - ch, r0, rs, fbuf + ((c - 1) & 1) * fstride, vbuf + ((c - 1) & 1) * ch);
    if (more) cp_wait_all_but_one(); else cp_wait_all();
    __syncwarp();
    const C* fr = fbuf + (c & 1) * fstride;
    const C* vr = vbuf + (c & 1) * ch;
    for (int i = r1 - 1; i >= r0; --i) {
      const C* row = fr + (size_t)(i - r0) * rs;
      const int own = i & 31;
      const bool s1 = (i >> 5) & 1;
      C z = czero<C>();
      if (lane == own) {
        z = csubT(vr[i - r0], csel(s1, acc1, acc0));
        if (s1) acc1 = czero<C>(); else acc0 = czero<C>();
      }
      z.x = __shfl_sync(0xffffffffu, z.x, own);
      z.y = __shfl_sync(0xffffffffu, z.y, own);
      if (lane == own) x[i] = z;
      // rows k in [i-b, i-1] owned by this lane: k = i - 1 - ((i - 1 - lane) & 31), then k - 32
      int k = i - 1 - ((i - 1 - lane) & 31);
      if (k >= 0 && k >= i - b) {
        C d = cmul(row[k - i + b], z);
        if ((k >> 5) & 1) acc1 = caddT(acc1, d); else acc0 = caddT(acc0, d);
      }
      k -= 32;
      if (k >= 0 && k >= i - b) {
        C d = cmul(row[k - i + b], z);
        if ((k >> 5) & 1) acc1 = caddT(acc1, d); else acc0 = caddT(acc0, d);
      }
    }
    __syncwarp();
  }
}

// Two systems that share one factor (the two ports of one frequency) per
// warp, 16 lanes each, for half-widths b <= 15: row k's pending sum lives in
// half-lane k % 16.  The factor chunks are shared by both halves; each half
// streams its own right-hand side (x0, x1, in place).
template <class C>
__device__ void band_solve_pair(int n, int b, int rs, const C* __restrict__ facT, const C* __restrict__ fac, C* x0,
                                C* x1, C* smem) {
  const int lane = threadIdx.x & 31;
  const int h = lane >> 4, hl = lane & 15;
  const int ch = band_chunk(b);
  const size_t fstride = (size_t)ch * rs;
  C* fbuf = smem;                       // [2][ch * rs]
  C* vbuf = smem + 2 * fstride;         // [2 buffers][2 halves][ch]
  const int nchunk = (n + ch - 1) / ch;
  C* xh = h ? x1 : x0;
  auto issue = [&](const C* F, int r0, int r1, int buf) {
    constexpr int per = 16 / sizeof(C);
    const int nf = (r1 - r0) * rs;
    const C* src = F + (size_t)r0 * rs;
    C* fb = fbuf + buf * fstride;
    for (int e = per * lane; e < nf; e += 32 * per) cp_async16(fb + e, src + e);
    C* vb = vbuf + (buf * 2 + h) * ch;
    for (int e = per * hl; e < r1 - r0; e += 16 * per) cp_async16(vb + e, xh + r0 + e);
    cp_commit();
  };
  __threadfence();
  __syncwarp();
  C acc = czero<C>();
  issue(facT, 0, min(n, ch), 0);
  for (int c = 0; c < nchunk; ++c) {
    const int r0 = c * ch, r1 = min(n, r0 + ch);
    const bool more = c + 1 < nchunk;
    if (more) issue(facT, r1, min(n, r1 + ch), (c + 1) & 1);
    if (more) cp_wait_all_but_one(); else cp_wait_all();
    __syncwarp();
    const C* fr = fbuf + (c & 1) * fstride;
    const C* vr = vbuf + ((c & 1) * 2 + h) * ch;
    for (int i = r0; i < r1; ++i) {
      const C* col = fr + (size_t)(i - r0) * rs;
      const int own = i & 15;
      const int t = (hl - i - 1) & 15;
      const C lv = col[t < b ? t : 0];          // independent of y: load early
      C y = czero<C>();
      if (hl == own) {
        y = csubT(vr[i - r0], acc);
        acc = czero<C>();
      }
      y.x = __shfl_sync(0xffffffffu, y.x, own, 16);
      y.y = __shfl_sync(0xffffffffu, y.y, own, 16);
      if (hl == own) xh[i] = cmul(y, col[b]);
      if (t < b && i + 1 + t < n) acc = cfma(lv, y, acc);
    }
    __syncwarp();
  }
  __syncwarp();
  __threadfence();
  __syncwarp();
  acc = czero<C>();
  {
    const int c = nchunk - 1;
    issue(fac, c * ch, n, c & 1);
  }
  for (int c = nchunk - 1; c >= 0; --c) {
    const int r0 = c * ch, r1 = min(n, r0 + ch);
    const bool more = c > 0;
    if (more) issue(fac, r0 - ch, r0, (c - 1) & 1);
    if (more) cp_wait_all_but_one(); else cp_wait_all();
    __syncwarp();
    const C* fr = fbuf + (c & 1) * fstride;
    const C* vr = vbuf + ((c & 1) * 2 + h) * ch;
    for (int i = r1 - 1; i >= r0; --i) {
      const C* row = fr + (size_t)(i - r0) * rs;
      const int own = i & 15;
      const int k = i - 1 - ((i - 1 - hl) & 15);
      const bool upd = k >= 0 && k >= i - b;
      const C lv = row[upd ? k - i + b : 0];
      C z = czero<C>();
      if (hl == own) {
        z = csubT(vr[i - r0], acc);
        acc = czero<C>();
      }
      z.x = __shfl_sync(0xffffffffu, z.x, own, 16);
      z.y = __shfl_sync(0xffffffffu, z.y, own, 16);
      if (hl == own) xh[i] = z;
      if (upd) acc = cfma(lv, z, acc);
    }
    __syncwarp();
  }
}

// 1/D on the diagonal; the column-form copy facT (facT[i][t] = L[i+1+t][i],
// facT[i][b] = 1/D_i); optional FP32 copies of both (row stride even).
// One thread per (frequency row, entry).
__global__ void k_band_finish(int nf, int n, int b, cplx* __restrict__ fac, cplx* __restrict__ facT,
                              float2* __restrict__ fac32, float2* __restrict__ facT32) {
  const size_t nb1 = b + 1;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nf * n * nb1) return;
  const size_t rowg = e / nb1;          // global row (f * n + i)
  const int t = (int)(e % nb1);
  const int i = (int)(rowg % n);
  const size_t fbase = rowg - i;        // f * n
  const int rs32 = band_rs<float2>(b);
  if (t == b) {
    cplx inv = cdiv(make_double2(1.0, 0.0), fac[e]);
    fac[e] = inv;
    facT[e] = inv;
    if (fac32) {
      fac32[rowg * rs32 + b] = make_float2((float)inv.x, (float)inv.y);
      facT32[rowg * rs32 + b] = make_float2((float)inv.x, (float)inv.y);
      if (rs32 > (int)nb1) {
        fac32[rowg * rs32 + nb1] = make_float2(0.f, 0.f);
        facT32[rowg * rs32 + nb1] = make_float2(0.f, 0.f);
      }
    }
    return;
  }
  // row form entry (i, t) = L[i][i-b+t]
  cplx v = fac[e];
  if (fac32) fac32[rowg * rs32 + t] = make_float2((float)v.x, (float)v.y);
  // column form entry (i, t) = L[i+1+t][i] = row i+1+t, index b-1-t
  const int k = i + 1 + t;
  cplx w = make_double2(0.0, 0.0);
  if (k < n) w = fac[(fbase + k) * nb1 + (b - 1 - t)];
  facT[e] = w;
  if (fac32) facT32[rowg * rs32 + t] = make_float2((float)w.x, (float)w.y);
}

// W[f][g][:] = Q_vv(f)^-1 Q_vg(f)[:, g]: one warp per (f, g)
__global__ void k_border_solve(int n, int b, int ng, int nmat, const double* __restrict__ border_vg,
                               const cplx* __restrict__ zs, const double* __restrict__ wp_f,
                               const cplx* __restrict__ fac, const cplx* __restrict__ facT, cplx* __restrict__ Wb) {
  extern __shared__ cplx bsm[];
  const int f = blockIdx.x / ng, g = blockIdx.x % ng;
  const size_t vstride = (size_t)n * ng;
  cplx* x = Wb + ((size_t)f * ng + g) * n;
  for (int i = threadIdx.x; i < n; i += 32)
    x[i] = pencil(border_vg + (size_t)i * ng + g, vstride, nmat, zs + (size_t)f * nmat, wp_f[f]);
  __syncwarp();
  band_solve_warp<cplx>(n, b, b + 1, facT + (size_t)f * n * (b + 1), fac + (size_t)f * n * (b + 1), x, bsm);
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

// z = Q(f_s)^-1 v for every system; one warp per system; C = float2 (mixed
// precision triangular solves from an FP64-computed factor) or double2.
template <class C>
__global__ void k_band_apply(int nloop, int n, int b, int ng, int nport, int nmat, const int32_t* __restrict__ perm,
                             const double* __restrict__ border_vg, const cplx* __restrict__ zs,
                             const double* __restrict__ wp_f, const C* __restrict__ fac, const C* __restrict__ facT,
                             const cplx* __restrict__ Wb, const cplx* __restrict__ Sinv, const cplx* __restrict__ v,
                             cplx* __restrict__ z, C* __restrict__ scratch, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char bsm_raw[];
  C* bsm = reinterpret_cast<C*>(bsm_raw);
  __shared__ cplx tg[kMaxBorder], zg[kMaxBorder];
  const int s = blockIdx.x;
  if (active && !active[s]) return;
  const int f = s / nport;
  const int lane = threadIdx.x & 31;
  const cplx* vs = v + (size_t)s * nloop;
  cplx* zs_out = z + (size_t)s * nloop;
  C* x = scratch + (size_t)s * (size_t)((n + 2) & ~1);
  for (int i = lane; i < n; i += 32) {
    cplx vi = vs[perm[i]];
    if (sizeof(C) == 8) {
      reinterpret_cast<float2*>(x)[i] = make_float2((float)vi.x, (float)vi.y);
    } else {
      reinterpret_cast<cplx*>(x)[i] = vi;
    }
  }
  __syncwarp();
  band_solve_warp<C>(n, b, band_rs<C>(b), facT + (size_t)f * n * band_rs<C>(b), fac + (size_t)f * n * band_rs<C>(b),
                     x, bsm);
  auto xval = [&](int i) -> cplx {
    if (sizeof(C) == 8) {
      float2 t = reinterpret_cast<const float2*>(x)[i];
      return make_double2(t.x, t.y);
    }
    return reinterpret_cast<const cplx*>(x)[i];
  };
  if (ng > 0) {
    const cplx* zf = zs + (size_t)f * nmat;
    const double wp = wp_f[f];
    const size_t vstride = (size_t)n * ng;
    for (int g = 0; g < ng; ++g) {
      cplx acc = make_double2(0, 0);
      for (int i = lane; i < n; i += 32) acc = cadd(acc, cm(pencil(border_vg + (size_t)i * ng + g, vstride, nmat, zf, wp), xval(i)));
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
      cplx acc = xval(i);
      for (int g = 0; g < ng; ++g) acc = csub(acc, cm(Wb[((size_t)f * ng + g) * n + i], zg[g]));
      zs_out[perm[i]] = acc;
    }
    __syncwarp();
    if (lane < ng) zs_out[n + lane] = zg[lane];
  } else {
    for (int i = lane; i < n; i += 32) zs_out[perm[i]] = xval(i);
  }
}

// as k_band_apply, two systems (consecutive, same frequency) per warp
template <class C>
__global__ void k_band_apply_pair(int nloop, int n, int b, int ng, int nport, int nmat, const int32_t* __restrict__ perm,
                                  const double* __restrict__ border_vg, const cplx* __restrict__ zs,
                                  const double* __restrict__ wp_f, const C* __restrict__ fac,
                                  const C* __restrict__ facT, const cplx* __restrict__ Wb,
                                  const cplx* __restrict__ Sinv, const cplx* __restrict__ v, cplx* __restrict__ z,
                                  C* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char bsm_raw[];
  C* bsm = reinterpret_cast<C*>(bsm_raw);
  __shared__ cplx tg[2][kMaxBorder], zg[2][kMaxBorder];
  const int s0 = 2 * blockIdx.x;
  const int f = s0 / nport;
  const int lane = threadIdx.x & 31;
  const size_t xs = (size_t)((n + 2) & ~1);
  C* x0 = scratch + (size_t)s0 * xs;
  C* x1 = x0 + xs;
  for (int q = 0; q < 2; ++q) {
    const cplx* vs = v + (size_t)(s0 + q) * nloop;
    C* x = q ? x1 : x0;
    for (int i = lane; i < n; i += 32) {
      cplx vi = vs[perm[i]];
      if (sizeof(C) == 8) reinterpret_cast<float2*>(x)[i] = make_float2((float)vi.x, (float)vi.y);
      else reinterpret_cast<cplx*>(x)[i] = vi;
    }
  }
  __syncwarp();
  const int rs = band_rs<C>(b);
  band_solve_pair<C>(n, b, rs, facT + (size_t)f * n * rs, fac + (size_t)f * n * rs, x0, x1, bsm);
  for (int q = 0; q < 2; ++q) {
    const C* x = q ? x1 : x0;
    const cplx* vs = v + (size_t)(s0 + q) * nloop;
    cplx* zo = z + (size_t)(s0 + q) * nloop;
    auto xval = [&](int i) -> cplx {
      if (sizeof(C) == 8) {
        float2 t = reinterpret_cast<const float2*>(x)[i];
        return make_double2(t.x, t.y);
      }
      return reinterpret_cast<const cplx*>(x)[i];
    };
    if (ng > 0) {
      const cplx* zf = zs + (size_t)f * nmat;
      const double wp = wp_f[f];
      const size_t vstride = (size_t)n * ng;
      for (int g = 0; g < ng; ++g) {
        cplx acc = make_double2(0, 0);
        for (int i = lane; i < n; i += 32) acc = cadd(acc, cm(pencil(border_vg + (size_t)i * ng + g, vstride, nmat, zf, wp), xval(i)));
        acc = warp_sum(acc);
        if (lane == 0) tg[q][g] = csub(vs[n + g], acc);
      }
      __syncwarp();
      if (lane < ng) {
        cplx acc = make_double2(0, 0);
        for (int g2 = 0; g2 < ng; ++g2) acc = cadd(acc, cm(Sinv[((size_t)f * ng + lane) * ng + g2], tg[q][g2]));
        zg[q][lane] = acc;
      }
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        cplx acc = xval(i);
        for (int g = 0; g < ng; ++g) acc = csub(acc, cm(Wb[((size_t)f * ng + g) * n + i], zg[q][g]));
        zo[perm[i]] = acc;
      }
      __syncwarp();
      if (lane < ng) zo[n + lane] = zg[q][lane];
    } else {
      for (int i = lane; i < n; i += 32) zo[perm[i]] = xval(i);
    }
    __syncwarp();
  }
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
void band_factor(xrl_ctx* c, int nf, const cplx* zs, const double* wp, cplx* fac, cplx* facT, float2* fac32,
                 float2* facT32, cplx* Wb, cplx* Sinv, cudaStream_t s) {
  const Topo& T = c->topo;
  const int n = T.n_band, b = T.band, ng = T.n_border;
  size_t smem = sizeof(cplx) * (b + 1) * (b + 1);
  if (smem > 48 * 1024) XRL_CUDA(cudaFuncSetAttribute(k_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaEvent_t ev = prof_begin(c, s);
  k_band_factor<<<nf, 256, smem, s>>>(n, b, T.n_mat, c->d.band_val.p, zs, wp, fac);
  int launches = 1;
  const size_t bsd = band_smem_bytes<cplx>(b);
  if (bsd > 48 * 1024)
    XRL_CUDA(cudaFuncSetAttribute(k_border_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsd));
  // 1/D on the diagonal (and the FP32 copy for mixed-precision solves)
  {
    size_t tot = (size_t)nf * n * (b + 1);
    k_band_finish<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nf, n, b, fac, facT, fac32, facT32);
    ++launches;
  }
  if (ng > 0) {
    k_border_solve<<<nf * ng, 32, bsd, s>>>(n, b, ng, T.n_mat, c->d.border_vg.p, zs, wp, fac, facT, Wb);
    k_schur<<<nf, 32, 0, s>>>(n, ng, T.n_mat, c->d.border_vg.p, c->d.border_gg.p, zs, wp, Wb, Sinv);
    launches += 2;
  }
  prof_end(c, s, ev, PH_PREC, launches, 8.0 * nf * (double)n * b * b / 2.0, 16.0 * nf * (double)n * (b + 1) * 2.0);
  XRL_CUDA(cudaGetLastError());
}

void band_apply(xrl_ctx* c, int nsys, int nport, const cplx* zs, const double* wp, const cplx* fac,
                const cplx* facT, const float2* fac32, const float2* facT32, const cplx* Wb, const cplx* Sinv,
                const cplx* v, cplx* z, void* scratch, const int* active, cudaStream_t s) {
  const Topo& T = c->topo;
  cudaEvent_t ev = prof_begin(c, s);
  // systems 2q, 2q+1 share a frequency when nport is even; converged systems are
  // recomputed harmlessly on this path (their results are not used)
  const bool pair = T.band <= 15 && nport % 2 == 0 && nsys % 2 == 0;
  if (pair) {
    if (fac32) {
      const size_t bs = sizeof(float2) * ((size_t)2 * band_chunk(T.band) * band_rs<float2>(T.band) +
                                          4 * (size_t)band_chunk(T.band));
      k_band_apply_pair<float2><<<nsys / 2, 32, bs, s>>>(T.n_loops, T.n_band, T.band, T.n_border, nport, T.n_mat,
                                                         c->d.band_perm.p, c->d.border_vg.p, zs, wp, fac32, facT32,
                                                         Wb, Sinv, v, z, (float2*)scratch);
    } else {
      const size_t bs = sizeof(cplx) * ((size_t)2 * band_chunk(T.band) * band_rs<cplx>(T.band) +
                                        4 * (size_t)band_chunk(T.band));
      k_band_apply_pair<cplx><<<nsys / 2, 32, bs, s>>>(T.n_loops, T.n_band, T.band, T.n_border, nport, T.n_mat,
                                                       c->d.band_perm.p, c->d.border_vg.p, zs, wp, fac, facT, Wb,
                                                       Sinv, v, z, (cplx*)scratch);
    }
  } else if (fac32) {
    const size_t bs = band_smem_bytes<float2>(T.band) + 64;
    if (bs > 48 * 1024)
      XRL_CUDA(cudaFuncSetAttribute(k_band_apply<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs));
    k_band_apply<float2><<<nsys, 32, bs, s>>>(T.n_loops, T.n_band, T.band, T.n_border, nport, T.n_mat,
                                              c->d.band_perm.p, c->d.border_vg.p, zs, wp, fac32, facT32, Wb, Sinv, v, z,
                                              (float2*)scratch, active);
  } else {
    const size_t bs = band_smem_bytes<cplx>(T.band) + 64;
    if (bs > 48 * 1024)
      XRL_CUDA(cudaFuncSetAttribute(k_band_apply<cplx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs));
    k_band_apply<cplx><<<nsys, 32, bs, s>>>(T.n_loops, T.n_band, T.band, T.n_border, nport, T.n_mat,
                                            c->d.band_perm.p, c->d.border_vg.p, zs, wp, fac, facT, Wb, Sinv, v, z,
                                            (cplx*)scratch, active);
  }
  const double es = fac32 ? 8.0 : 16.0;
  prof_end(c, s, ev, PH_PREC, 1, 16.0 * nsys * (double)T.n_band * T.band,
           es * nsys * (double)T.n_band * (2.0 * T.band + 4.0));
  XRL_CUDA(cudaGetLastError());
}

}  // namespace xrl
