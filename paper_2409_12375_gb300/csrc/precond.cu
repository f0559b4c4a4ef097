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
//
// The band is solved by partitioning (the SPIKE scheme of Polizzi and Sameh,
// 2006), exactly up to rounding: Q_vv splits into P diagonal blocks A_j of m
// rows coupled through b x b corners B_j (rows of block j, columns of block
// j+1) and C_j = B_{j-1}^T.  With y_j = A_j^-1 f_j and the spikes
// V_j = A_j^-1 [0; B_j], W_j = A_j^-1 [C_j; 0] (m x b each),
//   x_j = y_j - V_j t_{j+1} - W_j u_{j-1},
// t_j, u_j the first and last b unknowns of block j.  Their 2b(P-1) values
// solve a block-tridiagonal system in z_j = (u_j, t_{j+1}):
//   E_j z_j + F_j z_{j-1} + G_j z_{j+1} = (y_j^bot, y_{j+1}^top),
//   E_j = [I, V_j^bot; W_{j+1}^top, I], F_j = [W_j^bot 0; 0 0], G_j = [0 0; 0 V_{j+1}^top],
// factored once by block LU (E^_j = E_j - F_j E^_{j-1}^-1 G_{j-1}, which only
// changes the top-right block, stored as E^_j^-1).  So
//  * factor: one warp per (frequency, block) for A_j = L D L^T, one warp per
//    spike column, one CTA per frequency for the reduced system;
//  * apply: one warp per (system pair, block) for y_j, one warp per system
//    for the reduced forward/backward substitution, one CTA per system for the
//    spike correction, the border correction and the scatter to loop order.
#include <vector>

#include "cplx.cuh"
#include "xrl_internal.hpp"

namespace xrl {

constexpr int kMaxBand = 63;     // window (b+1)^2 complex in shared memory
constexpr int kMaxBorder = 16;
constexpr double kNullPivot2 = 1e-20;   // (|pivot| / |original diagonal|)^2 below which a pivot is null

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
    // a stored pivot of exactly 0 is a deflated null pivot (k_band_factor_blk): 1/D := 0
    const cplx d = fac[e];
    cplx inv = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), d);
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

// S = Q_gg - Q_vg^T W, then S^-1 in place (Gauss-Jordan, partial pivoting); one CTA per f
__global__ void k_schur(int n, int ng, int nmat, const double* __restrict__ border_vg,
                        const double* __restrict__ border_gg, const cplx* __restrict__ zs,
                        const double* __restrict__ wp_f, const cplx* __restrict__ Wb, cplx* __restrict__ Sinv) {
  const int f = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ cplx A[kMaxBorder][2 * kMaxBorder];
  const cplx* z = zs + (size_t)f * nmat;
  const double wp = wp_f[f];
  const size_t vstride = (size_t)n * ng;
  // one (g1, g2) entry per warp at a time
  for (int pr = warp; pr < ng * ng; pr += nw) {
    const int g1 = pr / ng, g2 = pr % ng;
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
  __syncthreads();
  if (threadIdx.x == 0) {
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

template <class C>
__device__ __forceinline__ C to_c(cplx v);
template <>
__device__ __forceinline__ float2 to_c<float2>(cplx v) { return make_float2((float)v.x, (float)v.y); }
template <>
__device__ __forceinline__ double2 to_c<double2>(cplx v) { return v; }
__device__ __forceinline__ cplx to_d(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ cplx to_d(double2 v) { return v; }

__device__ __forceinline__ float cabs2T(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double cabs2T(double2 a) { return cabs2(a); }
__device__ __forceinline__ float2 crecipT(float2 a) {
  const float d = a.x * a.x + a.y * a.y;
  return make_float2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double2 crecipT(double2 a) { return cdiv(make_double2(1.0, 0.0), a); }
template <class C> __device__ __forceinline__ C cone();
template <> __device__ __forceinline__ float2 cone<float2>() { return make_float2(1.f, 0.f); }
template <> __device__ __forceinline__ double2 cone<double2>() { return make_double2(1.0, 0.0); }

// ---- partitioned (SPIKE) factor --------------------------------------------------------------

// LDL^T of the diagonal block j of Q_vv(f) (rows [s0, e0)), couplings to other
// blocks dropped; one warp per (f, j), the active (b+1) x (b+1) window in
// shared memory as a ring of rows.  fac[f][i][k]: k < b strictly lower L
// (column i - b + k), k = b the diagonal D.
__global__ void k_band_factor_blk(int n, int b, int P, int m, int nmat, const double* __restrict__ band_val,
                                  const cplx* __restrict__ zs, const double* __restrict__ wp_f,
                                  cplx* __restrict__ fac) {
  extern __shared__ cplx win[];   // [(b+1)][(b+1)] ring, then orig[b], then the pair table
  const int f = blockIdx.x / P, j = blockIdx.x % P;
  const int s0 = j * m, e0 = (j == P - 1) ? n : min(n, s0 + m);
  const int mm = e0 - s0;
  const int lane = threadIdx.x;
  const int nb1 = b + 1;
  const size_t stride = (size_t)n * nb1;
  const cplx* z = zs + (size_t)f * nmat;
  const double wp = wp_f[f];
  cplx* out = fac + (size_t)f * stride + (size_t)s0 * nb1;
  cplx* orig = win + nb1 * nb1;
  short2* pairs = reinterpret_cast<short2*>(orig + b);
  const int npair = b * (b + 1) / 2;
  for (int q = lane; q < npair; q += 32) {
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= q) ++ti;
    pairs[q] = make_short2((short)ti, (short)(q - ti * (ti + 1) / 2));
  }
  auto load_row = [&](int r, int slot) {
    for (int e = lane; e < nb1; e += 32) {
      cplx v = make_double2(0.0, 0.0);
      if (r < mm && e >= b - r) v = pencil(band_val + (size_t)(s0 + r) * nb1 + e, stride, nmat, z, wp);
      win[slot * nb1 + e] = v;
    }
  };
  for (int r = 0; r < nb1; ++r) load_row(r, r);
  __syncwarp();
  for (int k = 0; k < mm; ++k) {
    const int sk = k % nb1;
    // Null pivot: a pivot at rounding level of the row's own diagonal marks a
    // null direction of Q (loop currents with no panel current, e.g. the
    // checkerboard pattern of vertex loops on a grid of rectangles, which the
    // pulse basis of eq. 4 cannot see; Z shares it and the port right-hand
    // sides are orthogonal to it).  It is deflated: no elimination with it and
    // a stored pivot of 0 (1/D := 0), so the solve leaves that direction at zero.
    const cplx dk = win[sk * nb1 + b];
    const cplx a0 = pencil(band_val + (size_t)(s0 + k) * nb1 + b, stride, nmat, z, wp);
    const bool null_pivot = dk.x * dk.x + dk.y * dk.y <= kNullPivot2 * (a0.x * a0.x + a0.y * a0.y);
    const cplx inv = null_pivot ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), dk);
    __syncwarp();
    if (null_pivot && lane == 0) win[sk * nb1 + b] = make_double2(0.0, 0.0);
    for (int t = lane; t < b; t += 32) {
      const int i = k + 1 + t;
      cplx o = make_double2(0.0, 0.0);
      if (i < mm) {
        cplx* w = win + (i % nb1) * nb1 + (b - 1 - t);
        o = *w;
        *w = cm(o, inv);
      }
      orig[t] = o;
    }
    __syncwarp();
    for (int q = lane; q < npair; q += 32) {
      const short2 pq = pairs[q];
      const int i = k + 1 + pq.x;
      if (i < mm) {
        cplx* row = win + (i % nb1) * nb1;
        row[b - (pq.x - pq.y)] = csub(row[b - (pq.x - pq.y)], cm(row[b - 1 - pq.x], orig[pq.y]));
      }
    }
    __syncwarp();
    for (int e = lane; e < nb1; e += 32) out[(size_t)k * nb1 + e] = win[sk * nb1 + e];
    __syncwarp();
    load_row(k + nb1, sk);
    __syncwarp();
  }
}

// Spike columns: V_j[:, c] = A_j^-1 [0; B_j[:, c]] (col = c < b, j < P-1) and
// W_j[:, c] = A_j^-1 [C_j[:, c]; 0] (col = b + c, j > 0), stored by column,
// Vsp[f][c][i] for the rows i of block j.  B_j[r][c] = Q[e0-b+r][e0+c]
// (r >= c) and C_j[r][c] = Q[s0+r][s0-b+c] (c >= r) read from the band rows.
// One warp per (f, j, col); C = float2 (mixed precision, from the FP32
// factor copies) or double2.
template <class C>
__global__ void k_spike_cols(int n, int ns, int b, int P, int m, int nmat, const double* __restrict__ band_val,
                             const cplx* __restrict__ zs, const double* __restrict__ wp_f, const C* __restrict__ fac,
                             const C* __restrict__ facT, C* __restrict__ Vsp, C* __restrict__ Wsp) {
  extern __shared__ __align__(16) unsigned char ssm_raw[];
  C* ssm = reinterpret_cast<C*>(ssm_raw);
  const int col = blockIdx.x % (2 * b);
  const int j = (blockIdx.x / (2 * b)) % P;
  const int f = blockIdx.x / (2 * b * P);
  const int s0 = j * m, e0 = (j == P - 1) ? n : min(n, s0 + m);
  const int mm = e0 - s0;
  const int lane = threadIdx.x;
  const int nb1 = b + 1;
  const size_t stride = (size_t)n * nb1;
  const cplx* z = zs + (size_t)f * nmat;
  const double wp = wp_f[f];
  const bool isV = col < b;
  const int c = isV ? col : col - b;
  if (isV ? (j == P - 1) : (j == 0)) return;
  C* x = (isV ? Vsp : Wsp) + ((size_t)f * b + c) * ns + s0;
  for (int i = lane; i < mm; i += 32) {
    cplx v = make_double2(0.0, 0.0);
    if (isV) {
      const int r = i - (mm - b);
      if (r >= c && r < b) v = pencil(band_val + (size_t)(e0 + c) * nb1 + (r - c), stride, nmat, z, wp);
    } else {
      const int r = i;
      if (r <= c) v = pencil(band_val + (size_t)(s0 + r) * nb1 + (c - r), stride, nmat, z, wp);
    }
    x[i] = to_c<C>(v);
  }
  __syncwarp();
  const int rs = band_rs<C>(b);
  const size_t fo = ((size_t)f * n + s0) * rs;
  band_solve_warp<C>(mm, b, rs, facT + fo, fac + fo, x, ssm);
}

// In-place inverse of the n x n complex matrix A (row-major, leading dimension
// lda, shared memory) by Gauss-Jordan elimination with partial pivoting; all
// threads of the CTA.  piv: n ints of shared memory, colk: n elements.
template <class C>
__device__ void gj_inverse(C* A, int n, int lda, int* piv, C* colk, C* pinv_s) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      int p = k;
      auto best = cabs2T(A[k * lda + k]);
      for (int i = k + 1; i < n; ++i) {
        auto v = cabs2T(A[i * lda + k]);
        if (v > best) {
          best = v;
          p = i;
        }
      }
      piv[k] = p;
    }
    __syncthreads();
    const int p = piv[k];
    if (p != k)
      for (int cc = tid; cc < n; cc += nt) {
        C t = A[k * lda + cc];
        A[k * lda + cc] = A[p * lda + cc];
        A[p * lda + cc] = t;
      }
    __syncthreads();
    if (tid == 0) *pinv_s = crecipT(A[k * lda + k]);
    for (int i = tid; i < n; i += nt) colk[i] = A[i * lda + k];
    __syncthreads();
    const C pinv = *pinv_s;
    for (int cc = tid; cc < n; cc += nt) A[k * lda + cc] = cmul(cc == k ? cone<C>() : A[k * lda + cc], pinv);
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, cc = e % n;
      if (i == k) continue;
      const C a = cc == k ? czero<C>() : A[i * lda + cc];
      A[i * lda + cc] = csubT(a, cmul(A[k * lda + cc], colk[i]));
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < n; i += nt) {
        C t = A[i * lda + k];
        A[i * lda + k] = A[i * lda + p];
        A[i * lda + p] = t;
      }
    __syncthreads();
  }
}

// The same inverse by one warp for n <= 32: lane r owns row r in the
// elimination, the lanes span the columns in the row swaps and the scaling;
// warp-synchronous (no block barriers).  Called by warp 0 only.
template <class C>
__device__ void gj_inverse_warp(C* A, int n, int lda, int* piv) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < n; ++k) {
    auto best = (lane >= k && lane < n) ? cabs2T(A[lane * lda + k]) : decltype(cabs2T(A[0]))(-1);
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const auto ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ob > best || (ob == best && oi < idx)) {
        best = ob;
        idx = oi;
      }
    }
    const int p = idx;
    if (lane == 0) piv[k] = p;
    if (p != k)
      for (int cc = lane; cc < n; cc += 32) {
        C t = A[k * lda + cc];
        A[k * lda + cc] = A[p * lda + cc];
        A[p * lda + cc] = t;
      }
    __syncwarp();
    const C pinv = crecipT(A[k * lda + k]);
    const C colk = lane < n ? A[lane * lda + k] : czero<C>();
    __syncwarp();
    for (int cc = lane; cc < n; cc += 32) A[k * lda + cc] = cmul(cc == k ? cone<C>() : A[k * lda + cc], pinv);
    __syncwarp();
    if (lane < n && lane != k)
      for (int cc = 0; cc < n; ++cc) {
        const C a = cc == k ? czero<C>() : A[lane * lda + cc];
        A[lane * lda + cc] = csubT(a, cmul(A[k * lda + cc], colk));
      }
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int r = lane; r < n; r += 32) {
        C t = A[r * lda + k];
        A[r * lda + k] = A[r * lda + p];
        A[r * lda + p] = t;
      }
    __syncwarp();
  }
}

// Block LU of the reduced system, one CTA per frequency, sequential over j:
// record R[f][j] (6 b^2 elements) = [E^_j^-1 (2b x 2b, column-major) |
// W_j^bot ([c][r], zero for j = 0) | V_{j+1}^top ([c][r], zero for j = P-2)],
// everything one step of the reduced substitution reads.
template <class C>
__global__ void k_spike_reduce(int ns, int b, int P, int m, const C* __restrict__ Vsp, const C* __restrict__ Wsp,
                               C* __restrict__ R) {
  extern __shared__ __align__(16) unsigned char rsm_raw[];
  C* E = reinterpret_cast<C*>(rsm_raw);   // [B2][B2 + 1]: odd row stride, no bank conflicts by row
  const int B2 = 2 * b, ld = 2 * b + 1;
  C* X01 = E + B2 * ld;        // [b][b] top-right block of the previous inverse
  C* T = X01 + b * b;          // [b][b]
  C* colk = T + b * b;         // [B2]
  C* pinv = colk + B2;         // [1]
  int* piv = reinterpret_cast<int*>(pinv + 1);
  const int f = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const C* V = Vsp + (size_t)f * b * ns;
  const C* W = Wsp + (size_t)f * b * ns;
  const size_t RS = (size_t)6 * b * b;
  for (int j = 0; j + 1 < P; ++j) {
    const int sj = j * m, e = (j + 1) * m;
    for (int q = tid; q < B2 * B2; q += nt) {
      const int r = q / B2, cc = q % B2;
      C v = r == cc ? cone<C>() : czero<C>();
      if (r < b && cc >= b) v = V[(size_t)(cc - b) * ns + e - b + r];
      if (r >= b && cc < b) v = W[(size_t)cc * ns + e + (r - b)];
      E[r * ld + cc] = v;
    }
    if (j > 0) {
      // T = X01 V_j^top, then E_tr -= W_j^bot T
      for (int q = tid; q < b * b; q += nt) {
        const int r = q / b, cc = q % b;
        C acc = czero<C>();
        for (int k = 0; k < b; ++k) acc = cfma(X01[r * b + k], V[(size_t)cc * ns + sj + k], acc);
        T[q] = acc;
      }
      __syncthreads();
      for (int q = tid; q < b * b; q += nt) {
        const int r = q / b, cc = q % b;
        C acc = czero<C>();
        for (int k = 0; k < b; ++k) acc = cfma(W[(size_t)k * ns + e - b + r], T[k * b + cc], acc);
        E[r * ld + b + cc] = csubT(E[r * ld + b + cc], acc);
      }
    }
    __syncthreads();
    if (B2 <= 32) {
      if (tid < 32) gj_inverse_warp<C>(E, B2, ld, piv);
      __syncthreads();
    } else {
      gj_inverse<C>(E, B2, ld, piv, colk, pinv);
    }
    C* out = R + ((size_t)f * (P - 1) + j) * RS;
    for (int q = tid; q < B2 * B2; q += nt) {
      const int r = q / B2, cc = q % B2;
      out[(size_t)cc * B2 + r] = E[r * ld + cc];
    }
    for (int q = tid; q < b * b; q += nt) {
      const int cc = q / b, r = q % b;
      out[(size_t)4 * b * b + q] = j > 0 ? W[(size_t)cc * ns + e - b + r] : czero<C>();
      out[(size_t)5 * b * b + q] = j + 2 < P ? V[(size_t)cc * ns + e + r] : czero<C>();
    }
    for (int q = tid; q < b * b; q += nt) X01[q] = E[(q / b) * ld + b + q % b];
    __syncthreads();
  }
}

__global__ void k_to_f32(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ---- partitioned (SPIKE) apply ---------------------------------------------------------------
// Stage 1: y_j = A_j^-1 f_j for block j = blockIdx.y.  mode 0: the right-hand
// side is v[s][perm[i]] of system s (two systems sharing a frequency per warp
// when `pair`), stored in x[s] (stride xs); mode 1: it is column g of Q_vg(f),
// s = f * ng + g, solved in place in x = Wb.
template <class C>
__global__ void k_spike_y(int n, int b, int P, int m, int nper, int pair, int mode, int nloop, int ng, int nmat,
                          const int32_t* __restrict__ perm, const double* __restrict__ border_vg,
                          const cplx* __restrict__ zs, const double* __restrict__ wp_f, const C* __restrict__ fac,
                          const C* __restrict__ facT, const cplx* __restrict__ v, C* __restrict__ xb, size_t xs,
                          const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char ysm_raw[];
  C* ysm = reinterpret_cast<C*>(ysm_raw);
  const int lane = threadIdx.x;
  const int s0 = pair ? 2 * blockIdx.x : blockIdx.x;
  if (active && !active[s0] && (!pair || !active[s0 + 1])) return;
  const int f = s0 / nper, j = blockIdx.y;
  const int j0 = j * m, e0 = (j == P - 1) ? n : min(n, j0 + m);
  const int mm = e0 - j0;
  for (int q = 0; q < (pair ? 2 : 1); ++q) {
    C* x = xb + (size_t)(s0 + q) * xs + j0;
    if (mode == 0) {
      const cplx* vs = v + (size_t)(s0 + q) * nloop;
      for (int i = lane; i < mm; i += 32) x[i] = to_c<C>(vs[perm[j0 + i]]);
    } else {
      const int g = (s0 + q) % ng;
      const size_t vstride = (size_t)n * ng;
      for (int i = lane; i < mm; i += 32)
        x[i] = to_c<C>(pencil(border_vg + (size_t)(j0 + i) * ng + g, vstride, nmat, zs + (size_t)f * nmat, wp_f[f]));
    }
  }
  __syncwarp();
  const int rs = band_rs<C>(b);
  const size_t fo = ((size_t)f * n + j0) * rs;
  C* x0 = xb + (size_t)s0 * xs + j0;
  if (pair)
    band_solve_pair<C>(mm, b, rs, facT + fo, fac + fo, x0, x0 + xs, ysm);
  else
    band_solve_warp<C>(mm, b, rs, facT + fo, fac + fo, x0, ysm);
}

// cp.async of `bytes` (a multiple of 16) from global to shared memory by one warp
__device__ __forceinline__ void warp_copy_async(void* dst, const void* src, size_t bytes) {
  const int lane = threadIdx.x & 31;
  char* d = reinterpret_cast<char*>(dst);
  const char* g = reinterpret_cast<const char*>(src);
  for (size_t o = 16 * (size_t)lane; o < bytes; o += 32 * 16) cp_async16(d + o, g + o);
  cp_commit();
}

// Stage 2: the reduced block-tridiagonal system for z_j = (u_j, t_{j+1}),
// forward then backward; one CTA of four warps per system.  All interface rows
// of x and h_j (then z_j) live in shared memory (h is written to hb[s][j][2b]
// at the end); the records R[f][j] stream through a ring of kZDepth buffers
// with cp.async issued by warp 0 (one commit group per step, empty at the
// tail), so a step waits on shared memory only.  Each 2b x 2b product of a
// step is split over 128 threads: row r = tid % 64, column half tid / 64,
// partial sums combined through shared memory (2b <= 48).  kZDepth = 4, or 2
// where four records do not fit.
template <class C, int kZDepth>
__global__ void __launch_bounds__(128) k_spike_z(int n, int b, int P, int m, int nper, const C* __restrict__ R,
                                                 const C* __restrict__ xb, size_t xs, C* __restrict__ hb,
                                                 const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char zsm_raw[];
  const int B2 = 2 * b;
  const size_t RS = (size_t)6 * b * b;
  C* rbuf = reinterpret_cast<C*>(zsm_raw);   // [kZDepth][6 b^2]
  C* hs = rbuf + kZDepth * RS;               // [(P-1)][2b]
  C* gs = hs + (size_t)(P - 1) * B2;         // [(P-1)][2b] interface rows of x
  __shared__ C hp[32], tt[32], part[128];
  const int s = blockIdx.x;
  if (P < 2 || (active && !active[s])) return;
  const int f = s / nper, tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & 63, half = tid >> 6;
  const int nst = P - 1;
  const C* Rf = R + (size_t)f * nst * RS;
  const C* x = xb + (size_t)s * xs;
  C* h = hb + (size_t)s * nst * B2;
  // forward records 0 .. kZDepth-2 in flight, one group each
  if (warp == 0)
    for (int q = 0; q < kZDepth - 1; ++q) {
      if (q < nst) warp_copy_async(rbuf + (size_t)(q % kZDepth) * RS, Rf + (size_t)q * RS, RS * sizeof(C));
      else cp_commit();
    }
  for (int e = tid; e < nst * B2; e += blockDim.x) {
    const int j = e / B2, rr = e % B2;
    gs[e] = x[(j + 1) * m - b + rr];
  }
  for (int j = 0; j < nst; ++j) {
    // keep kZDepth - 1 groups ahead: issue record j + kZDepth - 1 (or an empty group)
    if (warp == 0) {
      const int jn = j + kZDepth - 1;
      if (jn < nst) warp_copy_async(rbuf + (size_t)(jn % kZDepth) * RS, Rf + (size_t)jn * RS, RS * sizeof(C));
      else cp_commit();
      asm volatile("cp.async.wait_group %0;\n" ::"n"(kZDepth - 1) : "memory");
    }
    __syncthreads();
    const C* Ej = rbuf + (size_t)(j % kZDepth) * RS;
    const C* Wj = Ej + 4 * b * b;
    C* g = gs + j * B2;
    if (j > 0 && tid < b) {
      C acc = czero<C>();
      for (int c = 0; c < b; ++c) acc = cfma(Wj[c * b + tid], hp[c], acc);
      g[tid] = csubT(g[tid], acc);
    }
    __syncthreads();
    {
      C a0 = czero<C>(), a1 = czero<C>();
      if (r < B2) {
        const int c0 = half * b;
        int c = 0;
        for (; c + 2 <= b; c += 2) {
          a0 = cfma(Ej[(c0 + c) * B2 + r], g[c0 + c], a0);
          a1 = cfma(Ej[(c0 + c + 1) * B2 + r], g[c0 + c + 1], a1);
        }
        for (; c < b; ++c) a0 = cfma(Ej[(c0 + c) * B2 + r], g[c0 + c], a0);
      }
      part[tid] = caddT(a0, a1);
    }
    __syncthreads();
    if (tid < B2) {
      const C acc = caddT(part[tid], part[64 + tid]);
      hs[j * B2 + tid] = acc;
      if (tid < b) hp[tid] = acc;
    }
  }
  if (warp == 0) cp_wait_all();
  __syncthreads();
  if (nst >= 2) {
    // backward over j = nst - 2 .. 0 (record j), the same ring
    const int nb = nst - 1;
    if (warp == 0)
      for (int q = 0; q < kZDepth - 1; ++q) {
        if (q < nb) warp_copy_async(rbuf + (size_t)(q % kZDepth) * RS, Rf + (size_t)(nb - 1 - q) * RS, RS * sizeof(C));
        else cp_commit();
      }
    for (int q = 0; q < nb; ++q) {
      const int j = nb - 1 - q;
      if (warp == 0) {
        const int qn = q + kZDepth - 1;
        if (qn < nb) warp_copy_async(rbuf + (size_t)(qn % kZDepth) * RS, Rf + (size_t)(nb - 1 - qn) * RS, RS * sizeof(C));
        else cp_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kZDepth - 1) : "memory");
      }
      __syncthreads();
      const C* Ej = rbuf + (size_t)(q % kZDepth) * RS;
      const C* Vt = Ej + 5 * b * b;
      const C* zn = hs + (j + 1) * B2 + b;
      if (tid < b) {
        C acc = czero<C>();
        for (int c = 0; c < b; ++c) acc = cfma(Vt[c * b + tid], zn[c], acc);
        tt[tid] = acc;
      }
      __syncthreads();
      {
        C a0 = czero<C>();
        if (r < B2) {
          const int c0 = half * ((b + 1) / 2), c1 = half ? b : (b + 1) / 2;
          for (int c = c0; c < c1; ++c) a0 = cfma(Ej[(size_t)(b + c) * B2 + r], tt[c], a0);
        }
        part[tid] = a0;
      }
      __syncthreads();
      if (tid < B2) hs[j * B2 + tid] = csubT(hs[j * B2 + tid], caddT(part[tid], part[64 + tid]));
    }
    if (warp == 0) cp_wait_all();
  }
  __syncthreads();
  for (int e = tid; e < nst * B2; e += blockDim.x) h[e] = hs[e];
}

constexpr int kSpikeRows = 1024;   // rows per CTA of the correction kernels

// Stage 3a: x_j = y_j - V_j t_{j+1} - W_j u_{j-1} in place for rows
// [blockIdx.y * kSpikeRows, +kSpikeRows) of system blockIdx.x; in mode 0 also
// the partial border sums part[s][chunk][g] = sum_i Q_vg[i][g] x_i.
template <class C>
__global__ void __launch_bounds__(256) k_spike_x(int n, int ns, int b, int P, int m, int nper, int mode, int ng,
                                                 int nmat,
                                                 const double* __restrict__ border_vg, const cplx* __restrict__ zs,
                                                 const double* __restrict__ wp_f, const C* __restrict__ Vsp,
                                                 const C* __restrict__ Wsp, const C* __restrict__ hb,
                                                 C* __restrict__ xb, size_t xs, cplx* __restrict__ part,
                                                 const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char xsm_raw[];
  C* hs = reinterpret_cast<C*>(xsm_raw);   // [(P-1)][2b]
  __shared__ cplx red[8][kMaxBorder];
  const int s = blockIdx.x;
  if (active && !active[s]) return;
  const int f = s / nper, tid = threadIdx.x, B2 = 2 * b;
  const int i0 = blockIdx.y * kSpikeRows, i1 = min(n, i0 + kSpikeRows);
  C* x = xb + (size_t)s * xs;
  if (P > 1) {
    const C* V = Vsp + (size_t)f * b * ns;
    const C* W = Wsp + (size_t)f * b * ns;
    for (int e = tid; e < (P - 1) * B2; e += blockDim.x) hs[e] = hb[(size_t)s * (P - 1) * B2 + e];
    __syncthreads();
    for (int i = i0 + tid; i < i1; i += blockDim.x) {
      const int j = min(i / m, P - 1);
      C y = x[i];
      if (j < P - 1) {
        const C* t = hs + j * B2 + b;
        for (int c = 0; c < b; ++c) y = csubT(y, cmul(V[(size_t)c * ns + i], t[c]));
      }
      if (j > 0) {
        const C* u = hs + (j - 1) * B2;
        for (int c = 0; c < b; ++c) y = csubT(y, cmul(W[(size_t)c * ns + i], u[c]));
      }
      x[i] = y;
    }
  }
  if (mode == 1 || ng == 0) return;
  const cplx* zf = zs + (size_t)f * nmat;
  const double wp = wp_f[f];
  const size_t vstride = (size_t)n * ng;
  cplx acc[kMaxBorder];
  for (int g = 0; g < ng; ++g) acc[g] = make_double2(0.0, 0.0);
  for (int i = i0 + tid; i < i1; i += blockDim.x) {
    const cplx xi = to_d(x[i]);
    for (int g = 0; g < ng; ++g)
      acc[g] = cadd(acc[g], cm(pencil(border_vg + (size_t)i * ng + g, vstride, nmat, zf, wp), xi));
  }
  const int w = tid >> 5, lane = tid & 31;
  for (int g = 0; g < ng; ++g) {
    cplx t = warp_sum(acc[g]);
    if (lane == 0) red[w][g] = t;
  }
  __syncthreads();
  if (tid < ng) {
    cplx t = make_double2(0.0, 0.0);
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = cadd(t, red[q][tid]);
    part[((size_t)s * gridDim.y + blockIdx.y) * ng + tid] = t;
  }
}

// Stage 3b (mode 0): t_g = v_g - sum of the partial border sums, z_g = S^-1 t_g,
// then z[s][perm[i]] = x_i - sum_g W_b[g][i] z_g and z[s][n + g] = z_g.
template <class C>
__global__ void __launch_bounds__(256) k_spike_out(int n, int nper, int nloop, int ng, int nchunk,
                                                   const int32_t* __restrict__ perm, const C* __restrict__ xb,
                                                   size_t xs, const cplx* __restrict__ part,
                                                   const cplx* __restrict__ Wb, const cplx* __restrict__ Sinv,
                                                   const cplx* __restrict__ v, cplx* __restrict__ z,
                                                   const int* __restrict__ active) {
  __shared__ cplx tg[kMaxBorder], zg[kMaxBorder];
  const int s = blockIdx.x;
  if (active && !active[s]) return;
  const int f = s / nper, tid = threadIdx.x;
  const int i0 = blockIdx.y * kSpikeRows, i1 = min(n, i0 + kSpikeRows);
  const C* x = xb + (size_t)s * xs;
  cplx* zo = z + (size_t)s * nloop;
  if (ng > 0) {
    if (tid < ng) {
      cplx t = make_double2(0.0, 0.0);
      for (int q = 0; q < nchunk; ++q) t = cadd(t, part[((size_t)s * nchunk + q) * ng + tid]);
      tg[tid] = csub(v[(size_t)s * nloop + n + tid], t);
    }
    __syncthreads();
    if (tid < ng) {
      cplx t = make_double2(0.0, 0.0);
      for (int g2 = 0; g2 < ng; ++g2) t = cadd(t, cm(Sinv[((size_t)f * ng + tid) * ng + g2], tg[g2]));
      zg[tid] = t;
      if (blockIdx.y == 0) zo[n + tid] = t;
    }
    __syncthreads();
  }
  for (int i = i0 + tid; i < i1; i += blockDim.x) {
    cplx a = to_d(x[i]);
    for (int g = 0; g < ng; ++g) a = csub(a, cm(Wb[((size_t)f * ng + g) * n + i], zg[g]));
    zo[perm[i]] = a;
  }
}

// ---- host ---------------------------------------------------------------------------------
bool band_fits(int band, int n_border) { return band <= kMaxBand && n_border <= kMaxBorder; }

bool band_usable(const xrl_ctx* c) { return band_fits(c->topo.band, c->topo.n_border) && c->topo.n_band > 0; }

void band_prepare(xrl_ctx* c) {
  const Topo& T = c->topo;
  c->d.band_perm.upload(c->alloc, T.band_perm);
  c->d.band_val.upload(c->alloc, T.band_val);
  c->d.border_vg.upload(c->alloc, T.border_vg);
  c->d.border_gg.upload(c->alloc, T.border_gg);
}

// Blocks of m rows (even, >= 4b; the last block takes the remainder and has
// at least 2b rows), at most 64 of them; one block (the plain band solve) for
// short bands or b > 24 (the reduced substitution keeps two 6 b^2 records in
// shared memory).
static void band_blocks(int n, int b, int* P, int* m) {
  const int pm = 64;
  if (n < 8 * b || b > 24) {
    *P = 1;
    *m = n;
    return;
  }
  int mm = std::max(4 * b, (n + pm - 1) / pm);
  mm = (mm + 1) & ~1;
  int p = (n + mm - 1) / mm;
  if (n - (p - 1) * mm < 2 * b) --p;
  *P = std::max(1, p);
  *m = *P == 1 ? n : mm;
}

static size_t spike_stride(int n) { return (size_t)((n + 1) & ~1); }

void band_alloc(xrl_ctx* c, BandWork& bw, int nf, int nsys, bool mixed) {
  const Topo& T = c->topo;
  const int n = T.n_band, b = T.band, ng = T.n_border;
  band_blocks(n, b, &bw.P, &bw.m);
  bw.nf = nf;
  bw.mixed = mixed;
  const int P1 = std::max(1, bw.P - 1);
  const size_t ns = spike_stride(n);
  const size_t xs = (size_t)((n + 2) & ~1);
  const int nchunk = (n + kSpikeRows - 1) / kSpikeRows;
  const size_t nsb = (size_t)std::max(nsys, nf * std::max(1, ng));   // systems of either solve
  bw.fac.alloc(c->alloc, (size_t)nf * n * (b + 1));
  bw.facT.alloc(c->alloc, (size_t)nf * n * (b + 1));
  bw.Wb.alloc(c->alloc, (size_t)nf * std::max(1, ng) * n);
  bw.Sinv.alloc(c->alloc, (size_t)nf * std::max(1, ng * ng));
  bw.part.alloc(c->alloc, (size_t)nsys * nchunk * std::max(1, ng));
  if (mixed) {
    const int rs = band_rs<float2>(b);
    bw.fac32.alloc(c->alloc, (size_t)nf * n * rs);
    bw.facT32.alloc(c->alloc, (size_t)nf * n * rs);
    if (bw.P > 1) {
      bw.Vsp32.alloc(c->alloc, (size_t)nf * b * ns);
      bw.Wsp32.alloc(c->alloc, (size_t)nf * b * ns);
      bw.R32.alloc(c->alloc, (size_t)nf * P1 * 6 * b * b);
    }
    if (ng > 0) bw.Wb32.alloc(c->alloc, (size_t)nf * ng * xs);
    bw.scr32.alloc(c->alloc, (size_t)nsys * xs);
    bw.hb32.alloc(c->alloc, nsb * P1 * 2 * b);
  } else {
    if (bw.P > 1) {
      bw.Vsp.alloc(c->alloc, (size_t)nf * b * ns);
      bw.Wsp.alloc(c->alloc, (size_t)nf * b * ns);
      bw.R.alloc(c->alloc, (size_t)nf * P1 * 6 * b * b);
    }
    bw.scr.alloc(c->alloc, (size_t)nsys * xs);
    bw.hb.alloc(c->alloc, nsb * P1 * 2 * b);
  }
}

// the three (mode 1) or four (mode 0) stages of one partitioned solve
template <class C>
static int spike_stages(xrl_ctx* c, const BandWork& bw, int nsys, int nper, int mode, const cplx* zs,
                        const double* wp, const C* fac, const C* facT, const C* Vsp, const C* Wsp, const C* R, C* xb,
                        size_t xs, C* hb, const cplx* v, cplx* z, const int* active, cudaStream_t s) {
  const Topo& T = c->topo;
  const int n = T.n_band, b = T.band, ng = T.n_border, P = bw.P, m = bw.m;
  const int nchunk = (n + kSpikeRows - 1) / kSpikeRows;
  const bool pair = mode == 0 && b <= 15 && nper % 2 == 0 && nsys % 2 == 0;
  const int ch = band_chunk(b);
  int launches = 0;
  const size_t ys = pair ? sizeof(C) * ((size_t)2 * ch * band_rs<C>(b) + 4 * (size_t)ch) : band_smem_bytes<C>(b);
  if (ys > 48 * 1024)
    XRL_CUDA(cudaFuncSetAttribute(k_spike_y<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ys));
  k_spike_y<C><<<dim3(pair ? nsys / 2 : nsys, P), 32, ys, s>>>(n, b, P, m, nper, pair ? 1 : 0, mode, T.n_loops, ng,
                                                              T.n_mat, c->d.band_perm.p, c->d.border_vg.p, zs, wp, fac,
                                                              facT, v, xb, xs, active);
  ++launches;
  if (P > 1) {
    const size_t rec = sizeof(C) * (size_t)6 * b * b, side = sizeof(C) * 2 * (size_t)(P - 1) * 2 * b;
    const bool deep = 4 * rec + side <= 200 * 1024;
    const size_t zsm = (deep ? 4 : 2) * rec + side;
    if (deep) {
      if (zsm > 48 * 1024)
        XRL_CUDA(cudaFuncSetAttribute(k_spike_z<C, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
      k_spike_z<C, 4><<<nsys, 128, zsm, s>>>(n, b, P, m, nper, R, xb, xs, hb, active);
    } else {
      if (zsm > 48 * 1024)
        XRL_CUDA(cudaFuncSetAttribute(k_spike_z<C, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
      k_spike_z<C, 2><<<nsys, 128, zsm, s>>>(n, b, P, m, nper, R, xb, xs, hb, active);
    }
    ++launches;
  }
  if (P > 1 || (mode == 0 && ng > 0)) {
    const size_t hs = sizeof(C) * (size_t)std::max(1, P - 1) * 2 * b;
    k_spike_x<C><<<dim3(nsys, nchunk), 256, hs, s>>>(n, (int)spike_stride(n), b, P, m, nper, mode, ng, T.n_mat,
                                                     c->d.border_vg.p, zs, wp, Vsp, Wsp, hb, xb, xs, bw.part.p,
                                                     active);
    ++launches;
  }
  if (mode == 0) {
    k_spike_out<C><<<dim3(nsys, nchunk), 256, 0, s>>>(n, nper, T.n_loops, ng, nchunk, c->d.band_perm.p, xb, xs,
                                                      bw.part.p, bw.Wb.p, bw.Sinv.p, v, z, active);
    ++launches;
  }
  XRL_CUDA(cudaGetLastError());
  return launches;
}

__global__ void k_wb_to_f64(size_t n, size_t xs, size_t tot, const float2* __restrict__ a, cplx* __restrict__ o) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tot) return;
  const size_t q = e / n, i = e % n;
  const float2 v = a[q * xs + i];
  o[e] = make_double2(v.x, v.y);
}

template <class C>
static int spike_factor(xrl_ctx* c, BandWork& bw, const cplx* zs, const double* wp, const C* fac, const C* facT,
                        C* Vsp, C* Wsp, C* R, cudaStream_t s) {
  const Topo& T = c->topo;
  const int n = T.n_band, b = T.band, nf = bw.nf, P = bw.P, m = bw.m;
  const size_t ns = spike_stride(n);
  const size_t bsd = band_smem_bytes<C>(b);
  if (bsd > 48 * 1024)
    XRL_CUDA(cudaFuncSetAttribute(k_spike_cols<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsd));
  k_spike_cols<C><<<nf * P * 2 * b, 32, bsd, s>>>(n, (int)ns, b, P, m, T.n_mat, c->d.band_val.p, zs, wp, fac,
                                                  facT, Vsp, Wsp);
  const size_t rsm = sizeof(C) * ((size_t)2 * b * (2 * b + 1) + 2 * (size_t)b * b + 2 * b + 1) + sizeof(int) * 2 * b;
  if (rsm > 48 * 1024)
    XRL_CUDA(cudaFuncSetAttribute(k_spike_reduce<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
  k_spike_reduce<C><<<nf, 256, rsm, s>>>((int)ns, b, P, m, Vsp, Wsp, R);
  return 2;
}

// factor Q(f) for bw.nf frequencies (zs [nf][nmat], wp [nf])
void band_factor(xrl_ctx* c, BandWork& bw, const cplx* zs, const double* wp, cudaStream_t s) {
  const Topo& T = c->topo;
  const int n = T.n_band, b = T.band, ng = T.n_border, nf = bw.nf, P = bw.P, m = bw.m;
  const int nb1 = b + 1;
  cudaEvent_t ev = prof_begin(c, s);
  size_t smem = sizeof(cplx) * ((size_t)nb1 * nb1 + b) + sizeof(short2) * (size_t)b * nb1 / 2 + 16;
  if (smem > 48 * 1024)
    XRL_CUDA(cudaFuncSetAttribute(k_band_factor_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_band_factor_blk<<<nf * P, 32, smem, s>>>(n, b, P, m, T.n_mat, c->d.band_val.p, zs, wp, bw.fac.p);
  int launches = 1;
  {
    size_t tot = (size_t)nf * n * nb1;
    k_band_finish<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nf, n, b, bw.fac.p, bw.facT.p, bw.fac32.p,
                                                                bw.facT32.p);
    ++launches;
  }
  // spikes and the reduced system: FP32 from the FP32 factor copies when the
  // solves run in FP32 (the preconditioner only needs to be close to Q^-1)
  if (P > 1)
    launches += bw.mixed ? spike_factor<float2>(c, bw, zs, wp, bw.fac32.p, bw.facT32.p, bw.Vsp32.p, bw.Wsp32.p,
                                                bw.R32.p, s)
                         : spike_factor<cplx>(c, bw, zs, wp, bw.fac.p, bw.facT.p, bw.Vsp.p, bw.Wsp.p, bw.R.p, s);
  if (ng > 0) {
    // W_b = Q_vv^-1 Q_vg, one "system" per (f, g)
    if (bw.mixed) {
      const size_t xs = (size_t)((n + 2) & ~1);
      launches += spike_stages<float2>(c, bw, nf * ng, ng, 1, zs, wp, bw.fac32.p, bw.facT32.p, bw.Vsp32.p,
                                       bw.Wsp32.p, bw.R32.p, bw.Wb32.p, xs, bw.hb32.p, nullptr, nullptr, nullptr, s);
      const size_t tot = (size_t)nf * ng * n;
      k_wb_to_f64<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((size_t)n, xs, tot, bw.Wb32.p, bw.Wb.p);
      ++launches;
    } else {
      launches += spike_stages<cplx>(c, bw, nf * ng, ng, 1, zs, wp, bw.fac.p, bw.facT.p, bw.Vsp.p, bw.Wsp.p,
                                     bw.R.p, bw.Wb.p, (size_t)n, bw.hb.p, nullptr, nullptr, nullptr, s);
    }
    k_schur<<<nf, 256, 0, s>>>(n, ng, T.n_mat, c->d.border_vg.p, c->d.border_gg.p, zs, wp, bw.Wb.p, bw.Sinv.p);
    ++launches;
  }
  prof_end(c, s, ev, PH_PREC, launches, 8.0 * nf * (double)n * b * b / 2.0, 16.0 * nf * (double)n * (b + 1) * 2.0);
  XRL_CUDA(cudaGetLastError());
}

// z = Q(f_s)^-1 v for nsys systems, f_s = s / nport (loop order in and out)
void band_apply(xrl_ctx* c, BandWork& bw, int nsys, int nport, const cplx* zs, const double* wp, const cplx* v,
                cplx* z, const int* active, cudaStream_t s) {
  const Topo& T = c->topo;
  cudaEvent_t ev = prof_begin(c, s);
  const size_t xs = (size_t)((T.n_band + 2) & ~1);
  int launches;
  if (bw.mixed)
    launches = spike_stages<float2>(c, bw, nsys, nport, 0, zs, wp, bw.fac32.p, bw.facT32.p, bw.Vsp32.p, bw.Wsp32.p,
                                    bw.R32.p, bw.scr32.p, xs, bw.hb32.p, v, z, active, s);
  else
    launches = spike_stages<cplx>(c, bw, nsys, nport, 0, zs, wp, bw.fac.p, bw.facT.p, bw.Vsp.p, bw.Wsp.p, bw.R.p,
                                  bw.scr.p, xs, bw.hb.p, v, z, active, s);
  const double es = bw.mixed ? 8.0 : 16.0;
  prof_end(c, s, ev, PH_PREC, launches, 16.0 * nsys * (double)T.n_band * T.band * (bw.P > 1 ? 3 : 1),
           es * nsys * (double)T.n_band * (2.0 * T.band + 4.0));
}

}  // namespace xrl
