// Fast multipole product y = P x on panels (Sec. II-C), sm_103a.
//
// The centroid-midpoint transformation turns each product into scalar 1/R
// potentials of panels, "the format of particle simulation" (Sec. II-C):
// source panel l carries the uniform charge density x_l / A_l and target k
// averages the potential over its area.  Phases per product, all on one
// stream, panels in Morton order with columns contiguous ([N][nc] layout):
//   P2P  near field of each leaf from the precomputed U-list blocks
//   P2M  leaf multipoles from the exact panel moments (setup, geom.cu)
//   M2M  upward, levels L-1 .. 2 (8 child-offset matrices)
//   M2L  V-list translations (offset-indexed matrices, level independent)
//   L2L  downward, levels 3 .. L
//   L2P  leaf locals averaged over the target panels (same moment table,
//        weight 1 for m = 0 and 2 for m > 0 of the real storage)
// Operators are real (p+1)^2 square matrices stored transposed ([in][out]).
// The template parameter T selects FP64 (the plain path) or FP32 (mixed
// precision, used inside the FP64 refinement loop).
#include <algorithm>
#include <vector>

#include "xrl_internal.hpp"

namespace xrl {

// ---- layout conversion ----------------------------------------------------------------
template <class T>
__global__ void k_to_morton(int N, int nc, const int32_t* __restrict__ perm, const T* __restrict__ x,
                            T* __restrict__ X) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * nc) return;
  int r = (int)(idx / nc), c = (int)(idx % nc);
  X[idx] = x[(size_t)c * N + perm[r]];
}

template <class T>
__global__ void k_from_morton(int N, int nc, const int32_t* __restrict__ perm, const T* __restrict__ Y,
                              T* __restrict__ y) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * nc) return;
  int r = (int)(idx / nc), c = (int)(idx % nc);
  y[(size_t)c * N + perm[r]] = Y[idx];
}

void launch_to_morton(const xrl_ctx* c, int nc, const double* x, double* X, cudaStream_t s) {
  size_t n = (size_t)c->N * nc;
  count_launch(const_cast<xrl_ctx*>(c));
  k_to_morton<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->N, nc, c->d.perm.p, x, X);
}

void launch_from_morton(const xrl_ctx* c, int nc, const double* Y, double* y, cudaStream_t s) {
  size_t n = (size_t)c->N * nc;
  count_launch(const_cast<xrl_ctx*>(c));
  k_from_morton<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->N, nc, c->d.perm.p, Y, y);
}

void launch_to_morton32(const xrl_ctx* c, int nc, const float* x, float* X, cudaStream_t s) {
  size_t n = (size_t)c->N * nc;
  count_launch(const_cast<xrl_ctx*>(c));
  k_to_morton<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->N, nc, c->d.perm.p, x, X);
}

void launch_from_morton32(const xrl_ctx* c, int nc, const float* Y, float* y, cudaStream_t s) {
  size_t n = (size_t)c->N * nc;
  count_launch(const_cast<xrl_ctx*>(c));
  k_from_morton<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->N, nc, c->d.perm.p, Y, y);
}

// ---- near field -------------------------------------------------------------------------
// One block per (leaf, column tile).  Thread t handles target ii = t / ct and
// column c0 + t % ct of the tile; the block walks the leaf's U-list.
template <class T>
__global__ void k_p2p(int nc, int ct, const int32_t* __restrict__ leaf_first, const int32_t* __restrict__ leaf_count,
                      const int32_t* __restrict__ u_ptr, const int32_t* __restrict__ u_src,
                      const int64_t* __restrict__ near_off, const int32_t* __restrict__ near_w,
                      const T* __restrict__ val, const T* __restrict__ X, T* __restrict__ Y) {
  const int B = blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const int nB = leaf_count[B], f0 = leaf_first[B], w = near_w[B];
  const T* vb = val + near_off[B];
  // U-lists have no fixed length (the bounding-sphere rule can make them
  // long): their entries are read from global memory, the same for all threads
  const int us = u_ptr[B], ue = u_ptr[B + 1];
  for (int t = threadIdx.x; t < nB * ct; t += blockDim.x) {
    int ii = t / ct, cc = t % ct;
    if (cc >= cn) continue;
    const T* row = vb + (size_t)ii * w;
    T acc = 0;
    int jj = 0;
    for (int s = us; s < ue; ++s) {
      const int S = __ldg(u_src + s);
      const T* xs = X + (size_t)__ldg(leaf_first + S) * nc + c0 + cc;
      const int n = __ldg(leaf_count + S);
      for (int j = 0; j < n; ++j) acc += row[jj + j] * xs[(size_t)j * nc];
      jj += n;
    }
    Y[(size_t)(f0 + ii) * nc + c0 + cc] = acc;
  }
}

// Near field for few columns (nc <= 8): one warp per target row.  The lanes
// stride along the row's values (coalesced) with the Morton index of each
// near column (near_src), accumulate all nc columns, and reduce by shuffles.
template <class T, int NC>
__global__ void __launch_bounds__(128) k_p2p_rows(int nc, const int32_t* __restrict__ leaf_first,
                                                  const int32_t* __restrict__ leaf_count,
                                                  const int64_t* __restrict__ near_off,
                                                  const int32_t* __restrict__ near_w,
                                                  const int64_t* __restrict__ col_off,
                                                  const int32_t* __restrict__ near_src, const T* __restrict__ val,
                                                  const T* __restrict__ X, T* __restrict__ Y) {
  const int B = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ii = blockIdx.y * 4 + warp;
  if (ii >= leaf_count[B]) return;
  const int w = near_w[B];
  const T* row = val + near_off[B] + (size_t)ii * w;
  const int32_t* src = near_src + col_off[B];
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0;
  for (int jj = lane; jj < w; jj += 32) {
    const T v = row[jj];
    const T* xs = X + (size_t)src[jj] * nc;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc) acc[c] += v * xs[c];
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T a = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    acc[c] = a;
  }
  if (lane == 0) {
    T* y = Y + (size_t)(leaf_first[B] + ii) * nc;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc) y[c] = acc[c];
  }
}

// FP32 near field, shared-memory tiled: one block per (leaf, 64-column tile,
// 64-row block), 128 threads as 16 row groups x 8 column groups; thread
// (ty, tx) owns rows ty + 16 i (i < 4) and columns 4 tx + j, 32 + 4 tx + j
// (j < 4).  The
// leaf's value block (row-major, width w) and the gathered source rows of X
// stream through shared memory in K-chunks of 32 near columns.
__global__ void __launch_bounds__(128) k_p2p_tiled(int nc, const int32_t* __restrict__ leaf_first,
                                                   const int32_t* __restrict__ leaf_count,
                                                   const int64_t* __restrict__ near_off, const int32_t* __restrict__ near_w,
                                                   const int64_t* __restrict__ col_off, const int32_t* __restrict__ near_src,
                                                   const float* __restrict__ val, const float* __restrict__ X,
                                                   float* __restrict__ Y) {
  constexpr int CT = 64, KC = 32, RB = 64;
  __shared__ __align__(16) float Vs[KC][RB + 4];  // transposed value chunk: [near column][row], padded
  __shared__ __align__(16) float Xs[KC][CT];
  const int B = blockIdx.x;
  const int c0 = blockIdx.y * CT;
  const int rb0 = blockIdx.z * RB;
  const int nB = leaf_count[B], f0 = leaf_first[B], w = near_w[B];
  if (rb0 >= nB) return;
  const int nr = min(RB, nB - rb0);
  const float* vb = val + near_off[B] + (size_t)rb0 * w;
  const int32_t* src = near_src + col_off[B];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < w; k0 += KC) {
    const int kn = min(KC, w - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < KC * RB; e += 128) {
      int r = e / KC, kk = e % KC;
      Vs[kk][r] = (r < nr && kk < kn) ? vb[(size_t)r * w + k0 + kk] : 0.f;
    }
    for (int e = threadIdx.x; e < KC * CT; e += 128) {
      int kk = e / CT, cc = e % CT;
      Xs[kk][cc] = (kk < kn && c0 + cc < nc) ? X[(size_t)src[k0 + kk] * nc + c0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      // columns 4 tx .. 4 tx + 3 and 32 + 4 tx .. : a quarter-warp's 16-byte loads are contiguous
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[kk][4 * tx]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[kk][32 + 4 * tx]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float v = Vs[kk][ty + 16 * i];
        acc[i][0] += v * x0.x;
        acc[i][1] += v * x0.y;
        acc[i][2] += v * x0.z;
        acc[i][3] += v * x0.w;
        acc[i][4] += v * x1.x;
        acc[i][5] += v * x1.y;
        acc[i][6] += v * x1.z;
        acc[i][7] += v * x1.w;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = ty + 16 * i;
    if (r >= nr) continue;
    float* yr = Y + (size_t)(f0 + rb0 + r) * nc + c0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) yr[cc] = acc[i][j];
    }
  }
}

// (hi, lo) = (fl32(x), fl32(x - hi)): the double-float split of FP64 values
__global__ void k_split_df(size_t n, const double* __restrict__ a, float2* __restrict__ o) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = a[i];
  const float hi = __double2float_rn(x);
  o[i] = make_float2(hi, __double2float_rn(x - (double)hi));
}

// Near field in FP64 accuracy on the FP32 pipes: the tiling of k_p2p_tiled
// with double-float operands (near values and X pre-split into (hi, lo)),
// exact products by FMA and accumulation as unevaluated float pairs with
// TwoSum (Knuth), ~2^-44 relative rounding per step.
__global__ void __launch_bounds__(128) k_p2p_df64(int nc, const int32_t* __restrict__ leaf_first,
                                                  const int32_t* __restrict__ leaf_count,
                                                  const int64_t* __restrict__ near_off,
                                                  const int32_t* __restrict__ near_w,
                                                  const int64_t* __restrict__ col_off,
                                                  const int32_t* __restrict__ near_src, const float2* __restrict__ val,
                                                  const float2* __restrict__ X, double* __restrict__ Y) {
  constexpr int CT = 64, KC = 16, RB = 64;
  __shared__ __align__(16) float2 Vs[KC][RB + 2];
  __shared__ __align__(16) float2 Xs[KC][CT];
  const int B = blockIdx.x;
  const int c0 = blockIdx.y * CT;
  const int rb0 = blockIdx.z * RB;
  const int nB = leaf_count[B], f0 = leaf_first[B], w = near_w[B];
  if (rb0 >= nB) return;
  const int nr = min(RB, nB - rb0);
  const float2* vb = val + near_off[B] + (size_t)rb0 * w;
  const int32_t* src = near_src + col_off[B];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float sh[4][8], sl[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[i][j] = sl[i][j] = 0.f;
  for (int k0 = 0; k0 < w; k0 += KC) {
    const int kn = min(KC, w - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < KC * RB; e += 128) {
      int r = e / KC, kk = e % KC;
      Vs[kk][r] = (r < nr && kk < kn) ? vb[(size_t)r * w + k0 + kk] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < KC * CT; e += 128) {
      int kk = e / CT, cc = e % CT;
      Xs[kk][cc] = (kk < kn && c0 + cc < nc) ? X[(size_t)src[k0 + kk] * nc + c0 + cc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int kk = 0; kk < KC; ++kk) {
      float2 x[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        x[q] = Xs[kk][4 * tx + q];
        x[4 + q] = Xs[kk][32 + 4 * tx + q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 v = Vs[kk][ty + 16 * i];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float p = v.x * x[q].x;
          const float pe = fmaf(v.x, x[q].x, -p);                 // exact product error
          const float cr = fmaf(v.x, x[q].y, v.y * x[q].x);       // cross terms
          const float t = sh[i][q] + p;                           // TwoSum(sh, p)
          const float bp = t - sh[i][q];
          const float e = (sh[i][q] - (t - bp)) + (p - bp);
          sl[i][q] += e + pe + cr;
          sh[i][q] = t;
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = ty + 16 * i;
    if (r >= nr) continue;
    double* yr = Y + (size_t)(f0 + rb0 + r) * nc + c0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) yr[cc] = (double)sh[i][j] + (double)sl[i][j];
    }
  }
}

// ---- expansions ----------------------------------------------------------------------------
// P2M: M[box][k][c] = sum_i S[i][k] X[i][c]
template <class T>
__global__ void k_p2m(int nc, int ct, int ncoef, int box0, const int32_t* __restrict__ leaf_first,
                      const int32_t* __restrict__ leaf_count, const T* __restrict__ S, const T* __restrict__ X,
                      T* __restrict__ M) {
  const int B = blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const int f0 = leaf_first[B], n = leaf_count[B];
  T* out = M + (size_t)(box0 + B) * ncoef * nc;
  for (int t = threadIdx.x; t < ncoef * ct; t += blockDim.x) {
    int k = t % ncoef, cc = t / ncoef;
    if (cc >= cn) continue;
    T acc = 0;
    for (int i = 0; i < n; ++i) acc += S[(size_t)(f0 + i) * ncoef + k] * X[(size_t)(f0 + i) * nc + c0 + cc];
    out[(size_t)k * nc + c0 + cc] = acc;
  }
}

// M2M: parent boxes [pb0, pb0 + gridDim.x); children contiguous at child_ptr
template <class T>
__global__ void k_m2m(int nc, int ct, int ncoef, int pb0, const int32_t* __restrict__ child_ptr,
                      const int32_t* __restrict__ oct, const T* __restrict__ Tt, T* __restrict__ M) {
  const int P = pb0 + blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const int cs = child_ptr[P], ce = child_ptr[P + 1];
  const size_t ne = (size_t)ncoef * nc;
  for (int t = threadIdx.x; t < ncoef * ct; t += blockDim.x) {
    int k = t % ncoef, cc = t / ncoef;
    if (cc >= cn) continue;
    T acc = 0;
    for (int ch = cs; ch < ce; ++ch) {
      const T* tm = Tt + (size_t)oct[ch] * ncoef * ncoef;
      const T* mc = M + (size_t)ch * ne + c0 + cc;
      for (int j = 0; j < ncoef; ++j) acc += tm[(size_t)j * ncoef + k] * mc[(size_t)j * nc];
    }
    M[(size_t)P * ne + (size_t)k * nc + c0 + cc] = acc;
  }
}

// M2L: target boxes [b0, b0 + gridDim.x); L[box] = sum over V-list
template <class T>
__global__ void k_m2l(int nc, int ct, int ncoef, int b0, const int32_t* __restrict__ v_ptr,
                      const int32_t* __restrict__ v_src, const int16_t* __restrict__ v_off,
                      const T* __restrict__ Tt, const T* __restrict__ M, T* __restrict__ L) {
  const int Bx = b0 + blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const int vs = v_ptr[Bx], ve = v_ptr[Bx + 1];
  const size_t ne = (size_t)ncoef * nc;
  for (int t = threadIdx.x; t < ncoef * ct; t += blockDim.x) {
    int k = t % ncoef, cc = t / ncoef;
    if (cc >= cn) continue;
    T acc = 0;
    for (int v = vs; v < ve; ++v) {
      const T* tm = Tt + (size_t)v_off[v] * ncoef * ncoef;
      const T* ms = M + (size_t)v_src[v] * ne + c0 + cc;
      for (int j = 0; j < ncoef; ++j) acc += tm[(size_t)j * ncoef + k] * ms[(size_t)j * nc];
    }
    L[(size_t)Bx * ne + (size_t)k * nc + c0 + cc] = acc;
  }
}

// M2L for few columns (ct <= 4 per column tile): one block per (target box,
// column tile), 8 warps splitting the V-list; lane l owns output
// coefficients l, l + 32, ... (coalesced table reads), and the warps' partial
// sums are added in shared memory.  ncoef <= 128.
template <class T>
__global__ void __launch_bounds__(256) k_m2l_warps(int nc, int ct, int ncoef, int b0,
                                                   const int32_t* __restrict__ v_ptr,
                                                   const int32_t* __restrict__ v_src,
                                                   const int16_t* __restrict__ v_off, const T* __restrict__ Tt,
                                                   const T* __restrict__ M, T* __restrict__ L) {
  __shared__ T part[8][128][4];
  const int Bx = b0 + blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vs = v_ptr[Bx], ve = v_ptr[Bx + 1];
  const size_t ne = (size_t)ncoef * nc;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0;
  for (int v = vs + warp; v < ve; v += 8) {
    const T* tm = Tt + (size_t)v_off[v] * ncoef * ncoef;
    const T* ms = M + (size_t)v_src[v] * ne + c0;
    for (int j = 0; j < ncoef; ++j) {
      T mj[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) mj[c] = c < cn ? ms[(size_t)j * nc + c] : (T)0;
      const T* tr = tm + (size_t)j * ncoef;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = lane + 32 * i;
        if (k < ncoef) {
          const T t = tr[k];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] += t * mj[c];
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) part[warp][lane + 32 * i][c] = acc[i][c];
  __syncthreads();
  for (int t = threadIdx.x; t < ncoef * cn; t += blockDim.x) {
    const int k = t % ncoef, c = t / ncoef;
    T sum = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += part[w][k][c];
    L[(size_t)Bx * ne + (size_t)k * nc + c0 + c] = sum;
  }
}

// M2L for few columns (nc <= 8) grouped by translation offset: one block per
// (offset, chunk of kOffChunk of its V-list pairs) stages that offset's
// table in shared memory once, and each warp applies it to one pair at a
// time (lane l owns output coefficients l, l + 32, ...), adding into the
// local expansions with atomics (L zeroed before).  At one column a table is
// 8 (p+1)^4 bytes for 2 (p+1)^4 flops per pair; read per pair, as in the
// list form, it made the product L2-bound, staged once per offset it is
// reused by every pair of that offset.
constexpr int kOffChunk = 64;
template <class T, int NC>
__global__ void __launch_bounds__(256) k_m2l_offsets(int nc, int ncoef, const int32_t* __restrict__ op_ptr,
                                                     const int32_t* __restrict__ op_tgt,
                                                     const int32_t* __restrict__ op_src, const T* __restrict__ Tt,
                                                     const T* __restrict__ M, T* __restrict__ L) {
  extern __shared__ __align__(16) unsigned char sm_off[];
  T* Ts = reinterpret_cast<T*>(sm_off);          // [ncoef][ncoef], [in][out]
  const int o = blockIdx.x;
  const int p0 = op_ptr[o] + blockIdx.y * kOffChunk;
  const int p1 = min(op_ptr[o + 1], p0 + kOffChunk);
  if (p0 >= p1) return;
  const T* tm = Tt + (size_t)o * ncoef * ncoef;
  for (int e = threadIdx.x; e < ncoef * ncoef; e += blockDim.x) Ts[e] = tm[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t ne = (size_t)ncoef * nc;
  for (int q = p0 + warp; q < p1; q += 8) {
    const T* ms = M + (size_t)op_src[q] * ne;
    T acc[6][NC];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[i][c] = 0;
    if (NC == 1) {
      // one column: the source expansion in registers (lane l holds
      // coefficients l, l + 32, ...), broadcast by shuffles, so the inner loop
      // reads only shared memory
      T mreg[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) mreg[i] = lane + 32 * i < ncoef ? ms[lane + 32 * i] : (T)0;
#pragma unroll
      for (int jb = 0; jb < 6; ++jb) {
        if (32 * jb >= ncoef) break;
        const int jn = min(32, ncoef - 32 * jb);
        for (int jj = 0; jj < jn; ++jj) {
          const T mj = __shfl_sync(0xffffffffu, mreg[jb], jj);
          const T* tr = Ts + (size_t)(32 * jb + jj) * ncoef;
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            const int k = lane + 32 * i;
            if (k < ncoef) acc[i][0] += tr[k] * mj;
          }
        }
      }
    } else {
#pragma unroll 4
      for (int j = 0; j < ncoef; ++j) {
        T mj[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) mj[c] = c < nc ? ms[(size_t)j * nc + c] : (T)0;
        const T* tr = Ts + (size_t)j * ncoef;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const int k = lane + 32 * i;
          if (k < ncoef) {
            const T t = tr[k];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[i][c] += t * mj[c];
          }
        }
      }
    }
    T* lt = L + (size_t)op_tgt[q] * ne;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int k = lane + 32 * i;
      if (k < ncoef)
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < nc) atomicAdd(lt + (size_t)k * nc + c, acc[i][c]);
    }
  }
}

// M2L, FP32, shared-memory tiled: one block per (target box, 64-column tile),
// 128 threads as 16 row groups x 8 column groups; thread (ty, tx) owns rows
// ty + 16 i (i < RI) and columns 4 tx + j, 32 + 4 tx + j (j < 4).  Per
// V-list pair the translation matrix (stored [in][out]) and the source
// multipole tile are staged in shared memory; the inner loop does 8 RI FMAs
// per RI + 2 shared loads (float4 for the columns).
template <int RI, bool ACC>
__global__ void __launch_bounds__(128) k_m2l_tiled(int nc, int ncoef, int b0, const int32_t* __restrict__ v_ptr,
                                                   const int32_t* __restrict__ v_src, const int16_t* __restrict__ v_off,
                                                   const float* __restrict__ Tt, const float* __restrict__ M,
                                                   float* __restrict__ L) {
  constexpr int CT = 64;
  extern __shared__ float sm32[];
  float* Ts = sm32;                       // [ncoef][16 * RI] (padded rows)
  float* Ms = sm32 + ncoef * 16 * RI;     // [ncoef][CT]
  const int Bx = b0 + blockIdx.x;
  const int c0 = blockIdx.y * CT;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int vs = v_ptr[Bx], ve = v_ptr[Bx + 1];
  const size_t ne = (size_t)ncoef * nc;
  const int ld = 16 * RI;
  float acc[RI][8];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int v = vs; v < ve; ++v) {
    const float* tm = Tt + (size_t)v_off[v] * ncoef * ncoef;
    const float* ms = M + (size_t)v_src[v] * ne + c0;
    __syncthreads();
    for (int e = threadIdx.x; e < ncoef * ld; e += 128) {
      int j = e / ld, k = e % ld;
      Ts[e] = k < ncoef ? tm[(size_t)j * ncoef + k] : 0.f;
    }
    for (int e = threadIdx.x; e < ncoef * CT; e += 128) {
      int j = e / CT, cc = e % CT;
      Ms[e] = (c0 + cc < nc) ? ms[(size_t)j * nc + cc] : 0.f;
    }
    __syncthreads();
    for (int j = 0; j < ncoef; ++j) {
      const float4 m0 = *reinterpret_cast<const float4*>(Ms + j * CT + 4 * tx);
      const float4 m1 = *reinterpret_cast<const float4*>(Ms + j * CT + 32 + 4 * tx);
      const float* tr = Ts + j * ld + ty;
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const float t = tr[16 * i];
        acc[i][0] += t * m0.x;
        acc[i][1] += t * m0.y;
        acc[i][2] += t * m0.z;
        acc[i][3] += t * m0.w;
        acc[i][4] += t * m1.x;
        acc[i][5] += t * m1.y;
        acc[i][6] += t * m1.z;
        acc[i][7] += t * m1.w;
      }
    }
  }
  float* out = L + (size_t)Bx * ne + c0;
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    int k = ty + 16 * i;
    if (k >= ncoef) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) out[(size_t)k * nc + cc] = ACC ? out[(size_t)k * nc + cc] + acc[i][j] : acc[i][j];
    }
  }
}

// M2L with FP64 operands evaluated on the FP32 pipes ("double-float"): each
// double is split into hi = fl32(x), lo = fl32(x - hi) when staged in shared
// memory, products use the FMA error-free transformation, and every output
// accumulates as an unevaluated float pair with TwoSum (Knuth), about 13 FP32
// operations per multiply-add and ~2^-44 relative rounding, against GB300's
// thin FP64 pipe.  One block per (target box, 64-column tile), 256 threads as
// 32 row groups x 8 column groups, rows ty + 32 i (i < 3, ncoef <= 96),
// columns 4 tx + j and 32 + 4 tx + j (j < 4).
template <bool ACC>
__global__ void __launch_bounds__(256) k_m2l_df64(int nc, int ncoef, int b0, const int32_t* __restrict__ v_ptr,
                                                  const int32_t* __restrict__ v_src, const int16_t* __restrict__ v_off,
                                                  const double* __restrict__ Tt, const double* __restrict__ M,
                                                  double* __restrict__ L) {
  constexpr int CT = 64, RI = 3, LD = 96;
  extern __shared__ float2 smd[];
  float2* Ts = smd;                 // [ncoef][LD]  (hi, lo)
  float2* Ms = smd + ncoef * LD;    // [ncoef][CT]
  const int Bx = b0 + blockIdx.x;
  const int c0 = blockIdx.y * CT;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int vs = v_ptr[Bx], ve = v_ptr[Bx + 1];
  const size_t ne = (size_t)ncoef * nc;
  float sh[RI][8], sl[RI][8];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[i][j] = sl[i][j] = 0.f;
  for (int v = vs; v < ve; ++v) {
    const double* tm = Tt + (size_t)v_off[v] * ncoef * ncoef;
    const double* ms = M + (size_t)v_src[v] * ne + c0;
    __syncthreads();
    for (int e = threadIdx.x; e < ncoef * LD; e += 256) {
      int j = e / LD, k = e % LD;
      double x = k < ncoef ? tm[(size_t)j * ncoef + k] : 0.0;
      float hi = __double2float_rn(x);
      Ts[e] = make_float2(hi, __double2float_rn(x - (double)hi));
    }
    for (int e = threadIdx.x; e < ncoef * CT; e += 256) {
      int j = e / CT, cc = e % CT;
      double x = (c0 + cc < nc) ? ms[(size_t)j * nc + cc] : 0.0;
      float hi = __double2float_rn(x);
      Ms[e] = make_float2(hi, __double2float_rn(x - (double)hi));
    }
    __syncthreads();
    for (int j = 0; j < ncoef; ++j) {
      float2 m[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        m[q] = Ms[j * CT + 4 * tx + q];
        m[4 + q] = Ms[j * CT + 32 + 4 * tx + q];
      }
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const float2 t = Ts[j * LD + ty + 32 * i];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float p = t.x * m[q].x;
          const float pe = fmaf(t.x, m[q].x, -p);                 // exact product error
          const float cr = fmaf(t.x, m[q].y, t.y * m[q].x);       // cross terms
          const float s = sh[i][q] + p;                           // TwoSum(sh, p)
          const float bp = s - sh[i][q];
          const float e = (sh[i][q] - (s - bp)) + (p - bp);
          sl[i][q] += e + pe + cr;
          sh[i][q] = s;
        }
      }
    }
  }
  double* out = L + (size_t)Bx * ne + c0;
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    int k = ty + 32 * i;
    if (k >= ncoef) continue;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cc = (q < 4) ? 4 * tx + q : 32 + 4 * tx + (q - 4);
      if (c0 + cc < nc) {
        const double r = (double)sh[i][q] + (double)sl[i][q];
        out[(size_t)k * nc + cc] = ACC ? out[(size_t)k * nc + cc] + r : r;
      }
    }
  }
}

// List-form translation out[b] (=, or += with acc) sum_v T[off[v]] in[src[v]]
// over v in [ptr[b], ptr[b+1]) for boxes b in [b0, b0 + nbx): M2L over the
// V-lists, M2M over the children, L2L from the parent.  Shared-memory tiled
// FP32 (or double-float FP64) kernels; callers check xlate_tiled() first.
template <int RI, bool ACC>
static void run_tiled(dim3 g, int nc, int ncoef, int b0, const int32_t* ptr, const int32_t* src,
                      const int16_t* off, const float* tm, const float* in, float* out, cudaStream_t s) {
  static bool set = false;
  const size_t sm = sizeof(float) * (size_t)ncoef * (16 * RI + 64);
  if (!set) {
    XRL_CUDA(cudaFuncSetAttribute(k_m2l_tiled<RI, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float) * 16 * RI * (16 * RI + 64))));
    set = true;
  }
  k_m2l_tiled<RI, ACC><<<g, 128, sm, s>>>(nc, ncoef, b0, ptr, src, off, tm, in, out);
}

template <bool ACC>
static void run_df64(dim3 g, int nc, int ncoef, int b0, const int32_t* ptr, const int32_t* src,
                     const int16_t* off, const double* tm, const double* in, double* out, cudaStream_t s) {
  static bool set = false;
  const size_t sm = sizeof(float2) * (size_t)ncoef * (96 + 64);
  if (!set) {
    XRL_CUDA(cudaFuncSetAttribute(k_m2l_df64<ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 160 * 8));
    set = true;
  }
  k_m2l_df64<ACC><<<g, 256, sm, s>>>(nc, ncoef, b0, ptr, src, off, tm, in, out);
}

template <class T>
static bool xlate_tiled(const xrl_ctx* c, int nc) {
  if (sizeof(T) == 4) return nc >= 32 && c->ncoef <= 16 * 11;
  return c->df64_m2l && nc >= 32 && c->ncoef <= 96;
}

template <class T>
static void launch_xlate(int nbx, int b0, int nc, int ncoef, const int32_t* ptr, const int32_t* src,
                         const int16_t* off, const T* tm, const T* in, T* out, bool acc, cudaStream_t s);

template <>
void launch_xlate<double>(int nbx, int b0, int nc, int ncoef, const int32_t* ptr, const int32_t* src,
                          const int16_t* off, const double* tm, const double* in, double* out, bool acc,
                          cudaStream_t s) {
  dim3 g(nbx, (nc + 63) / 64);
  if (acc)
    run_df64<true>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
  else
    run_df64<false>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
}

template <>
void launch_xlate<float>(int nbx, int b0, int nc, int ncoef, const int32_t* ptr, const int32_t* src,
                         const int16_t* off, const float* tm, const float* in, float* out, bool acc,
                         cudaStream_t s) {
  dim3 g(nbx, (nc + 63) / 64);
  if (ncoef <= 64) {
    if (acc) run_tiled<4, true>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
    else run_tiled<4, false>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
  } else if (ncoef <= 96) {
    if (acc) run_tiled<6, true>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
    else run_tiled<6, false>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
  } else {
    if (acc) run_tiled<11, true>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
    else run_tiled<11, false>(g, nc, ncoef, b0, ptr, src, off, tm, in, out, s);
  }
}

// P2M, FP32, shared-memory tiled: M[leaf][k][c] = sum_i S[i][k] X[i][c] as
// one small GEMM per leaf.  One CTA per (leaf, 64-column tile), 128 threads
// as 16 coefficient groups (k = ty + 16 i, i < RI) x 8 column groups; the
// leaf's panels stream in chunks of 32 (S rows and X rows in shared memory).
template <int RI>
__global__ void __launch_bounds__(128) k_p2m_tiled(int nc, int ncoef, int box0, const int32_t* __restrict__ leaf_first,
                                                   const int32_t* __restrict__ leaf_count, const float* __restrict__ S,
                                                   const float* __restrict__ X, float* __restrict__ M) {
  constexpr int CT = 64, KC = 32, LD = 16 * RI;
  __shared__ __align__(16) float Ss[KC][LD];
  __shared__ __align__(16) float Xs[KC][CT];
  const int B = blockIdx.x, c0 = blockIdx.y * CT;
  const int f0 = leaf_first[B], n = leaf_count[B];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float acc[RI][8];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int j0 = 0; j0 < n; j0 += KC) {
    const int kn = min(KC, n - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < KC * LD; e += 128) {
      const int j = e / LD, k = e % LD;
      Ss[j][k] = (j < kn && k < ncoef) ? S[(size_t)(f0 + j0 + j) * ncoef + k] : 0.f;
    }
    for (int e = threadIdx.x; e < KC * CT; e += 128) {
      const int j = e / CT, cc = e % CT;
      Xs[j][cc] = (j < kn && c0 + cc < nc) ? X[(size_t)(f0 + j0 + j) * nc + c0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < KC; ++j) {
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[j][4 * tx]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[j][32 + 4 * tx]);
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const float t = Ss[j][ty + 16 * i];
        acc[i][0] += t * x0.x;
        acc[i][1] += t * x0.y;
        acc[i][2] += t * x0.z;
        acc[i][3] += t * x0.w;
        acc[i][4] += t * x1.x;
        acc[i][5] += t * x1.y;
        acc[i][6] += t * x1.z;
        acc[i][7] += t * x1.w;
      }
    }
  }
  float* out = M + (size_t)(box0 + B) * ncoef * nc + c0;
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int k = ty + 16 * i;
    if (k >= ncoef) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) out[(size_t)k * nc + cc] = acc[i][j];
    }
  }
}

// L2P, FP32, shared-memory tiled: Y[i][c] += sum_k W[i][k] L[leaf][k][c] with the
// weighted moments W = (1/h) w_k S[i][k] (k_l2p_weights).
// One CTA per (leaf, 64-column tile, 64-panel block), 128 threads as 16 panel
// groups (i = ty + 16 q, q < 4) x 8 column groups; coefficients in chunks of 32.
__global__ void __launch_bounds__(128) k_l2p_tiled(int nc, int ncoef, int box0,
                                                   const int32_t* __restrict__ leaf_first,
                                                   const int32_t* __restrict__ leaf_count, const float* __restrict__ W,
                                                   const float* __restrict__ L, float* __restrict__ Y) {
  constexpr int CT = 64, KC = 32, RB = 64;
  __shared__ __align__(16) float As[KC][RB];
  __shared__ __align__(16) float Ls[KC][CT];
  const int B = blockIdx.x, c0 = blockIdx.y * CT, rb0 = blockIdx.z * RB;
  const int f0 = leaf_first[B], n = leaf_count[B];
  if (rb0 >= n) return;
  const int nr = min(RB, n - rb0);
  const float* lb = L + (size_t)(box0 + B) * ncoef * nc;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float acc[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[q][j] = 0.f;
  for (int k0 = 0; k0 < ncoef; k0 += KC) {
    const int kn = min(KC, ncoef - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < KC * RB; e += 128) {
      const int i = e / KC, k = e % KC;
      As[k][i] = (i < nr && k < kn) ? W[(size_t)(f0 + rb0 + i) * ncoef + k0 + k] : 0.f;
    }
    for (int e = threadIdx.x; e < KC * CT; e += 128) {
      const int k = e / CT, cc = e % CT;
      Ls[k][cc] = (k < kn && c0 + cc < nc) ? lb[(size_t)(k0 + k) * nc + c0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KC; ++k) {
      const float4 l0 = *reinterpret_cast<const float4*>(&Ls[k][4 * tx]);
      const float4 l1 = *reinterpret_cast<const float4*>(&Ls[k][32 + 4 * tx]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float a = As[k][ty + 16 * q];
        acc[q][0] += a * l0.x;
        acc[q][1] += a * l0.y;
        acc[q][2] += a * l0.z;
        acc[q][3] += a * l0.w;
        acc[q][4] += a * l1.x;
        acc[q][5] += a * l1.y;
        acc[q][6] += a * l1.z;
        acc[q][7] += a * l1.w;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = ty + 16 * q;
    if (i >= nr) continue;
    float* yr = Y + (size_t)(f0 + rb0 + i) * nc + c0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) yr[cc] += acc[q][j];
    }
  }
}

// L2L: child boxes [b0, b0 + gridDim.x) += T(oct) L[parent]
template <class T>
__global__ void k_l2l(int nc, int ct, int ncoef, int b0, const int32_t* __restrict__ parent,
                      const int32_t* __restrict__ oct, const T* __restrict__ Tt, T* __restrict__ L) {
  const int Bx = b0 + blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const size_t ne = (size_t)ncoef * nc;
  const T* tm = Tt + (size_t)oct[Bx] * ncoef * ncoef;
  const T* lp = L + (size_t)parent[Bx] * ne;
  for (int t = threadIdx.x; t < ncoef * ct; t += blockDim.x) {
    int k = t % ncoef, cc = t / ncoef;
    if (cc >= cn) continue;
    T acc = 0;
    for (int j = 0; j < ncoef; ++j) acc += tm[(size_t)j * ncoef + k] * lp[(size_t)j * nc + c0 + cc];
    L[(size_t)Bx * ne + (size_t)k * nc + c0 + cc] += acc;
  }
}

// L2P: Y[i][c] += (1/h) sum_k w_k S[i][k] L[leaf][k][c],  w = 1 (m = 0), 2 (m > 0)
template <class T>
__global__ void k_l2p(int nc, int ct, int ncoef, int box0, T inv_h, const int32_t* __restrict__ leaf_first,
                      const int32_t* __restrict__ leaf_count, const T* __restrict__ S, const T* __restrict__ L,
                      T* __restrict__ Y) {
  const int B = blockIdx.x;
  const int c0 = blockIdx.y * ct;
  const int cn = min(ct, nc - c0);
  const int f0 = leaf_first[B], n = leaf_count[B];
  const T* lb = L + (size_t)(box0 + B) * ncoef * nc;
  for (int t = threadIdx.x; t < n * ct; t += blockDim.x) {
    int ii = t / ct, cc = t % ct;
    if (cc >= cn) continue;
    const T* s = S + (size_t)(f0 + ii) * ncoef;
    T acc = 0;
    int k = 0;
    for (int nn = 0; k < ncoef; ++nn) {
      acc += s[k] * lb[(size_t)k * nc + c0 + cc];
      ++k;
      for (int m = 1; m <= nn; ++m) {
        acc += (T)2 * (s[k] * lb[(size_t)k * nc + c0 + cc] + s[k + 1] * lb[(size_t)(k + 1) * nc + c0 + cc]);
        k += 2;
      }
    }
    Y[(size_t)(f0 + ii) * nc + c0 + cc] += acc * inv_h;
  }
}

// P2M and L2P in FP64 accuracy on the FP32 pipes (the residual operator of the
// mixed mode): the tilings of k_p2m_tiled / k_l2p_tiled with double-float
// operands and the accumulation of k_p2p_df64 (exact products by FMA, sums as
// unevaluated float pairs, ~2^-44 per operation).
__device__ __forceinline__ float2 split_df(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

__device__ __forceinline__ void df_fma(float& sh, float& sl, float2 a, float2 b) {
  const float p = a.x * b.x;
  const float pe = fmaf(a.x, b.x, -p);
  const float cr = fmaf(a.x, b.y, a.y * b.x);
  const float t = sh + p;
  const float bp = t - sh;
  const float e = (sh - (t - bp)) + (p - bp);
  sl += e + pe + cr;
  sh = t;
}

// M[leaf][k][c] = sum_i S[i][k] X[i][c]; S pre-split, X split on load
template <int RI>
__global__ void __launch_bounds__(128) k_p2m_df64(int nc, int ncoef, int box0, const int32_t* __restrict__ leaf_first,
                                                  const int32_t* __restrict__ leaf_count, const float2* __restrict__ S,
                                                  const double* __restrict__ X, double* __restrict__ M) {
  constexpr int CT = 64, KC = 16, LD = 16 * RI;
  __shared__ __align__(16) float2 Ss[KC][LD];
  __shared__ __align__(16) float2 Xs[KC][CT];
  const int B = blockIdx.x, c0 = blockIdx.y * CT;
  const int f0 = leaf_first[B], n = leaf_count[B];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float sh[RI][8], sl[RI][8];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[i][j] = sl[i][j] = 0.f;
  for (int j0 = 0; j0 < n; j0 += KC) {
    const int kn = min(KC, n - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < KC * LD; e += 128) {
      const int j = e / LD, k = e % LD;
      Ss[j][k] = (j < kn && k < ncoef) ? S[(size_t)(f0 + j0 + j) * ncoef + k] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < KC * CT; e += 128) {
      const int j = e / CT, cc = e % CT;
      Xs[j][cc] = (j < kn && c0 + cc < nc) ? split_df(X[(size_t)(f0 + j0 + j) * nc + c0 + cc]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int j = 0; j < KC; ++j) {
      float2 x[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        x[q] = Xs[j][4 * tx + q];
        x[4 + q] = Xs[j][32 + 4 * tx + q];
      }
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const float2 t = Ss[j][ty + 16 * i];
#pragma unroll
        for (int q = 0; q < 8; ++q) df_fma(sh[i][q], sl[i][q], t, x[q]);
      }
    }
  }
  double* out = M + (size_t)(box0 + B) * ncoef * nc + c0;
#pragma unroll
  for (int i = 0; i < RI; ++i) {
    const int k = ty + 16 * i;
    if (k >= ncoef) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) out[(size_t)k * nc + cc] = (double)sh[i][j] + (double)sl[i][j];
    }
  }
}

// Y[i][c] += sum_k W[i][k] L[leaf][k][c]; W (weighted moments) pre-split, L split on load
__global__ void __launch_bounds__(128) k_l2p_df64(int nc, int ncoef, int box0, const int32_t* __restrict__ leaf_first,
                                                  const int32_t* __restrict__ leaf_count, const float2* __restrict__ W,
                                                  const double* __restrict__ L, double* __restrict__ Y) {
  constexpr int CT = 64, KC = 16, RB = 64;
  __shared__ __align__(16) float2 As[KC][RB];
  __shared__ __align__(16) float2 Ls[KC][CT];
  const int B = blockIdx.x, c0 = blockIdx.y * CT, rb0 = blockIdx.z * RB;
  const int f0 = leaf_first[B], n = leaf_count[B];
  if (rb0 >= n) return;
  const int nr = min(RB, n - rb0);
  const double* lb = L + (size_t)(box0 + B) * ncoef * nc;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  float sh[4][8], sl[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 8; ++j) sh[q][j] = sl[q][j] = 0.f;
  for (int k0 = 0; k0 < ncoef; k0 += KC) {
    const int kn = min(KC, ncoef - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < KC * RB; e += 128) {
      const int i = e / KC, k = e % KC;
      As[k][i] = (i < nr && k < kn) ? W[(size_t)(f0 + rb0 + i) * ncoef + k0 + k] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < KC * CT; e += 128) {
      const int k = e / CT, cc = e % CT;
      Ls[k][cc] = (k < kn && c0 + cc < nc) ? split_df(lb[(size_t)(k0 + k) * nc + c0 + cc]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = 0; k < KC; ++k) {
      float2 l[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        l[q] = Ls[k][4 * tx + q];
        l[4 + q] = Ls[k][32 + 4 * tx + q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 w = As[k][ty + 16 * q];
#pragma unroll
        for (int j = 0; j < 8; ++j) df_fma(sh[q][j], sl[q][j], w, l[j]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = ty + 16 * q;
    if (i >= nr) continue;
    double* yr = Y + (size_t)(f0 + rb0 + i) * nc + c0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int cc = (j < 4) ? 4 * tx + j : 32 + 4 * tx + (j - 4);
      if (c0 + cc < nc) yr[cc] += (double)sh[q][j] + (double)sl[q][j];
    }
  }
}

// split of the weighted moments (1 or 2) S / h for k_l2p_df64
__global__ void k_l2p_weights_df(size_t n, int ncoef, double inv_h, const double* __restrict__ S,
                                 float2* __restrict__ w) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % ncoef);
  int r = 0;
  while ((r + 1) * (r + 1) <= k) ++r;
  w[i] = split_df(S[i] * (r * r == k ? inv_h : 2.0 * inv_h));
}

template <class T>
__global__ void k_cast(size_t n, const double* __restrict__ a, T* __restrict__ b) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

// L2P weights folded into an FP32 copy of the moments: w[i][k] = S[i][k] (1 or 2) / h,
// 1 for the m = 0 coefficients (k = n^2), 2 otherwise (the m < 0 half of the expansion)
__global__ void k_l2p_weights(size_t n, int ncoef, double inv_h, const double* __restrict__ S, float* __restrict__ w) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % ncoef);
  int r = 0;
  while ((r + 1) * (r + 1) <= k) ++r;
  w[i] = (float)(S[i] * (r * r == k ? inv_h : 2.0 * inv_h));
}

// ---- host side ---------------------------------------------------------------------------
void fmm_prepare(xrl_ctx* c) {
  const Tree& t = c->tree;
  std::vector<double> m2m, l2l, m2l;
  build_translations(c->p, t.m2l_offsets, m2m, l2l, m2l);
  c->d.t_m2m.upload(c->alloc, m2m);
  c->d.t_l2l.upload(c->alloc, l2l);
  c->d.t_m2l.upload(c->alloc, m2l);
  const int nb = t.n_boxes();
  // children ranges (children of box b are contiguous in the next level)
  std::vector<int32_t> cptr(nb + 1, 0);
  for (int b = 0; b < nb; ++b)
    if (t.parent[b] >= 0) cptr[t.parent[b] + 1]++;
  for (int b = 0; b < nb; ++b) cptr[b + 1] += cptr[b];
  // children of box P start at the first child index: since boxes are sorted by
  // level then key, the first child of P is level_off[l+1] + (count of children of earlier boxes)
  std::vector<int32_t> child_ptr(nb + 1, 0);
  for (int l = 0; l <= t.L; ++l) {
    int base = (l + 1 <= t.L) ? t.level_off[l + 1] : t.level_off[t.L + 1];
    int run = base;
    for (int b = t.level_off[l]; b < t.level_off[l + 1]; ++b) {
      child_ptr[b] = run;
      run += cptr[b + 1] - cptr[b];
    }
  }
  child_ptr[nb] = nb;
  c->d.box_child_ptr.upload(c->alloc, child_ptr);
  c->d.box_parent.upload(c->alloc, t.parent);
  c->d.box_oct.upload(c->alloc, t.octant);
  // list-form arrays: M2M lists are the children (source = box id), L2L
  // lists the single parent (one entry per box)
  std::vector<int32_t> iota(nb + 1);
  std::vector<int16_t> oct16(nb);
  for (int b = 0; b <= nb; ++b) iota[b] = b;
  for (int b = 0; b < nb; ++b) oct16[b] = (int16_t)std::max(0, t.octant[b]);
  c->d.box_iota.upload(c->alloc, iota);
  c->d.box_oct16.upload(c->alloc, oct16);
  std::vector<int32_t> vptr(t.v_ptr.begin(), t.v_ptr.end());
  c->d.v_ptr32.upload(c->alloc, vptr);
  {
    // V-list pairs grouped by offset (for the few-column M2L)
    const int noff = (int)(t.m2l_offsets.size() / 3);
    std::vector<int32_t> optr(noff + 1, 0), otgt(t.v_src.size()), osrc(t.v_src.size());
    for (size_t k = 0; k < t.v_off.size(); ++k) optr[t.v_off[k] + 1]++;
    c->max_off_pairs = 0;
    for (int o = 0; o < noff; ++o) {
      c->max_off_pairs = std::max(c->max_off_pairs, optr[o + 1]);
      optr[o + 1] += optr[o];
    }
    std::vector<int32_t> pos(optr.begin(), optr.end() - 1);
    for (int b = 0; b < nb; ++b)
      for (int64_t k = t.v_ptr[b]; k < t.v_ptr[b + 1]; ++k) {
        const int q = pos[t.v_off[k]]++;
        otgt[q] = b;
        osrc[q] = t.v_src[k];
      }
    c->d.op_ptr.upload(c->alloc, optr);
    c->d.op_tgt.upload(c->alloc, otgt);
    c->d.op_src.upload(c->alloc, osrc);
    // the offset table in shared memory (opt-in above 48 KB), set here, outside any stream capture.
    // The attribute belongs to the kernel, not to this context: it only ever grows, so that a
    // context of lower order cannot shrink it below what another context's launches need.
    static int s8_set = 0;
    const int s8 = (int)(sizeof(double) * c->ncoef * c->ncoef), s4 = s8 / 2;
    if (c->ncoef <= 192 && s8 > s8_set) {
      XRL_CUDA(cudaFuncSetAttribute(k_m2l_offsets<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8));
      XRL_CUDA(cudaFuncSetAttribute(k_m2l_offsets<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8));
      XRL_CUDA(cudaFuncSetAttribute(k_m2l_offsets<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
      XRL_CUDA(cudaFuncSetAttribute(k_m2l_offsets<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
      s8_set = s8;
    }
  }
  c->d.v_src.upload(c->alloc, t.v_src);
  c->d.v_off.upload(c->alloc, t.v_off);
  tc_prepare(c);
  // FP32 copies for the mixed-precision path
  auto cast = [&](const DBuf<double>& a, DBuf<float>& b) {
    b.alloc(c->alloc, a.n);
    if (a.n) k_cast<float><<<(unsigned)((a.n + 255) / 256), 256, 0, c->stream>>>(a.n, a.p, b.p);
  };
  cast(c->d.t_m2m, c->d.t_m2m32);
  cast(c->d.t_l2l, c->d.t_l2l32);
  cast(c->d.t_m2l, c->d.t_m2l32);
  // the FP32 near-field copy is made on first use: products on the tensor
  // cores (>= 64 columns) read the near-block image instead
  c->d.near_val32 = DBuf<float>();
  cast(c->d.mom, c->d.mom32);
  c->d.mom_hl.alloc(c->alloc, c->d.mom.n);
  c->d.momw_hl.alloc(c->alloc, c->d.mom.n);
  if (c->d.mom.n) {
    const unsigned nb = (unsigned)((c->d.mom.n + 255) / 256);
    k_split_df<<<nb, 256, 0, c->stream>>>(c->d.mom.n, c->d.mom.p, c->d.mom_hl.p);
    k_l2p_weights_df<<<nb, 256, 0, c->stream>>>(c->d.mom.n, c->ncoef, (double)(1 << t.L) / t.side, c->d.mom.p,
                                               c->d.momw_hl.p);
  }
  c->d.mom32w.alloc(c->alloc, c->d.mom.n);
  if (c->d.mom.n)
    k_l2p_weights<<<(unsigned)((c->d.mom.n + 255) / 256), 256, 0, c->stream>>>(
        c->d.mom.n, c->ncoef, (double)(1 << t.L) / t.side, c->d.mom.p, c->d.mom32w.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(c->stream));
}

// The FP64-accurate near field of the mixed solver's residuals reads an extra
// image of the near blocks: integer slices (~10 B per padded entry) or the
// double-float split (8 B per entry), made on first use.  Each is made only
// if it fits beside what the context holds (free device memory plus the
// context's cached blocks, less a reserve for the products' work buffers);
// otherwise the residual takes the next path down, and at the end the plain
// FP64 kernel, which reads the FP64 values themselves.
static bool image_fits(xrl_ctx* c, double bytes) {
  size_t fr = 0, tot = 0;
  XRL_CUDA(cudaMemGetInfo(&fr, &tot));
  const double reserve = std::max(8e9, 0.05 * (double)tot);
  return bytes <= (double)fr + (double)c->alloc.cached - reserve;
}

template <class T>
static void fmm_apply_t(xrl_ctx* c, int nc, const T* X, T* Y, const T* near, const T* mom, const T* tm2m,
                        const T* tl2l, const T* tm2l, T* Mx, T* Lx, cudaStream_t s) {
  const Tree& t = c->tree;
  const int ncoef = c->ncoef;
  const int nl = t.n_leaves();
  const int L = t.L;
  const double h = t.side / (double)(1 << L);
  const double sz = sizeof(T);
  const double N = c->N;
  const double nne = (double)c->stats.near_nnz;
  const double e2 = 2.0 * ncoef * ncoef * (double)nc;       // flops of one translation (all columns)
  const double ebytes = (double)ncoef * nc * sz;            // one expansion (all columns)
  // column tiles: p2p uses ct columns per block; expansion kernels ncoef*ct threads
  const int ct_p = nc < 8 ? nc : 8;
  const int ct_e = nc < 4 ? nc : 4;
  dim3 gp(nl, (nc + ct_p - 1) / ct_p);
  cudaEvent_t ev = prof_begin(c, s);
  int nl_p2p = 1;
  // FP32 pass with the tensor-core near field and upward pass: the near field
  // runs on a second stream beside P2M -> M2M -> M2L -> L2L (it only reads
  // the packed X image that P2M also reads) and joins before the L2P adds
  // into Y, so its CTAs fill the SMs that the small far-field kernels leave
  // idle.  With the phase profiler on, the passes run in sequence so that each
  // phase's events time it alone.
  const bool fork =
      sizeof(T) == 4 && tcp_usable(c, nc) && tcm_usable(c, nc) && c->stream2 != nullptr && !c->prof.on;
  cudaStream_t sp = fork ? c->stream2 : s;
  if (sizeof(T) == 4 && tcp_usable(c, nc)) {
    tc_p2p_fork(c, nc, (const float*)X, (float*)Y, s, sp);
    nl_p2p = 2;
  } else if (sizeof(T) == 8 && c->df64_m2l && tcp_usable(c, nc) &&
             (c->d.ozp_vimg.n > 0 || image_fits(c, (double)c->ozp_img_bytes))) {
    tc_p2p64(c, nc, (const double*)X, (double*)Y, s);
    nl_p2p = 2;
  } else if (sizeof(T) == 4 && nc >= 32) {
    dim3 gt(nl, (nc + 63) / 64, (c->max_leaf + 63) / 64);
    k_p2p_tiled<<<gt, 128, 0, s>>>(nc, c->d.leaf_first.p, c->d.leaf_count.p, c->d.near_off.p, c->d.near_w.p,
                                   c->d.near_col_off.p, c->d.near_src.p, (const float*)near, (const float*)X,
                                   (float*)Y);
  } else if (sizeof(T) == 8 && c->df64_m2l && nc >= 32 &&
             (c->d.near_hl.n > 0 || image_fits(c, 8.0 * (double)c->d.near_val.n))) {
    if (c->d.near_hl.n == 0) {
      c->d.near_hl.alloc(c->alloc, c->d.near_val.n);
      k_split_df<<<(unsigned)((c->d.near_val.n + 255) / 256), 256, 0, s>>>(c->d.near_val.n, c->d.near_val.p,
                                                                         c->d.near_hl.p);
      count_launch(c);
    }
    const size_t nx = (size_t)c->N * nc;
    c->d.x_hl.ensure(c->alloc, nx);
    k_split_df<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(nx, (const double*)X, c->d.x_hl.p);
    dim3 gt(nl, (nc + 63) / 64, (c->max_leaf + 63) / 64);
    k_p2p_df64<<<gt, 128, 0, s>>>(nc, c->d.leaf_first.p, c->d.leaf_count.p, c->d.near_off.p, c->d.near_w.p,
                                  c->d.near_col_off.p, c->d.near_src.p, c->d.near_hl.p, c->d.x_hl.p, (double*)Y);
    count_launch(c);
  } else {
    if (nc <= 8) {
      dim3 gr(nl, (c->max_leaf + 3) / 4);
      if (nc == 1)
        k_p2p_rows<T, 1><<<gr, 128, 0, s>>>(nc, c->d.leaf_first.p, c->d.leaf_count.p, c->d.near_off.p, c->d.near_w.p,
                                            c->d.near_col_off.p, c->d.near_src.p, near, X, Y);
      else
        k_p2p_rows<T, 8><<<gr, 128, 0, s>>>(nc, c->d.leaf_first.p, c->d.leaf_count.p, c->d.near_off.p, c->d.near_w.p,
                                            c->d.near_col_off.p, c->d.near_src.p, near, X, Y);
    } else
    k_p2p<T><<<gp, 128, 0, s>>>(nc, ct_p, c->d.leaf_first.p, c->d.leaf_count.p, c->d.u_ptr32.p, c->d.u_src.p,
                                c->d.near_off.p, c->d.near_w.p, near, X, Y);
  }
  prof_end(c, sp, ev, sizeof(T) == 8 ? PH_P2P64 : PH_P2P, nl_p2p, 2.0 * nne * nc, nne * sz + 2.0 * N * nc * sz);
  if (fork) XRL_CUDA(cudaEventRecord(c->ev_join, sp));
  const int ecols = (nc + ct_e - 1) / ct_e;
  const int leaf0 = t.level_off[L];
  // FP32 pass: P2M and M2M on the tensor cores too (P2M reuses the
  // transposed-X image that the near field just packed).  L2L and L2P stay on
  // the CUDA cores: one pair per target, where the tensor-core pipeline's
  // per-CTA setup measured slower than the tiled kernels.
  const bool tcm = sizeof(T) == 4 && tcm_usable(c, nc);
  ev = prof_begin(c, s);
  if (tcm)
    tc_p2m(c, nc, (float*)Mx, s);
  else if (sizeof(T) == 4 && nc >= 32 && ncoef <= 96)
    k_p2m_tiled<6><<<dim3(nl, (nc + 63) / 64), 128, 0, s>>>(nc, ncoef, leaf0, c->d.leaf_first.p, c->d.leaf_count.p,
                                                            (const float*)mom, (const float*)X, (float*)Mx);
  else if (sizeof(T) == 8 && c->df64_m2l && nc >= 32 && ncoef <= 96)
    k_p2m_df64<6><<<dim3(nl, (nc + 63) / 64), 128, 0, s>>>(nc, ncoef, leaf0, c->d.leaf_first.p, c->d.leaf_count.p,
                                                           c->d.mom_hl.p, (const double*)X, (double*)Mx);
  else
    k_p2m<T><<<dim3(nl, ecols), 256, 0, s>>>(nc, ct_e, ncoef, leaf0, c->d.leaf_first.p, c->d.leaf_count.p, mom, X,
                                             Mx);
  prof_end(c, s, ev, PH_P2M, 1, 2.0 * N * ncoef * nc, N * ncoef * sz + N * nc * sz + nl * ebytes);
  ev = prof_begin(c, s);
  const bool tiled = xlate_tiled<T>(c, nc);
  const bool tcm64 = sizeof(T) == 8 && c->df64_m2l && tc64_usable(c, nc);
  for (int l = L - 1; l >= 2; --l) {
    int nbx = t.level_off[l + 1] - t.level_off[l];
    if (tcm)
      tc_m2m(c, l, nc, (float*)Mx, s);
    else if (tcm64)
      tc_m2m64(c, l, nc, (double*)Mx, s);
    else if (tiled)
      launch_xlate<T>(nbx, t.level_off[l], nc, ncoef, c->d.box_child_ptr.p, c->d.box_iota.p, c->d.box_oct16.p, tm2m,
                      Mx, Mx, false, s);
    else
      k_m2m<T><<<dim3(nbx, ecols), 256, 0, s>>>(nc, ct_e, ncoef, t.level_off[l], c->d.box_child_ptr.p,
                                                c->d.box_oct.p, tm2m, Mx);
  }
  {
    double nch = (double)(t.level_off[L + 1] - t.level_off[std::min(3, L + 1)]);
    double npar = (double)(t.level_off[L] - t.level_off[2]);
    prof_end(c, s, ev, PH_M2M, std::max(0, L - 2) * (tcm || tcm64 ? 2 : 1), e2 * nch, (nch + npar) * ebytes);
  }
  {
    int b0 = t.level_off[2];
    int nbx = t.level_off[L + 1] - b0;
    ev = prof_begin(c, s);
    int nl_m2l = 1;
    if (sizeof(T) == 4 && tc_usable(c, nc)) {
      tc_m2l(c, nbx, b0, nc, (const float*)Mx, (float*)Lx, s);
      nl_m2l = 2;
    } else if (sizeof(T) == 8 && c->df64_m2l && tc64_usable(c, nc)) {
      tc_m2l64(c, nbx, b0, nc, (const double*)Mx, (double*)Lx, s);
      nl_m2l = 2;
    } else if (tiled) {
      launch_xlate<T>(nbx, b0, nc, ncoef, c->d.v_ptr32.p, c->d.v_src.p, c->d.v_off.p, tm2l, Mx, Lx, false, s);
    } else {
      if (nc <= 8 && ncoef <= 192 && c->d.op_ptr.n > 0 && (c->max_off_pairs + kOffChunk - 1) / kOffChunk <= 65535) {
        const int noff = (int)(t.m2l_offsets.size() / 3);
        const size_t smem = sizeof(T) * (size_t)ncoef * ncoef;
        XRL_CUDA(cudaMemsetAsync(Lx + (size_t)b0 * ncoef * nc, 0, sizeof(T) * (size_t)nbx * ncoef * nc, s));
        const dim3 g(noff, (c->max_off_pairs + kOffChunk - 1) / kOffChunk);
        if (nc == 1) {
          k_m2l_offsets<T, 1><<<g, 256, smem, s>>>(nc, ncoef, c->d.op_ptr.p, c->d.op_tgt.p, c->d.op_src.p, tm2l, Mx,
                                                   Lx);
        } else {
          k_m2l_offsets<T, 8><<<g, 256, smem, s>>>(nc, ncoef, c->d.op_ptr.p, c->d.op_tgt.p, c->d.op_src.p, tm2l, Mx,
                                                   Lx);
        }
        count_launch(c);
      } else if (ncoef <= 128 && nc <= 16)
        k_m2l_warps<T><<<dim3(nbx, ecols), 256, 0, s>>>(nc, ct_e, ncoef, b0, c->d.v_ptr32.p, c->d.v_src.p,
                                                        c->d.v_off.p, tm2l, Mx, Lx);
      else
      k_m2l<T><<<dim3(nbx, ecols), 256, 0, s>>>(nc, ct_e, ncoef, b0, c->d.v_ptr32.p, c->d.v_src.p, c->d.v_off.p,
                                                tm2l, Mx, Lx);
    }
    prof_end(c, s, ev, sizeof(T) == 8 ? PH_M2L64 : PH_M2L, nl_m2l, e2 * (double)t.v_src.size(),
             2.0 * nbx * ebytes);
  }
  ev = prof_begin(c, s);
  for (int l = 3; l <= L; ++l) {
    int nbx = t.level_off[l + 1] - t.level_off[l];
    if (tiled)
      launch_xlate<T>(nbx, t.level_off[l], nc, ncoef, c->d.box_iota.p, c->d.box_parent.p, c->d.box_oct16.p, tl2l,
                      Lx, Lx, true, s);
    else
      k_l2l<T><<<dim3(nbx, ecols), 256, 0, s>>>(nc, ct_e, ncoef, t.level_off[l], c->d.box_parent.p,
                                                c->d.box_oct.p, tl2l, Lx);
  }
  {
    double nch = (double)(t.level_off[L + 1] - t.level_off[std::min(3, L + 1)]);
    prof_end(c, s, ev, PH_L2L, std::max(0, L - 2), e2 * nch, 2.0 * nch * ebytes);
  }
  if (fork) XRL_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
  ev = prof_begin(c, s);
  if (sizeof(T) == 4 && nc >= 32)
    k_l2p_tiled<<<dim3(nl, (nc + 63) / 64, (c->max_leaf + 63) / 64), 128, 0, s>>>(
        nc, ncoef, leaf0, c->d.leaf_first.p, c->d.leaf_count.p, c->d.mom32w.p, (const float*)Lx, (float*)Y);
  else if (sizeof(T) == 8 && c->df64_m2l && nc >= 32)
    k_l2p_df64<<<dim3(nl, (nc + 63) / 64, (c->max_leaf + 63) / 64), 128, 0, s>>>(
        nc, ncoef, leaf0, c->d.leaf_first.p, c->d.leaf_count.p, c->d.momw_hl.p, (const double*)Lx, (double*)Y);
  else
    k_l2p<T><<<dim3(nl, ecols), 128, 0, s>>>(nc, ct_e, ncoef, leaf0, (T)(1.0 / h), c->d.leaf_first.p,
                                             c->d.leaf_count.p, mom, Lx, Y);
  prof_end(c, s, ev, PH_L2P, 1, 2.0 * N * ncoef * nc, N * ncoef * sz + 2.0 * N * nc * sz + nl * ebytes);
  XRL_CUDA(cudaGetLastError());
}

void fmm_apply(xrl_ctx* c, int nc, const double* X, double* Y, cudaStream_t s) {
  size_t ne = (size_t)c->tree.n_boxes() * c->ncoef * nc;
  c->d.Mexp.ensure(c->alloc, ne);
  c->d.Lexp.ensure(c->alloc, ne);
  fmm_apply_t<double>(c, nc, X, Y, c->d.near_val.p, c->d.mom.p, c->d.t_m2m.p, c->d.t_l2l.p, c->d.t_m2l.p,
                      c->d.Mexp.p, c->d.Lexp.p, s);
}

// FP64 product with caller-provided expansion buffers (each at least
// n_boxes * (p+1)^2 * nc doubles).  Allocates nothing while c->df64_m2l is
// false (the FP64-accurate residual mode of a mixed solve creates its
// double-float and integer-slice images on first use) and the profiler is off.
void fmm_apply_into(xrl_ctx* c, int nc, const double* X, double* Y, double* Mx, double* Lx, cudaStream_t s) {
  fmm_apply_t<double>(c, nc, X, Y, c->d.near_val.p, c->d.mom.p, c->d.t_m2m.p, c->d.t_l2l.p, c->d.t_m2l.p, Mx, Lx,
                      s);
}

void fmm_apply32(xrl_ctx* c, int nc, const float* X, float* Y, cudaStream_t s) {
  if (!tcp_usable(c, nc) && c->d.near_val32.n == 0 && c->d.near_val.n > 0) {
    c->d.near_val32.alloc(c->alloc, c->d.near_val.n);
    k_cast<float><<<(unsigned)((c->d.near_val.n + 255) / 256), 256, 0, s>>>(c->d.near_val.n, c->d.near_val.p,
                                                                          c->d.near_val32.p);
    count_launch(c);
  }
  size_t ne = (size_t)c->tree.n_boxes() * c->ncoef * nc;
  c->d.M32.ensure(c->alloc, ne);
  c->d.L32.ensure(c->alloc, ne);
  fmm_apply_t<float>(c, nc, X, Y, c->d.near_val32.p, c->d.mom32.p, c->d.t_m2m32.p, c->d.t_l2l32.p,
                     c->d.t_m2l32.p, c->d.M32.p, c->d.L32.p, s);
}

}  // namespace xrl
