// Tensor-core (tcgen05) list-form translation for the FP32 FMM pass
// (Sec. II-C): out[b] (=, or +=) sum_v T[off[v]] in[src[v]] over the V-list of
// target box b, for 128-column tiles of the right-hand sides.
//
// Per (target box, 128-column tile) one CTA accumulates D[c][n] (c = column,
// n = output coefficient) in tensor memory: D = sum_v A_v B_v with
// A_v[c][k] = in[src[v]][k][c] (128 x Kp) and B_v[k][n] = T[off[v]][k][n]
// (Kp x Np), Kp, Np the coefficient count (p+1)^2 padded to 16.  FP32
// accuracy comes from a three-piece BF16 split x = x0 + x1 + x2 (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); residual ~2^-27 |x|) and the six
// products x_i y_j with i + j <= 2 (the dropped ones are ~2^-27 relative), all
// exact in FP32 and accumulated in FP32 by the tensor core.  The two-target
// M2L (64-coefficient tiles) instead splits power-of-two-scaled operands into
// two FP16 pieces (22 bits) and runs three products: ~2^-21 per term, below
// the expansion's own truncation, in half the MMAs (see k_tch_pack_a).  (A
// two-piece TF32 split reaches the same ~2^-21 at half the FP16 rate.)
//
// Operands live in global memory as "packed images" in the tensor core's
// K-major, no-swizzle shared-memory layout, so that one pipeline stage is two
// plain bulk copies (cp.async.bulk) and no thread touches the operand bytes:
//   per operand of R rows: K chunks of 32 (the last one kc = Kp - 32 c),
//   each chunk [x0 | x1 | x2], each piece [R/8 row groups][kc/8 core columns]
//   of 8 x 16-byte core matrices (row r at +16 (r % 8), column k at +2 (k % 8)).
// The translation tables are packed once per context (from FP64, so the
// split is that of the exact table); the expansions once per product.
//
// Warp roles: warp 0 lane 0 issues the bulk copies, warp 1 lane 0 issues the
// MMAs (one thread, as tcgen05.mma requires), the other warps drain the
// accumulators (warp w reads TMEM lanes 32 (w % 4) .. + 31): warps 2..5 in
// k_xlate_tc, warps 2..9 in k_xlate_tc2 and k_xlate_oz (one half of the
// accumulator columns each).  Every wait is
// bounded; on a timeout the kernel raises *err, drains its own copies and
// frees its tensor memory.
//
// Kernels: k_xlate_tc (one target per CTA: M2L at order 8, P2M, the M2M
// levels), k_xlate_tc2 (two sibling targets per CTA over their merged list:
// the M2L at <= 64 coefficients and the near field), k_xlate_oz (the
// FP64-accurate M2L, M2M and near field in integer slices).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "xrl_internal.hpp"

namespace xrl {

namespace {

constexpr int TC_ROWS = 128;     // columns per tile (MMA M)
constexpr int TC_KC = 32;        // K chunk per pipeline stage (elements)
constexpr int TC_STAGES = 4;
constexpr int TC_PIECES = 3;
constexpr int TCH_PIECES = 2;     // FP16 pieces of the two-target M2L operands
constexpr int TCH_TOP = 14;       // scaled operands stay below 2^14 (FP16 max 65504)
constexpr long long TC_WAIT_CYCLES = 4000000000ll;   // ~2 s at the maximum SM clock

// bytes of one K chunk (all pieces) of an operand of R rows
__host__ __device__ inline int tc_chunk_bytes(int R, int kc) { return TC_PIECES * R * kc * 2; }

// byte offset of element (r, k), piece h, in the packed image of R rows x Kp
__host__ __device__ inline size_t tc_img_off(int R, int Kp, int r, int k, int h) {
  const int c = k >> 5;
  const int kc = (Kp - 32 * c) < 32 ? (Kp - 32 * c) : 32;
  const int kq = (k & 31) >> 3;
  return (size_t)tc_chunk_bytes(R, 32) * c + (size_t)h * R * kc * 2 + ((size_t)(r >> 3) * (kc >> 3) + kq) * 128 +
         (r & 7) * 16 + (k & 7) * 2;
}

// the same layout with `pc` pieces per chunk
__host__ __device__ inline int oz_chunk_bytes(int R, int kc, int pc) { return pc * R * kc * 2; }
__host__ __device__ inline size_t oz_img_off(int R, int Kp, int r, int k, int h, int pc) {
  const int c = k >> 5;
  const int kc = (Kp - 32 * c) < 32 ? (Kp - 32 * c) : 32;
  const int kq = (k & 31) >> 3;
  return (size_t)oz_chunk_bytes(R, 32, pc) * c + (size_t)h * R * kc * 2 + ((size_t)(r >> 3) * (kc >> 3) + kq) * 128 +
         (r & 7) * 16 + (k & 7) * 2;
}

constexpr unsigned kMaxGridY = 65535u;   // grid.y limit: larger target counts launch in slices
constexpr int OZ_S = 5;          // integer slices of 7 bits
constexpr int OZ_STAGES = 3;

__device__ __forceinline__ uint32_t sm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
__device__ __forceinline__ uint16_t f16_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
__device__ __forceinline__ float f16_val(uint16_t b) { return __half2float(__ushort_as_half(b)); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(sm_u32(b)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the phase of parity `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity))
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sm_u32(dst)),
               "l"(src), "r"(bytes), "r"(sm_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte step
// between the two core matrices along K, sbo = byte step between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_u32(bar))
               : "memory");
}

}  // namespace

// Pack FP32 expansions in[box][k][col] (boxes [b0, b0 + gridDim.x), column
// tile blockIdx.y) into the A image; columns >= nc and k >= ncoef are zero.
// One thread per (row, 8-element core row): three 16-byte stores.
__global__ void k_tc_pack_a(int nc, int ncoef, int Kp, int b0, const float* __restrict__ in,
                            uint16_t* __restrict__ img) {
  const int ct = blockIdx.y;
  const float* src = in + (size_t)(b0 + blockIdx.x) * ncoef * nc + (size_t)ct * TC_ROWS;
  char* dst = reinterpret_cast<char*>(img) + ((size_t)blockIdx.x * gridDim.y + ct) * (size_t)(TC_PIECES * 2 * TC_ROWS * Kp);
  const int nq = Kp >> 3;
  for (int e = threadIdx.x; e < TC_ROWS * nq; e += blockDim.x) {
    const int r = e & (TC_ROWS - 1), kq = e >> 7;
    const bool col_ok = ct * TC_ROWS + r < nc;
    uint16_t p0[8], p1[8], p2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * kq + q;
      const float x = (col_ok && k < ncoef) ? src[(size_t)k * nc + r] : 0.f;
      p0[q] = bf16_bits(x);
      const float r1 = x - bf16_val(p0[q]);
      p1[q] = bf16_bits(r1);
      p2[q] = bf16_bits(r1 - bf16_val(p1[q]));
    }
    uint4 v0, v1, v2;
    v0.x = p0[0] | (uint32_t)p0[1] << 16; v0.y = p0[2] | (uint32_t)p0[3] << 16;
    v0.z = p0[4] | (uint32_t)p0[5] << 16; v0.w = p0[6] | (uint32_t)p0[7] << 16;
    v1.x = p1[0] | (uint32_t)p1[1] << 16; v1.y = p1[2] | (uint32_t)p1[3] << 16;
    v1.z = p1[4] | (uint32_t)p1[5] << 16; v1.w = p1[6] | (uint32_t)p1[7] << 16;
    v2.x = p2[0] | (uint32_t)p2[1] << 16; v2.y = p2[2] | (uint32_t)p2[3] << 16;
    v2.z = p2[4] | (uint32_t)p2[5] << 16; v2.w = p2[6] | (uint32_t)p2[7] << 16;
    *reinterpret_cast<uint4*>(dst + tc_img_off(TC_ROWS, Kp, r, 8 * kq, 0)) = v0;
    *reinterpret_cast<uint4*>(dst + tc_img_off(TC_ROWS, Kp, r, 8 * kq, 1)) = v1;
    *reinterpret_cast<uint4*>(dst + tc_img_off(TC_ROWS, Kp, r, 8 * kq, 2)) = v2;
  }
}

// Pack translation tables T[o][k_in][n_out] (FP64, [in][out]) into B images
// of Np rows (n) by Kp (k), one per table (blockIdx.x); split from FP64.
__global__ void k_tc_pack_b(int ncoef, int Kp, int Np, const double* __restrict__ T, uint16_t* __restrict__ img) {
  const int o = blockIdx.x;
  const double* tm = T + (size_t)o * ncoef * ncoef;
  char* dst = reinterpret_cast<char*>(img) + (size_t)o * (size_t)(TC_PIECES * 2 * Np * Kp);
  for (int e = threadIdx.x; e < Np * Kp; e += blockDim.x) {
    const int r = e % Np, k = e / Np;
    const double x = (r < ncoef && k < ncoef) ? tm[(size_t)k * ncoef + r] : 0.0;
    const uint16_t b0 = bf16_bits(__double2float_rn(x));
    const double r1 = x - (double)bf16_val(b0);
    const uint16_t b1 = bf16_bits(__double2float_rn(r1));
    const double r2 = r1 - (double)bf16_val(b1);
    const uint16_t b2 = bf16_bits(__double2float_rn(r2));
    *reinterpret_cast<uint16_t*>(dst + tc_img_off(Np, Kp, r, k, 0)) = b0;
    *reinterpret_cast<uint16_t*>(dst + tc_img_off(Np, Kp, r, k, 1)) = b1;
    *reinterpret_cast<uint16_t*>(dst + tc_img_off(Np, Kp, r, k, 2)) = b2;
  }
}

// ---- two-piece FP16 operands of the two-target M2L ------------------------------------
// x = x0 + x1 with x0 = fp16(x), x1 = fp16(x - x0) keeps 22 significant bits;
// the three products x0 y0, x0 y1, x1 y0 leave ~2^-21 relative per term, below
// the order-7 truncation of the expansion (~1e-6), in half the MMAs of the
// three-piece BF16 split.  FP16 has a 5-bit exponent, so both operands are
// scaled by powers of two (exact): the coefficient equilibration 2^-d_k (A)
// and 2^d_k (B) of the FP64-accurate path, then per A row (one right-hand
// side column of one source box) 2^(TCH_TOP - e_A) and per B column (one
// output coefficient n, over all tables) 2^(TCH_TOP - e_n), with 2^e the
// power of two above the row's / column's largest entry.  The epilogue
// multiplies each pair's partial sums by its row scale 2^(e_A - TCH_TOP) and
// the finished sum by 2^(e_n - TCH_TOP).  Entries far below their row or
// column maximum keep fewer bits (FP16 subnormals), an absolute error below
// 2^-38 of that maximum.

// Pack FP32 multipoles in[box][k][col] (boxes [b0, b0 + gridDim.x), column
// tile blockIdx.y) into the two-piece FP16 A image; ascale[tile][r] receives
// the row's 2^(e_A - TCH_TOP).  Columns >= nc and k >= ncoef are zero.
__global__ void k_tch_pack_a(int nc, int ncoef, int Kp, int b0, const int32_t* __restrict__ dk,
                             const float* __restrict__ in, uint16_t* __restrict__ img, float* __restrict__ ascale) {
  __shared__ int eA[TC_ROWS];
  const int ct = blockIdx.y;
  const size_t tile = (size_t)blockIdx.x * gridDim.y + ct;
  const float* src = in + (size_t)(b0 + blockIdx.x) * ncoef * nc + (size_t)ct * TC_ROWS;
  char* dst = reinterpret_cast<char*>(img) + tile * (size_t)(TCH_PIECES * 2 * TC_ROWS * Kp);
  for (int r = threadIdx.x; r < TC_ROWS; r += blockDim.x) {
    float mx = 0.f;
    if (ct * TC_ROWS + r < nc)
      for (int k = 0; k < ncoef; ++k) mx = fmaxf(mx, fabsf(ldexpf(src[(size_t)k * nc + r], -dk[k])));
    const int e = mx > 0.f ? ilogbf(mx) + 1 : 0;
    eA[r] = e;
    ascale[tile * TC_ROWS + r] = ldexpf(1.f, e - TCH_TOP);
  }
  __syncthreads();
  const int nq = Kp >> 3;
  for (int e = threadIdx.x; e < TC_ROWS * nq; e += blockDim.x) {
    const int r = e & (TC_ROWS - 1), kq = e >> 7;
    const bool col_ok = ct * TC_ROWS + r < nc;
    const int sh = TCH_TOP - eA[r];
    uint16_t p0[8], p1[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * kq + q;
      const float x = (col_ok && k < ncoef) ? ldexpf(src[(size_t)k * nc + r], sh - dk[k]) : 0.f;
      p0[q] = f16_bits(x);
      p1[q] = f16_bits(x - f16_val(p0[q]));
    }
    uint4 v0, v1;
    v0.x = p0[0] | (uint32_t)p0[1] << 16; v0.y = p0[2] | (uint32_t)p0[3] << 16;
    v0.z = p0[4] | (uint32_t)p0[5] << 16; v0.w = p0[6] | (uint32_t)p0[7] << 16;
    v1.x = p1[0] | (uint32_t)p1[1] << 16; v1.y = p1[2] | (uint32_t)p1[3] << 16;
    v1.z = p1[4] | (uint32_t)p1[5] << 16; v1.w = p1[6] | (uint32_t)p1[7] << 16;
    *reinterpret_cast<uint4*>(dst + oz_img_off(TC_ROWS, Kp, r, 8 * kq, 0, TCH_PIECES)) = v0;
    *reinterpret_cast<uint4*>(dst + oz_img_off(TC_ROWS, Kp, r, 8 * kq, 1, TCH_PIECES)) = v1;
  }
}

// Pack the FP64 M2L tables T[o][k_in][n_out] into two-piece FP16 B images (Np
// rows n by Kp), T'[k][n] = T[k][n] 2^(d_k + TCH_TOP - en[n]).
__global__ void k_tch_pack_b(int ncoef, int Kp, int Np, const int32_t* __restrict__ dk, const int32_t* __restrict__ en,
                             const double* __restrict__ T, uint16_t* __restrict__ img) {
  const int o = blockIdx.x;
  const double* tm = T + (size_t)o * ncoef * ncoef;
  char* dst = reinterpret_cast<char*>(img) + (size_t)o * (size_t)(TCH_PIECES * 2 * Np * Kp);
  for (int e = threadIdx.x; e < Np * Kp; e += blockDim.x) {
    const int r = e % Np, k = e / Np;
    const double x = (r < ncoef && k < ncoef) ? ldexp(tm[(size_t)k * ncoef + r], dk[k] + TCH_TOP - en[r]) : 0.0;
    const uint16_t b0 = f16_bits(__double2float_rn(x));
    const uint16_t b1 = f16_bits(__double2float_rn(x - (double)f16_val(b0)));
    *reinterpret_cast<uint16_t*>(dst + oz_img_off(Np, Kp, r, k, 0, TCH_PIECES)) = b0;
    *reinterpret_cast<uint16_t*>(dst + oz_img_off(Np, Kp, r, k, 1, TCH_PIECES)) = b1;
  }
}

// Largest |S[i][k]| per coefficient k of the panel moments (positive doubles
// order as their bit patterns); out[] zeroed by the caller.
__global__ void k_colmax_abs(size_t n, int ncoef, const double* __restrict__ S, unsigned long long* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    atomicMax(out + (i % ncoef), (unsigned long long)__double_as_longlong(fabs(S[i])));
}

// Largest |T[o][k][n] 2^d_k| per output coefficient n over all tables.
__global__ void k_tch_colmax(size_t n, int ncoef, const int32_t* __restrict__ dk, const double* __restrict__ T,
                             unsigned long long* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)((i / ncoef) % ncoef);
    atomicMax(out + (i % ncoef), (unsigned long long)__double_as_longlong(fabs(ldexp(T[i], dk[k]))));
  }
}

// Pair sources of one tensor-core launch (D[col][n] = sum over pairs A B).
// Grids are (column tile, target): the tiles of one target are issued side by
// side, so the operand both share (the table or the near block) is fetched
// from DRAM once and served from L2 to the others.
//  * mode 0 (M2L, M2M, L2L): targets are boxes b0 + blockIdx.y with pairs
//    [ptr[b], ptr[b+1]); A = the expansion image of box src[v] (tile ct),
//    B = table off[v], K = Kp, N = NP; out[box][k][col], ncoef rows.
//  * mode 1 (P2P): targets are leaves blockIdx.y with their U-list pairs; A =
//    the transposed-X image of leaf src[v] (K = its panels padded to 16),
//    B = the pair's near block (N = the target's panels padded to 16);
//    out = Y[panel][col], one row per target panel.
//  * mode 2 (P2M): target leaf L = blockIdx.y, one pair: A = leaf L's
//    transposed-X image, B = its moment image (pair_boff[L]), N = NP;
//    out[box b0 + L][k][col].
struct XlPairs {
  int mode, b0, src0, nct, Kp, sum_pc, ncoef;
  int y0;                // first target of this launch (grid.y is capped at 65535)
  size_t a_img, b_img;   // mode 0: bytes of one (box, tile) A image and of one table image
  int a_row_bytes;       // bytes per K element of an A image (pieces x 128 x 2)
  const int32_t* ptr;
  const int32_t* src;
  const int16_t* off;
  const int32_t* leaf_a0;   // padded panel offset of each leaf
  const int32_t* leaf_pc;   // padded panel count
  const int32_t* leaf_f0;   // first panel
  const int32_t* leaf_n;    // panel count
  const int64_t* pair_boff; // byte offset of each pair's (mode 1) or leaf's (mode 2) B image
};

__device__ __forceinline__ void xl_pair(const XlPairs& p, int v, int ct, size_t& aoff, size_t& boff, int& K) {
  if (p.mode == 0) {
    aoff = ((size_t)(p.src[v] - p.src0) * p.nct + ct) * p.a_img;
    boff = (size_t)p.off[v] * p.b_img;
    K = p.Kp;
  } else {
    const int S = p.mode == 1 ? p.src[v] : v;
    aoff = ((size_t)ct * p.sum_pc + p.leaf_a0[S]) * (size_t)p.a_row_bytes;
    boff = (size_t)p.pair_boff[v];
    K = p.leaf_pc[S];
  }
}

// target of this CTA: pair range, N, output rows and base row index
__device__ __forceinline__ void xl_target(const XlPairs& p, int NPmax, int& vs, int& ve, int& N, int& nrows,
                                          size_t& row0) {
  if (p.mode == 0) {
    const int Bx = p.b0 + p.y0 + (int)blockIdx.y;
    vs = p.ptr[Bx];
    ve = p.ptr[Bx + 1];
    N = NPmax;
    nrows = p.ncoef;
    row0 = (size_t)Bx * p.ncoef;
  } else if (p.mode == 1) {
    const int T = p.y0 + (int)blockIdx.y;
    vs = p.ptr[T];
    ve = p.ptr[T + 1];
    nrows = p.leaf_n[T];
    N = (nrows + 15) & ~15;
    row0 = (size_t)p.leaf_f0[T];
  } else {
    const int L = p.y0 + (int)blockIdx.y;
    vs = L;
    ve = L + 1;
    N = NPmax;
    nrows = p.ncoef;
    row0 = (size_t)(p.b0 + L) * p.ncoef;
  }
}

struct TcArgs {
  XlPairs pr;
  int nc;
  const char* aimg;
  const char* bimg;
  float* out;
  int32_t* err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(b)) : "memory");
}

// acc[n] += both accumulators of one pair buffer (small first), columns n < NL
template <int NP, int NL>
__device__ __forceinline__ void drain_pair(float (&acc)[NP], uint32_t taddr) {
#pragma unroll
  for (int s = 1; s >= 0; --s) {
    uint32_t r[NL];
#pragma unroll
    for (int n0 = 0; n0 < NL; n0 += 16)
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
          "[%16];"
          : "=r"(r[n0 + 0]), "=r"(r[n0 + 1]), "=r"(r[n0 + 2]), "=r"(r[n0 + 3]), "=r"(r[n0 + 4]), "=r"(r[n0 + 5]),
            "=r"(r[n0 + 6]), "=r"(r[n0 + 7]), "=r"(r[n0 + 8]), "=r"(r[n0 + 9]), "=r"(r[n0 + 10]), "=r"(r[n0 + 11]),
            "=r"(r[n0 + 12]), "=r"(r[n0 + 13]), "=r"(r[n0 + 14]), "=r"(r[n0 + 15])
          : "r"(taddr + 128u * s + (uint32_t)n0)
          : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int n = 0; n < NL; ++n) acc[n] += __uint_as_float(r[n]);
  }
}

// Warps: 0 = bulk-copy producer (lane 0; the whole warp owns the TMEM
// allocation), 1 = MMA issuer (lane 0), 2..5 = accumulator drain/epilogue.
// TMEM (512 columns): for the pair buffer q in {0, 1} the x0 y0 products go to
// columns 256 q and the five small products to 256 q + 128.  After every
// pair the epilogue warps add both into FP32 registers (IEEE
// round-to-nearest), so the tensor core only ever accumulates the MMAs of one
// pair: its truncating block accumulation would otherwise bias sums over
// thousands of MMAs.
template <int NP>
__global__ void __launch_bounds__(192, 1) k_xlate_tc(TcArgs a) {
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_stage = tc_chunk_bytes(TC_ROWS, TC_KC);
  const int stage_bytes = a_stage + tc_chunk_bytes(NP, TC_KC);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + TC_STAGES * stage_bytes);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* tfull = empty + TC_STAGES;   // [2]: pair buffer written
  uint64_t* tfree = tfull + 2;           // [2]: pair buffer drained
  uint64_t* mdone = tfree + 2;           // all MMAs of this CTA complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 1);
  int* bad = reinterpret_cast<int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x;
  int vs, ve, N, nrows;
  size_t row0;
  xl_target(a.pr, NP, vs, ve, N, nrows, row0);
  const int nv = ve - vs;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&tfull[q], 1);
      mbar_init(&tfree[q], 4);
    }
    mbar_init(mdone, 1);
    *bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tslot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool stop = false;
      for (int v = vs; v < ve && !stop; ++v) {
        size_t aoff, boff;
        int K;
        xl_pair(a.pr, v, ct, aoff, boff, K);
        const int nchv = (K + TC_KC - 1) / TC_KC;
        for (int c = 0; c < nchv; ++c, ++it) {
          const int st = it % TC_STAGES, u = it / TC_STAGES;
          if (u > 0 && !mbar_wait(&empty[st], (u - 1) & 1)) {
            atomicExch(bad, 1);
            stop = true;
            break;
          }
          const int kc = min(TC_KC, K - TC_KC * c);
          const char* asrc = a.aimg + aoff + (size_t)a_stage * c;
          const char* bsrc = a.bimg + boff + (size_t)tc_chunk_bytes(N, TC_KC) * c;
          const uint32_t ab = tc_chunk_bytes(TC_ROWS, kc), bb = tc_chunk_bytes(N, kc);
          uint8_t* sa = base + (size_t)st * stage_bytes;
          mbar_expect_tx(&full[st], ab + bb);
          bulk_g2s(sa, asrc, ab, &full[st]);
          bulk_g2s(sa + a_stage, bsrc, bb, &full[st]);
          issued = it + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // D f32, A and B bf16, K-major both, N, M = 128
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
      int it = 0;
      bool stop = false;
      for (int v = vs, j = 0; v < ve && !stop; ++v, ++j) {
        size_t aoff, boff;
        int K;
        xl_pair(a.pr, v, ct, aoff, boff, K);
        const int nchv = (K + TC_KC - 1) / TC_KC;
        const int q = j & 1;
        if (j >= 2 && !mbar_wait(&tfree[q], ((j >> 1) - 1) & 1)) {
          atomicExch(bad, 1);
          break;
        }
        for (int c = 0; c < nchv; ++c, ++it) {
          const int st = it % TC_STAGES, u = it / TC_STAGES;
          if (!mbar_wait(&full[st], u & 1)) {
            atomicExch(bad, 1);
            stop = true;
            break;
          }
          tc_fence_after();
          const int kc = min(TC_KC, K - TC_KC * c);
          const uint32_t sa = sm_u32(base + (size_t)st * stage_bytes);
          const uint32_t sb = sa + a_stage;
          const uint32_t pa = TC_ROWS * kc * 2, pb = N * kc * 2;   // piece strides
          const uint32_t sbo = 16 * kc;                            // (kc / 8) cores of 128 B
          const uint32_t dbig = tbase + 256u * q, dsmall = dbig + 128u;
          // descriptors differ only in the start-address field (address >> 4,
          // no carry below 256 KB): build two, offset the rest
          const uint64_t dA = sdesc(sa, 128, sbo), dB = sdesc(sb, 128, sbo);
          const uint64_t pa16 = pa >> 4, pb16 = pb >> 4;
#pragma unroll
          for (int ks = 0; ks < TC_KC / 16; ++ks) {
            if (ks * 16 >= kc) break;
            const uint64_t k16 = 16u * ks;
            const uint64_t a0 = dA + k16, a1 = a0 + pa16, a2 = a1 + pa16;
            const uint64_t b0 = dB + k16, b1 = b0 + pb16, b2 = b1 + pb16;
            const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(dbig, a0, b0, idesc, accum);
            mma_bf16(dsmall, a1, b1, idesc, accum);
            mma_bf16(dsmall, a0, b2, idesc, 1u);
            mma_bf16(dsmall, a2, b0, idesc, 1u);
            mma_bf16(dsmall, a0, b1, idesc, 1u);
            mma_bf16(dsmall, a1, b0, idesc, 1u);
          }
          tc_commit(&empty[st]);
          if (c == nchv - 1) tc_commit(&tfull[q]);
        }
      }
      tc_commit(mdone);
      if (!mbar_wait(mdone, 0)) atomicExch(bad, 1);
    }
    __syncwarp();
  } else {
    // epilogue warps: TMEM lane quarter warp % 4 = columns of this thread
    const int quarter = warp & 3;
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    float acc[NP];
#pragma unroll
    for (int n = 0; n < NP; ++n) acc[n] = 0.f;
    for (int j = 0; j < nv; ++j) {
      const int q = j & 1;
      bool ok = mbar_wait(&tfull[q], (j >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);   // the loads below need the whole warp
      if (!ok) {
        atomicExch(bad, 1);
        break;
      }
      tc_fence_after();
      if (NP > 64 && N <= 64)   // warp-uniform: only the columns this target's MMAs wrote
        drain_pair<NP, 64>(acc, tbase + lane_base + 256u * q);
      else
        drain_pair<NP, NP>(acc, tbase + lane_base + 256u * q);

      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[q]);
    }
    const int col = ct * TC_ROWS + 32 * quarter + lane;
    if (col < a.nc) {
      float* outp = a.out + row0 * a.nc + col;
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (n < nrows) outp[(size_t)n * a.nc] = acc[n];
    }
  }
  __syncthreads();
  if (*bad) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    // drain this CTA's own copies still in flight
    if (warp == 0 && lane == 0)
      for (int it = issued > TC_STAGES ? issued - TC_STAGES : 0; it < issued; ++it)
        mbar_wait(&full[it % TC_STAGES], (it / TC_STAGES) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512) : "memory");
  }
}

// ---- two sibling targets per CTA (M2L at 64 coefficients; the near field) --------------
// Sibling targets share most of their interaction lists, so one CTA takes a
// pair of them (t1, t2) and walks the merged list of their sources: per
// source, the A image (the source's multipoles, or its transposed X rows, for
// 128 columns) is fetched once and multiplied by [B1 | B2] with N = N1 + N2
// (t1 in D columns [0, N1), t2 in [64, 64 + N2)), or by the
// one B present.  Per MMA that is up to twice the output columns for the same
// A operand, and one shared-memory A read serves both targets.  t2 always
// starts at row / column 64 (so N1, N2 <= 64 when a group has two targets;
// t1's rows [N1, 64) of B are not loaded and its D columns there are never
// read).  Same pieces, products, TMEM buffers (big at 256 q, small at
// 256 q + 128), per-entry promotion and bounded waits as k_xlate_tc; a target
// absent from an entry has its columns of D skipped by the MMAs and the drain.
//  * mode 0 (M2L): targets and sources are boxes, N1 = N2 = 64, entry
//    operands: A of source box gsrc (K = Kp), B = table image gv_t.
//  * mode 1 (P2P): targets and sources are leaves, N_t = the target's padded
//    panel count, A = transposed-X rows of source leaf gsrc (K = its padded
//    panel count), B = near-block image of U-list pair gv_t.
struct Tc2Args {
  int mode, nc, nct, Kp, ncoef, src0, sum_pc;
  int y0;                              // first group of this launch (grid.y is capped at 65535)
  size_t a_img, b_img;                 // mode 0: bytes of one (box, tile) A image / one table image
  int a_row_bytes;                     // mode 1: bytes per K element of the X image
  const int32_t* gptr;                 // merged list of group g: [gptr[g], gptr[g + 1])
  const int32_t* gsrc;                 // source box (mode 0, global id) or leaf (mode 1)
  const int32_t* gv1;                  // t1's table (mode 0) or U-list pair (mode 1), -1: absent
  const int32_t* gv2;
  const int32_t* gt1;                  // target box / leaf of group g (gt2 = -1: single target)
  const int32_t* gt2;
  const int32_t* leaf_a0;              // mode 1: padded panel offset, padded count, first panel, count
  const int32_t* leaf_pc;
  const int32_t* leaf_f0;
  const int32_t* leaf_n;
  const int64_t* pair_boff;            // mode 1: byte offset of each pair's near-block image
  const float* ascale;                 // mode 0: 2^(e_A - TCH_TOP) per (source box, tile, row)
  const float* oscale;                 // mode 0: 2^(e_n - TCH_TOP) per output coefficient n
  const char* aimg;
  const char* bimg;
  float* out;
  int32_t* err;
};

// acc[n] += (sc *) both accumulators (small first) for the columns n < ncol
// (warp-uniform) of one 64-column half at taddr; 32 columns per wait
template <bool SCALE>
__device__ __forceinline__ void drain_cols(float (&acc)[64], uint32_t taddr, int ncol, float sc) {
#pragma unroll
  for (int s = 1; s >= 0; --s) {
#pragma unroll
    for (int h = 0; h < 64; h += 32) {
      if (h >= ncol) break;
      uint32_t r[32];
#pragma unroll
      for (int n0 = 0; n0 < 32; n0 += 16)
        if (h + n0 < ncol)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(r[n0 + 0]), "=r"(r[n0 + 1]), "=r"(r[n0 + 2]), "=r"(r[n0 + 3]), "=r"(r[n0 + 4]),
                "=r"(r[n0 + 5]), "=r"(r[n0 + 6]), "=r"(r[n0 + 7]), "=r"(r[n0 + 8]), "=r"(r[n0 + 9]),
                "=r"(r[n0 + 10]), "=r"(r[n0 + 11]), "=r"(r[n0 + 12]), "=r"(r[n0 + 13]), "=r"(r[n0 + 14]),
                "=r"(r[n0 + 15])
              : "r"(taddr + 128u * s + (uint32_t)(h + n0))
              : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int n = 0; n < 32; ++n)
        if (h + n < ncol)
          acc[h + n] = SCALE ? fmaf(__uint_as_float(r[n]), sc, acc[h + n]) : acc[h + n] + __uint_as_float(r[n]);
    }
  }
}

// MODE 0 (M2L): two-piece FP16 operands, three products (x0 y0 into the big
// accumulator, x0 y1 + x1 y0 into the small one), per-pair row scales and a
// per-coefficient output scale.  MODE 1 (near field): three-piece BF16, six
// products.
template <int MODE>
__global__ void __launch_bounds__(320, 1) k_xlate_tc2(Tc2Args a) {
  constexpr int PC = MODE == 0 ? TCH_PIECES : TC_PIECES;
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_stage = oz_chunk_bytes(TC_ROWS, TC_KC, PC);
  const int stage_bytes = a_stage + oz_chunk_bytes(128, TC_KC, PC);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + TC_STAGES * stage_bytes);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* tfull = empty + TC_STAGES;
  uint64_t* tfree = tfull + 2;
  uint64_t* mdone = tfree + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 1);
  int* bad = reinterpret_cast<int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x, g = a.y0 + (int)blockIdx.y;
  const int vs = a.gptr[g], ve = a.gptr[g + 1];
  const int nv = ve - vs;
  const int t1 = a.gt1[g], t2 = a.gt2[g];
  const int N1 = MODE == 0 ? 64 : a.leaf_pc[t1];
  const int N2 = t2 < 0 ? 0 : (MODE == 0 ? 64 : a.leaf_pc[t2]);
  const int PW = t2 < 0 ? N1 : 64 + N2;   // rows of a merged B piece
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&tfull[q], 1);
      mbar_init(&tfree[q], 8);
    }
    mbar_init(mdone, 1);
    *bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tslot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool stop = false;
      for (int v = vs; v < ve && !stop; ++v) {
        const int S = a.gsrc[v];
        const size_t aoff = MODE == 0 ? ((size_t)(S - a.src0) * a.nct + ct) * a.a_img
                                        : ((size_t)ct * a.sum_pc + a.leaf_a0[S]) * (size_t)a.a_row_bytes;
        const int K = MODE == 0 ? a.Kp : a.leaf_pc[S];
        const int vt[2] = {a.gv1[v], a.gv2[v]};
        const int Nt[2] = {N1, N2};
        const int nchv = (K + TC_KC - 1) / TC_KC;
        for (int c = 0; c < nchv; ++c, ++it) {
          const int st = it % TC_STAGES, u = it / TC_STAGES;
          if (u > 0 && !mbar_wait(&empty[st], (u - 1) & 1)) {
            atomicExch(bad, 1);
            stop = true;
            break;
          }
          const int kc = min(TC_KC, K - TC_KC * c);
          const uint32_t ab = oz_chunk_bytes(TC_ROWS, kc, PC);
          uint8_t* sa = base + (size_t)st * stage_bytes;
          uint8_t* sb = sa + a_stage;
          uint32_t bb = 0;
          for (int t = 0; t < 2; ++t)
            if (vt[t] >= 0) bb += PC * Nt[t] * kc * 2;
          mbar_expect_tx(&full[st], ab + bb);
          bulk_g2s(sa, a.aimg + aoff + (size_t)a_stage * c, ab, &full[st]);
          // piece h of target t's B chunk -> rows [64 t, 64 t + N_t) of merged piece h
          for (int t = 0; t < 2; ++t) {
            if (vt[t] < 0) continue;
            const uint32_t pbytes = Nt[t] * kc * 2;
            const char* bsrc = a.bimg + (MODE == 0 ? (size_t)vt[t] * a.b_img : (size_t)a.pair_boff[vt[t]]) +
                               (size_t)oz_chunk_bytes(Nt[t], TC_KC, PC) * c;
            uint8_t* bdst = sb + (size_t)t * 64 * kc * 2;
            for (int h = 0; h < PC; ++h)
              bulk_g2s(bdst + (size_t)h * PW * kc * 2, bsrc + (size_t)h * pbytes, pbytes, &full[st]);
          }
          issued = it + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // D F32; A, B BF16 (MODE 1) or F16 (MODE 0, type code 0); K-major
      const uint32_t id0 =
          (1u << 4) | (MODE == 0 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(TC_ROWS >> 4) << 24);
      int it = 0;
      bool stop = false;
      for (int v = vs, j = 0; v < ve && !stop; ++v, ++j) {
        const bool p1 = a.gv1[v] >= 0, p2 = a.gv2[v] >= 0;
        const int K = MODE == 0 ? a.Kp : a.leaf_pc[a.gsrc[v]];
        const int nchv = (K + TC_KC - 1) / TC_KC;
        const int q = j & 1;
        if (j >= 2 && !mbar_wait(&tfree[q], ((j >> 1) - 1) & 1)) {
          atomicExch(bad, 1);
          break;
        }
        const int Nm = p1 && p2 ? 64 + N2 : (p1 ? N1 : N2);
        const uint32_t idesc = id0 | ((uint32_t)(Nm >> 3) << 17);
        const uint32_t dcol = p1 ? 0u : 64u;   // t2 alone: rows and columns from 64
        for (int c = 0; c < nchv; ++c, ++it) {
          const int st = it % TC_STAGES, u = it / TC_STAGES;
          if (!mbar_wait(&full[st], u & 1)) {
            atomicExch(bad, 1);
            stop = true;
            break;
          }
          tc_fence_after();
          const int kc = min(TC_KC, K - TC_KC * c);
          const uint32_t sa = sm_u32(base + (size_t)st * stage_bytes);
          const uint32_t sb = sa + a_stage + dcol * kc * 2;
          const uint32_t pa = TC_ROWS * kc * 2, pb = PW * kc * 2;   // piece strides
          const uint32_t sbo = 16 * kc;
          const uint32_t dbig = tbase + 256u * q + dcol, dsmall = dbig + 128u;
          const uint64_t dA = sdesc(sa, 128, sbo), dB = sdesc(sb, 128, sbo);
          const uint64_t pa16 = pa >> 4, pb16 = pb >> 4;
#pragma unroll
          for (int ks = 0; ks < TC_KC / 16; ++ks) {
            if (ks * 16 >= kc) break;
            const uint64_t k16 = 16u * ks;
            const uint64_t a0 = dA + k16, a1 = a0 + pa16, a2 = a1 + pa16;
            const uint64_t b0 = dB + k16, b1 = b0 + pb16, b2 = b1 + pb16;
            const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(dbig, a0, b0, idesc, accum);
            if (MODE == 0) {
              mma_bf16(dsmall, a0, b1, idesc, accum);
              mma_bf16(dsmall, a1, b0, idesc, 1u);
            } else {
              mma_bf16(dsmall, a1, b1, idesc, accum);
              mma_bf16(dsmall, a0, b2, idesc, 1u);
              mma_bf16(dsmall, a2, b0, idesc, 1u);
              mma_bf16(dsmall, a0, b1, idesc, 1u);
              mma_bf16(dsmall, a1, b0, idesc, 1u);
            }
          }
          tc_commit(&empty[st]);
          if (c == nchv - 1) tc_commit(&tfull[q]);
        }
      }
      tc_commit(mdone);
      if (!mbar_wait(mdone, 0)) atomicExch(bad, 1);
    }
    __syncwarp();
  } else {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its columns of the right-hand
    // sides) and accumulator columns [64 h, 64 h + 64), h = (w - 2) / 4: target
    // t1 (h = 0) or t2 (h = 1), or rows 64 h.. of a lone target
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    float acc[64];
#pragma unroll
    for (int n = 0; n < 64; ++n) acc[n] = 0.f;
    for (int j = 0; j < nv; ++j) {
      const int q = j & 1;
      const bool p1 = a.gv1[vs + j] >= 0, p2 = a.gv2[vs + j] >= 0;
      bool ok = mbar_wait(&tfull[q], (j >> 1) & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        atomicExch(bad, 1);
        break;
      }
      tc_fence_after();
      int ncol;
      if (MODE == 0)
        ncol = (half == 0 ? p1 : p2) ? 64 : 0;
      else if (t2 < 0)
        ncol = p1 ? min(64, N1 - 64 * half) : 0;
      else
        ncol = half == 0 ? (p1 ? N1 : 0) : (p2 ? N2 : 0);
      if (ncol > 0) {
        const uint32_t tq = tbase + lane_base + 256u * q + 64u * half;
        if (MODE == 0)   // this row's scale for the pair's source box
          drain_cols<true>(acc, tq, 64,
                           a.ascale[((size_t)(a.gsrc[vs + j] - a.src0) * a.nct + ct) * TC_ROWS + 32 * quarter + lane]);
        else
          drain_cols<false>(acc, tq, ncol, 1.f);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[q]);
    }
    const int col = ct * TC_ROWS + 32 * quarter + lane;
    const int tg = (t2 < 0 || half == 0) ? t1 : t2;          // this half's target
    const int r0 = (t2 < 0) ? 64 * half : 0;                 // its first row in this half
    if (col < a.nc && !(MODE == 0 && t2 < 0 && half == 1)) {
      const int nr = (MODE == 0 ? a.ncoef : a.leaf_n[tg]) - r0;
      const size_t row = MODE == 0 ? (size_t)tg * a.ncoef : (size_t)a.leaf_f0[tg] + r0;
      float* o = a.out + row * a.nc + col;
#pragma unroll
      for (int n = 0; n < 64; ++n)
        if (n < nr) o[(size_t)n * a.nc] = MODE == 0 ? acc[n] * __ldg(a.oscale + n) : acc[n];
    }
  }
  __syncthreads();
  if (*bad) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 0 && lane == 0)
      for (int it = issued > TC_STAGES ? issued - TC_STAGES : 0; it < issued; ++it)
        mbar_wait(&full[it % TC_STAGES], (it / TC_STAGES) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512) : "memory");
  }
}

template <int MODE>
static size_t tc2_smem() {
  constexpr int PC = MODE == 0 ? TCH_PIECES : TC_PIECES;
  return (size_t)TC_STAGES * (oz_chunk_bytes(TC_ROWS, TC_KC, PC) + oz_chunk_bytes(128, TC_KC, PC)) + 1024 + 128;
}

template <int MODE>
static void launch_tc2_m(xrl_ctx* c, dim3 grid, const Tc2Args& g, cudaStream_t s) {
  static bool set = false;
  if (!set) {
    XRL_CUDA(
        cudaFuncSetAttribute(k_xlate_tc2<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc2_smem<MODE>()));
    set = true;
  }
  Tc2Args a = g;
  for (unsigned y0 = 0; y0 < grid.y; y0 += kMaxGridY) {
    a.y0 = (int)y0;
    k_xlate_tc2<MODE><<<dim3(grid.x, std::min(kMaxGridY, grid.y - y0)), 320, tc2_smem<MODE>(), s>>>(a);
    if (y0 > 0) count_launch(c);   // callers count one launch per translation
  }
}

static void launch_tc2(xrl_ctx* c, dim3 grid, const Tc2Args& g, cudaStream_t s) {
  if (g.mode == 0)
    launch_tc2_m<0>(c, grid, g, s);
  else
    launch_tc2_m<1>(c, grid, g, s);
}

// ---- FP64-accurate translation (Ozaki-style integer slices) ------------------------------
// For the FP64 refinement residuals: each row of A (one column c of the
// source multipoles, scale 2^eA = the power of two above max_k |M[k][c]|) and
// each column of B (one output n of the table, 2^fB likewise) is cut into
// OZ_S integer slices, x 2^-e = sum_i a_i 2^-7(i+1), |a_i| <= 128, stored in
// BF16 as a_i 2^(e-7) (exact: 8 significant bits).  A product of two slices is
// then a_i b_j 2^(eA+fB-14), and every sum over k and over the slice pairs of
// one class s = i + j is an integer multiple of that power of two below
// 5 * 81 * 2^14 < 2^24: the tensor core's FP32 accumulation is exact whatever
// its rounding.  The classes s <= OZ_S - 1 (15 products) accumulate in five
// TMEM accumulators; after every V-list pair the epilogue forms
// sum_s 2^-7s D_s and adds it into double-float registers.  Truncation
// (dropped slices and products) ~2^-35 of max|M| max|T| per row and column.
// The solid-harmonic coefficients span many octaves across the order k, so
// both operands are first equilibrated exactly by powers of two,
// M'[k] = 2^-d_k M[k], T'[k] = 2^d_k T[k] (T'^T M' = T^T M), with 2^d_k the
// size of the largest panel moment of index k.

// Pack FP64 expansions in[box][k][col] into the OZ_S-slice A image.  One CTA
// per (box, column tile); first the row scales, then the slices.
__global__ void k_oz_pack_a(int nc, int ncoef, int Kp, int b0, const int32_t* __restrict__ dk,
                            const double* __restrict__ in, uint16_t* __restrict__ img) {
  __shared__ int eA[TC_ROWS];
  const int ct = blockIdx.y;
  const double* src = in + (size_t)(b0 + blockIdx.x) * ncoef * nc + (size_t)ct * TC_ROWS;
  char* dst = reinterpret_cast<char*>(img) + ((size_t)blockIdx.x * gridDim.y + ct) * (size_t)(OZ_S * 2 * TC_ROWS * Kp);
  for (int r = threadIdx.x; r < TC_ROWS; r += blockDim.x) {
    double mx = 0.0;
    if (ct * TC_ROWS + r < nc)
      for (int k = 0; k < ncoef; ++k) mx = fmax(mx, fabs(ldexp(src[(size_t)k * nc + r], -dk[k])));
    eA[r] = mx > 0.0 ? ilogb(mx) + 1 : 0;
  }
  __syncthreads();
  const int nq = Kp >> 3;
  for (int e = threadIdx.x; e < TC_ROWS * nq; e += blockDim.x) {
    const int r = e & (TC_ROWS - 1), kq = e >> 7;
    const bool col_ok = ct * TC_ROWS + r < nc;
    const int ea = eA[r];
    uint16_t sl[OZ_S][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * kq + q;
      double x = (col_ok && k < ncoef) ? ldexp(src[(size_t)k * nc + r], -ea - dk[k]) : 0.0;
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        const double a = rint(x * 128.0);
        x = x * 128.0 - a;
        sl[i][q] = bf16_bits(ldexpf((float)a, ea - 7));
      }
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      uint4 v;
      v.x = sl[i][0] | (uint32_t)sl[i][1] << 16;
      v.y = sl[i][2] | (uint32_t)sl[i][3] << 16;
      v.z = sl[i][4] | (uint32_t)sl[i][5] << 16;
      v.w = sl[i][6] | (uint32_t)sl[i][7] << 16;
      *reinterpret_cast<uint4*>(dst + oz_img_off(TC_ROWS, Kp, r, 8 * kq, i, OZ_S)) = v;
    }
  }
}

// Pack FP64 tables T[o][k_in][n_out] into OZ_S-slice B images (Np rows n by Kp).
__global__ void k_oz_pack_b(int ncoef, int Kp, int Np, const int32_t* __restrict__ dk, const double* __restrict__ T,
                            uint16_t* __restrict__ img) {
  __shared__ int fB[128];
  const int o = blockIdx.x;
  const double* tm = T + (size_t)o * ncoef * ncoef;
  char* dst = reinterpret_cast<char*>(img) + (size_t)o * (size_t)(OZ_S * 2 * Np * Kp);
  for (int r = threadIdx.x; r < Np; r += blockDim.x) {
    double mx = 0.0;
    if (r < ncoef)
      for (int k = 0; k < ncoef; ++k) mx = fmax(mx, fabs(ldexp(tm[(size_t)k * ncoef + r], dk[k])));
    fB[r] = mx > 0.0 ? ilogb(mx) + 1 : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Np * Kp; e += blockDim.x) {
    const int r = e % Np, k = e / Np;
    const int fb = fB[r];
    double x = (r < ncoef && k < ncoef) ? ldexp(tm[(size_t)k * ncoef + r], dk[k] - fb) : 0.0;
    for (int i = 0; i < OZ_S; ++i) {
      const double a = rint(x * 128.0);
      x = x * 128.0 - a;
      *reinterpret_cast<uint16_t*>(dst + oz_img_off(Np, Kp, r, k, i, OZ_S)) = bf16_bits(ldexpf((float)a, fb - 7));
    }
  }
}

struct OzArgs {
  XlPairs pr;
  int nc;
  const char* aimg;
  const char* bimg;
  double* out;
  int32_t* err;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Warps: 0 = bulk copies (lane 0; the whole warp owns TMEM), 1 = MMA issuer
// (lane 0), 2..9 = epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and
// outputs n in [NP/2 h, NP/2 (h + 1)), h = (w - 2) / 4.  TMEM: class s at
// columns NP s (5 NP <= 480).  One accumulator set: the MMAs of pair j+1 start once every
// epilogue warp has loaded pair j (tfree).
template <int NP>
__global__ void __launch_bounds__(320, 1) k_xlate_oz(OzArgs a) {
  constexpr int NH = NP / 2;   // output columns per epilogue half
  extern __shared__ uint8_t oz_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_stage = oz_chunk_bytes(TC_ROWS, TC_KC, OZ_S);
  const int stage_bytes = a_stage + oz_chunk_bytes(NP, TC_KC, OZ_S);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + OZ_STAGES * stage_bytes);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* tfull = empty + OZ_STAGES;
  uint64_t* tfree = tfull + 1;
  uint64_t* mdone = tfree + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 1);
  int* bad = reinterpret_cast<int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x;
  int vs, ve, N, nrows;
  size_t row0;
  xl_target(a.pr, NP, vs, ve, N, nrows, row0);
  const int nv = ve - vs;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tfree, 8);
    mbar_init(mdone, 1);
    *bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tslot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      bool stop = false;
      for (int v = vs; v < ve && !stop; ++v) {
        size_t aoff, boff;
        int K;
        xl_pair(a.pr, v, ct, aoff, boff, K);
        const int nchv = (K + TC_KC - 1) / TC_KC;
        for (int c = 0; c < nchv; ++c, ++it) {
          const int st = it % OZ_STAGES, u = it / OZ_STAGES;
          if (u > 0 && !mbar_wait(&empty[st], (u - 1) & 1)) {
            atomicExch(bad, 1);
            stop = true;
            break;
          }
          const int kc = min(TC_KC, K - TC_KC * c);
          const char* asrc = a.aimg + aoff + (size_t)a_stage * c;
          const char* bsrc = a.bimg + boff + (size_t)oz_chunk_bytes(N, TC_KC, OZ_S) * c;
          const uint32_t ab = oz_chunk_bytes(TC_ROWS, kc, OZ_S), bb = oz_chunk_bytes(N, kc, OZ_S);
          uint8_t* sa = base + (size_t)st * stage_bytes;
          mbar_expect_tx(&full[st], ab + bb);
          bulk_g2s(sa, asrc, ab, &full[st]);
          bulk_g2s(sa + a_stage, bsrc, bb, &full[st]);
          issued = it + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
      int it = 0;
      bool stop = false;
      for (int v = vs, j = 0; v < ve && !stop; ++v, ++j) {
        size_t aoff, boff;
        int K;
        xl_pair(a.pr, v, ct, aoff, boff, K);
        const int nchv = (K + TC_KC - 1) / TC_KC;
        if (j >= 1 && !mbar_wait(tfree, (j - 1) & 1)) {
          atomicExch(bad, 1);
          break;
        }
        for (int c = 0; c < nchv; ++c, ++it) {
          const int st = it % OZ_STAGES, u = it / OZ_STAGES;
          if (!mbar_wait(&full[st], u & 1)) {
            atomicExch(bad, 1);
            stop = true;
            break;
          }
          tc_fence_after();
          const int kc = min(TC_KC, K - TC_KC * c);
          const uint32_t sa = sm_u32(base + (size_t)st * stage_bytes);
          const uint32_t sb = sa + a_stage;
          const uint32_t pa = TC_ROWS * kc * 2, pb = N * kc * 2;
          const uint32_t sbo = 16 * kc;
          const uint64_t dA = sdesc(sa, 128, sbo), dB = sdesc(sb, 128, sbo);
          const uint64_t pa16 = pa >> 4, pb16 = pb >> 4;
#pragma unroll
          for (int ks = 0; ks < TC_KC / 16; ++ks) {
            if (ks * 16 >= kc) break;
            uint64_t da[OZ_S], db[OZ_S];
#pragma unroll
            for (int h = 0; h < OZ_S; ++h) {
              da[h] = dA + 16u * ks + h * pa16;
              db[h] = dB + 16u * ks + h * pb16;
            }
            const bool first = c == 0 && ks == 0;
#pragma unroll
            for (int sc = 0; sc < OZ_S; ++sc)
#pragma unroll
              for (int i = 0; i <= sc; ++i)
                mma_bf16(tbase + (uint32_t)NP * sc, da[i], db[sc - i], idesc, (first && i == 0) ? 0u : 1u);
          }
          tc_commit(&empty[st]);
          if (c == nchv - 1) tc_commit(tfull);
        }
      }
      tc_commit(mdone);
      if (!mbar_wait(mdone, 0)) atomicExch(bad, 1);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    float ah[NH], al[NH];
#pragma unroll
    for (int n = 0; n < NH; ++n) ah[n] = al[n] = 0.f;
    for (int j = 0; j < nv; ++j) {
      bool ok = mbar_wait(tfull, j & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        atomicExch(bad, 1);
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int n0 = 0; n0 < NH; n0 += 8) {
        uint32_t r[OZ_S][8];
#pragma unroll
        for (int sc = 0; sc < OZ_S; ++sc)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(r[sc][0]), "=r"(r[sc][1]), "=r"(r[sc][2]), "=r"(r[sc][3]), "=r"(r[sc][4]),
                         "=r"(r[sc][5]), "=r"(r[sc][6]), "=r"(r[sc][7])
                       : "r"(tbase + lane_base + (uint32_t)NP * sc + (uint32_t)(NH * half + n0))
                       : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (n0 == NH - 8) {
          // every value of this pair is in registers: let the next pair's MMAs start
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tfree);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          // sum_s 2^-7s D_s as a float pair.  Classes 2-4 (below 2^-14 of the
          // leading class) are summed in plain FP32: their rounding, ~2^-24 of
          // their sum, is ~2^-38 of the result, under the slices' own 2^-35
          // truncation.  Classes 0 and 1 and the running sum take error-free
          // additions.  (Scaling by a power of two is exact, as is the product
          // by the constant.)
          const float t = fmaf(__uint_as_float(r[4][q]), 0x1p-28f,
                               fmaf(__uint_as_float(r[3][q]), 0x1p-21f, __uint_as_float(r[2][q]) * 0x1p-14f));
          float h, e;
          two_sum(__uint_as_float(r[0][q]), __uint_as_float(r[1][q]) * 0x1p-7f, h, e);
          const float l = e + t;
          two_sum(ah[n0 + q], h, ah[n0 + q], e);
          al[n0 + q] += e + l;
        }
      }
    }
    const int col = ct * TC_ROWS + 32 * quarter + lane;
    if (col < a.nc) {
      double* outp = a.out + row0 * a.nc + col;
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        const int n = NH * half + q;
        if (n < nrows) outp[(size_t)n * a.nc] = (double)ah[q] + (double)al[q];
      }
    }
  }
  __syncthreads();
  if (*bad) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 0 && lane == 0)
      for (int it = issued > OZ_STAGES ? issued - OZ_STAGES : 0; it < issued; ++it)
        mbar_wait(&full[it % OZ_STAGES], (it / OZ_STAGES) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512) : "memory");
  }
}

// ---- near field on the tensor cores: packing ----------------------------------------------
// Transposed-X image (A operand of mode 1): for leaf S and column tile ct the
// rows are the columns ct*128 + r and K runs over the leaf's panels (padded to
// 16); images of all leaves of one tile are contiguous, [ct][padded panel].
__global__ void k_tcp_pack_x(int nc, int sum_pc, const int32_t* __restrict__ leaf_f0,
                             const int32_t* __restrict__ leaf_n, const int32_t* __restrict__ leaf_a0,
                             const int32_t* __restrict__ leaf_pc, const float* __restrict__ X,
                             uint16_t* __restrict__ img) {
  const int S = blockIdx.x, ct = blockIdx.y;
  const int pc = leaf_pc[S], n = leaf_n[S], f0 = leaf_f0[S];
  char* dst = reinterpret_cast<char*>(img) + ((size_t)ct * sum_pc + leaf_a0[S]) * (size_t)(TC_PIECES * TC_ROWS * 2);
  for (int e = threadIdx.x; e < TC_ROWS * (pc >> 3); e += blockDim.x) {
    const int r = e & (TC_ROWS - 1), kq = e >> 7;
    const int col = ct * TC_ROWS + r;
    uint16_t p0[8], p1[8], p2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * kq + q;
      const float x = (col < nc && k < n) ? X[(size_t)(f0 + k) * nc + col] : 0.f;
      p0[q] = bf16_bits(x);
      const float r1 = x - bf16_val(p0[q]);
      p1[q] = bf16_bits(r1);
      p2[q] = bf16_bits(r1 - bf16_val(p1[q]));
    }
    uint4 v0, v1, v2;
    v0.x = p0[0] | (uint32_t)p0[1] << 16; v0.y = p0[2] | (uint32_t)p0[3] << 16;
    v0.z = p0[4] | (uint32_t)p0[5] << 16; v0.w = p0[6] | (uint32_t)p0[7] << 16;
    v1.x = p1[0] | (uint32_t)p1[1] << 16; v1.y = p1[2] | (uint32_t)p1[3] << 16;
    v1.z = p1[4] | (uint32_t)p1[5] << 16; v1.w = p1[6] | (uint32_t)p1[7] << 16;
    v2.x = p2[0] | (uint32_t)p2[1] << 16; v2.y = p2[2] | (uint32_t)p2[3] << 16;
    v2.z = p2[4] | (uint32_t)p2[5] << 16; v2.w = p2[6] | (uint32_t)p2[7] << 16;
    *reinterpret_cast<uint4*>(dst + tc_img_off(TC_ROWS, pc, r, 8 * kq, 0)) = v0;
    *reinterpret_cast<uint4*>(dst + tc_img_off(TC_ROWS, pc, r, 8 * kq, 1)) = v1;
    *reinterpret_cast<uint4*>(dst + tc_img_off(TC_ROWS, pc, r, 8 * kq, 2)) = v2;
  }
}

// Near-matrix block of U-list pair v (B operand of mode 1), from the FP64
// values: rows n < N_T (target panels, padded to 16), K = the source leaf's
// panels (padded to 16).  One CTA per pair.
__global__ void k_tcp_pack_v(const int32_t* __restrict__ pair_tgt, const int32_t* __restrict__ u_src,
                             const int32_t* __restrict__ pair_col, const int32_t* __restrict__ leaf_n,
                             const int32_t* __restrict__ leaf_pc, const int64_t* __restrict__ near_off,
                             const int32_t* __restrict__ near_w, const int64_t* __restrict__ pair_boff,
                             const double* __restrict__ val, uint16_t* __restrict__ img) {
  const int v = blockIdx.x;
  const int T = pair_tgt[v], S = u_src[v];
  const int nT = leaf_n[T], nS = leaf_n[S], N = (nT + 15) & ~15, pc = leaf_pc[S], w = near_w[T];
  const double* vb = val + near_off[T] + pair_col[v];
  char* dst = reinterpret_cast<char*>(img) + pair_boff[v];
  for (int e = threadIdx.x; e < N * pc; e += blockDim.x) {
    const int r = e % N, k = e / N;
    const double x = (r < nT && k < nS) ? vb[(size_t)r * w + k] : 0.0;
    const uint16_t b0 = bf16_bits(__double2float_rn(x));
    const double r1 = x - (double)bf16_val(b0);
    const uint16_t b1 = bf16_bits(__double2float_rn(r1));
    const uint16_t b2 = bf16_bits(__double2float_rn(r1 - (double)bf16_val(b1)));
    *reinterpret_cast<uint16_t*>(dst + tc_img_off(N, pc, r, k, 0)) = b0;
    *reinterpret_cast<uint16_t*>(dst + tc_img_off(N, pc, r, k, 1)) = b1;
    *reinterpret_cast<uint16_t*>(dst + tc_img_off(N, pc, r, k, 2)) = b2;
  }
}

// The same two operands as integer slices for the FP64-accurate near field:
// X rows scaled per (leaf, column), near blocks per (pair, target panel), each
// by the power of two above its largest magnitude (see k_oz_pack_a).
__global__ void k_ozp_pack_x(int nc, int sum_pc, const int32_t* __restrict__ leaf_f0,
                             const int32_t* __restrict__ leaf_n, const int32_t* __restrict__ leaf_a0,
                             const int32_t* __restrict__ leaf_pc, const double* __restrict__ X,
                             uint16_t* __restrict__ img) {
  __shared__ int eA[TC_ROWS];
  const int S = blockIdx.x, ct = blockIdx.y;
  const int pc = leaf_pc[S], n = leaf_n[S], f0 = leaf_f0[S];
  char* dst = reinterpret_cast<char*>(img) + ((size_t)ct * sum_pc + leaf_a0[S]) * (size_t)(OZ_S * TC_ROWS * 2);
  for (int r = threadIdx.x; r < TC_ROWS; r += blockDim.x) {
    const int col = ct * TC_ROWS + r;
    double mx = 0.0;
    if (col < nc)
      for (int k = 0; k < n; ++k) mx = fmax(mx, fabs(X[(size_t)(f0 + k) * nc + col]));
    eA[r] = mx > 0.0 ? ilogb(mx) + 1 : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TC_ROWS * (pc >> 3); e += blockDim.x) {
    const int r = e & (TC_ROWS - 1), kq = e >> 7;
    const int col = ct * TC_ROWS + r;
    const int ea = eA[r];
    uint16_t sl[OZ_S][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * kq + q;
      double x = (col < nc && k < n) ? ldexp(X[(size_t)(f0 + k) * nc + col], -ea) : 0.0;
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) {
        const double a = rint(x * 128.0);
        x = x * 128.0 - a;
        sl[i][q] = bf16_bits(ldexpf((float)a, ea - 7));
      }
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      uint4 v;
      v.x = sl[i][0] | (uint32_t)sl[i][1] << 16;
      v.y = sl[i][2] | (uint32_t)sl[i][3] << 16;
      v.z = sl[i][4] | (uint32_t)sl[i][5] << 16;
      v.w = sl[i][6] | (uint32_t)sl[i][7] << 16;
      *reinterpret_cast<uint4*>(dst + oz_img_off(TC_ROWS, pc, r, 8 * kq, i, OZ_S)) = v;
    }
  }
}

__global__ void k_ozp_pack_v(const int32_t* __restrict__ pair_tgt, const int32_t* __restrict__ u_src,
                             const int32_t* __restrict__ pair_col, const int32_t* __restrict__ leaf_n,
                             const int32_t* __restrict__ leaf_pc, const int64_t* __restrict__ near_off,
                             const int32_t* __restrict__ near_w, const int64_t* __restrict__ pair_boff,
                             const double* __restrict__ val, uint16_t* __restrict__ img) {
  __shared__ int fB[96];
  const int v = blockIdx.x;
  const int T = pair_tgt[v], S = u_src[v];
  const int nT = leaf_n[T], nS = leaf_n[S], N = (nT + 15) & ~15, pc = leaf_pc[S], w = near_w[T];
  const double* vb = val + near_off[T] + pair_col[v];
  char* dst = reinterpret_cast<char*>(img) + pair_boff[v];
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    double mx = 0.0;
    if (r < nT)
      for (int k = 0; k < nS; ++k) mx = fmax(mx, fabs(vb[(size_t)r * w + k]));
    fB[r] = mx > 0.0 ? ilogb(mx) + 1 : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * pc; e += blockDim.x) {
    const int r = e % N, k = e / N;
    const int fb = fB[r];
    double x = (r < nT && k < nS) ? ldexp(vb[(size_t)r * w + k], -fb) : 0.0;
    for (int i = 0; i < OZ_S; ++i) {
      const double a = rint(x * 128.0);
      x = x * 128.0 - a;
      *reinterpret_cast<uint16_t*>(dst + oz_img_off(N, pc, r, k, i, OZ_S)) = bf16_bits(ldexpf((float)a, fb - 7));
    }
  }
}

// Moment images of the leaves for P2M on the tensor cores (mode 2), from the
// FP64 moments S[panel][k] in 3 BF16 pieces: rows n = coefficients (Np),
// K = the leaf's panels padded to 16, value S[f0 + k][n].
__device__ __forceinline__ void put3(char* dst, size_t o0, size_t o1, size_t o2, double x) {
  const uint16_t b0 = bf16_bits(__double2float_rn(x));
  const double r1 = x - (double)bf16_val(b0);
  const uint16_t b1 = bf16_bits(__double2float_rn(r1));
  const uint16_t b2 = bf16_bits(__double2float_rn(r1 - (double)bf16_val(b1)));
  *reinterpret_cast<uint16_t*>(dst + o0) = b0;
  *reinterpret_cast<uint16_t*>(dst + o1) = b1;
  *reinterpret_cast<uint16_t*>(dst + o2) = b2;
}

__global__ void k_tcm_pack_p2m(int ncoef, int Np, const int32_t* __restrict__ leaf_f0,
                               const int32_t* __restrict__ leaf_n, const int32_t* __restrict__ leaf_pc,
                               const int64_t* __restrict__ boff, const double* __restrict__ S,
                               uint16_t* __restrict__ img) {
  const int L = blockIdx.x;
  const int f0 = leaf_f0[L], n = leaf_n[L], pc = leaf_pc[L];
  char* dst = reinterpret_cast<char*>(img) + boff[L];
  for (int e = threadIdx.x; e < Np * pc; e += blockDim.x) {
    const int r = e % Np, k = e / Np;
    const double x = (r < ncoef && k < n) ? S[(size_t)(f0 + k) * ncoef + r] : 0.0;
    put3(dst, tc_img_off(Np, pc, r, k, 0), tc_img_off(Np, pc, r, k, 1), tc_img_off(Np, pc, r, k, 2), x);
  }
}

// ---- host side ---------------------------------------------------------------------------

static int tc_kpad(int ncoef) { return (ncoef + 15) & ~15; }
static int tc_npad(int ncoef) { return (ncoef + 15) & ~15; }

bool tc_usable(const xrl_ctx* c, int nc) {
  return c->opt.tensor_cores != 0 && nc >= 64 && tc_npad(c->ncoef) <= 96 && c->d.tc_bimg.n > 0;
}

static XlPairs m2l_pairs(const xrl_ctx* c, int b0, int nct, int pieces, size_t a_img, size_t b_img) {
  XlPairs p = {};
  p.mode = 0;
  p.b0 = b0;
  p.src0 = c->tree.level_off[2];
  p.nct = nct;
  p.Kp = tc_kpad(c->ncoef);
  p.ncoef = c->ncoef;
  p.a_img = a_img;
  p.b_img = b_img;
  p.a_row_bytes = pieces * TC_ROWS * 2;
  p.ptr = c->d.v_ptr32.p;
  p.src = c->d.v_src.p;
  p.off = c->d.v_off.p;
  return p;
}

static XlPairs p2p_pairs(const xrl_ctx* c, int nct, int pieces, const int64_t* boff) {
  XlPairs p = {};
  p.mode = 1;
  p.nct = nct;
  p.sum_pc = c->tcp_sum_pc;
  p.a_row_bytes = pieces * TC_ROWS * 2;
  p.ptr = c->d.u_ptr32.p;
  p.src = c->d.u_src.p;
  p.leaf_a0 = c->d.tcp_a0.p;
  p.leaf_pc = c->d.tcp_pc.p;
  p.leaf_f0 = c->d.leaf_first.p;
  p.leaf_n = c->d.leaf_count.p;
  p.pair_boff = boff;
  return p;
}

template <int NP>
static void launch_tc(xrl_ctx* c, dim3 g, const TcArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)TC_STAGES * (tc_chunk_bytes(TC_ROWS, TC_KC) + tc_chunk_bytes(NP, TC_KC)) + 1024 + 128;
  static bool set = false;
  if (!set) {
    XRL_CUDA(cudaFuncSetAttribute(k_xlate_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set = true;
  }
  TcArgs b = a;
  for (unsigned y0 = 0; y0 < g.y; y0 += kMaxGridY) {
    b.pr.y0 = (int)y0;
    k_xlate_tc<NP><<<dim3(g.x, std::min(kMaxGridY, g.y - y0)), 192, smem, s>>>(b);
    if (y0 > 0) count_launch(c);   // callers count one launch per translation
  }
}

template <int NP>
static void launch_oz_np(xrl_ctx* c, dim3 g, const OzArgs& a, cudaStream_t s) {
  const size_t smem =
      (size_t)OZ_STAGES * (oz_chunk_bytes(TC_ROWS, TC_KC, OZ_S) + oz_chunk_bytes(NP, TC_KC, OZ_S)) + 1024 + 128;
  static bool set = false;
  if (!set) {
    XRL_CUDA(cudaFuncSetAttribute(k_xlate_oz<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set = true;
  }
  OzArgs b = a;
  for (unsigned y0 = 0; y0 < g.y; y0 += kMaxGridY) {
    b.pr.y0 = (int)y0;
    k_xlate_oz<NP><<<dim3(g.x, std::min(kMaxGridY, g.y - y0)), 320, smem, s>>>(b);
    if (y0 > 0) count_launch(c);   // callers count one launch per translation
  }
}

static void launch_oz(xrl_ctx* c, int Np, dim3 g, const OzArgs& a, cudaStream_t s) {
  if (Np <= 64)
    launch_oz_np<64>(c, g, a, s);
  else
    launch_oz_np<96>(c, g, a, s);
}

static void p2p_groups(xrl_ctx* c, const std::vector<int32_t>& pc);

// Near-field layout for the tensor cores: leaves padded to 16 panels, the
// pair offsets of the near-block images, and the FP32 images themselves.
static void tcp_prepare(xrl_ctx* c) {
  const Tree& t = c->tree;
  const int nl = t.n_leaves();
  int maxn = 0;
  for (int L = 0; L < nl; ++L) maxn = std::max(maxn, (int)t.leaf_count[L]);
  if (maxn > 96 || nl == 0) return;
  std::vector<int32_t> a0(nl), pc(nl);
  int sum = 0;
  for (int L = 0; L < nl; ++L) {
    pc[L] = ((int)t.leaf_count[L] + 15) & ~15;
    a0[L] = sum;
    sum += pc[L];
  }
  const size_t np = t.u_src.size();
  std::vector<int32_t> tgt(np), col(np);
  std::vector<int64_t> boff(np), zoff(np);
  int64_t b = 0, z = 0;
  for (int T = 0; T < nl; ++T) {
    int cacc = 0;
    const int N = ((int)t.leaf_count[T] + 15) & ~15;
    for (int64_t q = t.u_ptr[T]; q < t.u_ptr[T + 1]; ++q) {
      const int S = t.u_src[q];
      tgt[q] = T;
      col[q] = cacc;
      cacc += t.leaf_count[S];
      boff[q] = b;
      zoff[q] = z;
      b += (int64_t)TC_PIECES * 2 * N * pc[S];
      z += (int64_t)OZ_S * 2 * N * pc[S];
    }
  }
  c->tcp_sum_pc = sum;
  c->stats.near_nnz_padded = b / (TC_PIECES * 2);
  c->tcp_img_bytes = b;
  c->ozp_img_bytes = z;
  c->d.tcp_a0.upload(c->alloc, a0);
  c->d.tcp_pc.upload(c->alloc, pc);
  c->d.tcp_tgt.upload(c->alloc, tgt);
  c->d.tcp_col.upload(c->alloc, col);
  c->d.tcp_boff.upload(c->alloc, boff);
  c->d.ozp_boff.upload(c->alloc, zoff);
  c->d.tcp_vimg.alloc(c->alloc, (size_t)(b / 2));
  p2p_groups(c, pc);
  k_tcp_pack_v<<<(unsigned)np, 256, 0, c->stream>>>(c->d.tcp_tgt.p, c->d.u_src.p, c->d.tcp_col.p, c->d.leaf_count.p,
                                                    c->d.tcp_pc.p, c->d.near_off.p, c->d.near_w.p, c->d.tcp_boff.p,
                                                    c->d.near_val.p, c->d.tcp_vimg.p);
  XRL_CUDA(cudaGetLastError());
}

// Images of the upward pass of the FP32 product (the 8 M2M tables, the
// leaves' P2M moment images); needs the near-field layout of tcp_prepare.
static void tcm_prepare(xrl_ctx* c) {
  const Tree& t = c->tree;
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = tc_npad(ncoef);
  const int nl = t.n_leaves();
  c->d.tc_m2m_img.alloc(c->alloc, (size_t)8 * TC_PIECES * Np * Kp);
  k_tc_pack_b<<<8, 256, 0, c->stream>>>(ncoef, Kp, Np, c->d.t_m2m.p, c->d.tc_m2m_img.p);
  std::vector<int64_t> b2(nl);
  int64_t o2 = 0;
  for (int L = 0; L < nl; ++L) {
    const int n = t.leaf_count[L], pc = (n + 15) & ~15;
    b2[L] = o2;
    o2 += (int64_t)TC_PIECES * 2 * Np * pc;
  }
  c->d.tcm_boff2.upload(c->alloc, b2);
  c->d.tcm_p2m_img.alloc(c->alloc, (size_t)(o2 / 2));
  k_tcm_pack_p2m<<<nl, 256, 0, c->stream>>>(ncoef, Np, c->d.leaf_first.p, c->d.leaf_count.p, c->d.tcp_pc.p,
                                             c->d.tcm_boff2.p, c->d.mom.p, c->d.tcm_p2m_img.p);
  XRL_CUDA(cudaGetLastError());
}

// Sibling pairs for k_xlate_tc2: consecutive targets with the same parent
// are taken two at a time when `pairable` allows (else alone); each group's
// lists (sorted by source) are merged by source.  lptr/lsrc: the targets'
// interaction lists; an entry's value is `val(i)` for list position i.
template <class Parent, class Pairable, class Val>
static void build_groups(int n_t, int t0, const std::vector<int64_t>& lptr, const std::vector<int32_t>& lsrc,
                         Parent parent, Pairable pairable, Val val, xrl_ctx* c, DBuf<int32_t>& dptr,
                         DBuf<int32_t>& dsrc, DBuf<int32_t>& dt1, DBuf<int32_t>& dt2, DBuf<int32_t>& dv1,
                         DBuf<int32_t>& dv2) {
  std::vector<int32_t> gptr{0}, gsrc, gt1, gt2, gv1, gv2;
  for (int b = t0; b < t0 + n_t;) {
    const int b2 = (b + 1 < t0 + n_t && parent(b + 1) == parent(b) && pairable(b, b + 1)) ? b + 1 : -1;
    gt1.push_back(b);
    gt2.push_back(b2);
    int64_t i = lptr[b], ie = lptr[b + 1];
    int64_t j = b2 >= 0 ? lptr[b2] : 0, je = b2 >= 0 ? lptr[b2 + 1] : 0;
    while (i < ie || j < je) {
      const int si = i < ie ? lsrc[i] : INT32_MAX, sj = j < je ? lsrc[j] : INT32_MAX;
      const int sm = std::min(si, sj);
      gsrc.push_back(sm);
      gv1.push_back(si == sm ? val(i++) : -1);
      gv2.push_back(sj == sm ? val(j++) : -1);
    }
    gptr.push_back((int32_t)gsrc.size());
    b = b2 >= 0 ? b2 + 1 : b + 1;
  }
  dptr.upload(c->alloc, gptr);
  dsrc.upload(c->alloc, gsrc);
  dt1.upload(c->alloc, gt1);
  dt2.upload(c->alloc, gt2);
  dv1.upload(c->alloc, gv1);
  dv2.upload(c->alloc, gv2);
}

// M2L groups over all boxes of levels >= 2 (entry value: the table index)
static void m2l_groups(xrl_ctx* c) {
  const Tree& t = c->tree;
  const int b0 = t.level_off[2];
  build_groups(t.n_boxes() - b0, b0, t.v_ptr, t.v_src, [&](int b) { return t.parent[b]; },
               [](int, int) { return true; }, [&](int64_t i) { return (int32_t)t.v_off[i]; }, c, c->d.m2l_gptr,
               c->d.m2l_gsrc, c->d.m2l_gt1, c->d.m2l_gt2, c->d.m2l_gv1, c->d.m2l_gv2);
}

// near-field groups over the leaves (entry value: the U-list pair index);
// two leaves share a CTA when both have at most 64 padded panels
static void p2p_groups(xrl_ctx* c, const std::vector<int32_t>& pc) {
  const Tree& t = c->tree;
  const int leaf0 = t.level_off[t.L];
  build_groups(t.n_leaves(), 0, t.u_ptr, t.u_src, [&](int T) { return t.parent[leaf0 + T]; },
               [&](int T1, int T2) { return pc[T1] <= 64 && pc[T2] <= 64; },
               [](int64_t q) { return (int32_t)q; }, c, c->d.p2p_gptr, c->d.p2p_gsrc, c->d.p2p_gt1,
               c->d.p2p_gt2, c->d.p2p_gv1, c->d.p2p_gv2);
}

static void tch_prepare(xrl_ctx* c, int noff);

void tc_prepare(xrl_ctx* c) {
  const int ncoef = c->ncoef;
  if (c->opt.tensor_cores == 0) return;
  c->d.tc_err.alloc(c->alloc, 1);
  XRL_CUDA(cudaMemsetAsync(c->d.tc_err.p, 0, sizeof(int32_t), c->stream));
  tcp_prepare(c);
  // expansions of 49..96 coefficients (orders 6-8) take the 64- and 96-wide
  // tiles; smaller orders stay on the CUDA-core translation kernels
  if (tc_npad(ncoef) > 96 || tc_npad(ncoef) < 64) return;
  const int Kp = tc_kpad(ncoef), Np = tc_npad(ncoef);
  const int noff = (int)(c->tree.m2l_offsets.size() / 3);
  if (noff == 0) return;
  c->d.tc_bimg.alloc(c->alloc, (size_t)noff * TC_PIECES * Np * Kp);
  k_tc_pack_b<<<noff, 256, 0, c->stream>>>(ncoef, Kp, Np, c->d.t_m2l.p, c->d.tc_bimg.p);
  XRL_CUDA(cudaGetLastError());
  if (Np == 64) {
    m2l_groups(c);
    tch_prepare(c, noff);
  }
  if (c->d.tcp_vimg.n > 0) tcm_prepare(c);
}

bool tcm_usable(const xrl_ctx* c, int nc) {
  return tc_usable(c, nc) && tcp_usable(c, nc) && c->d.tcm_p2m_img.n > 0;
}

static void launch_tc_np(xrl_ctx* c, int Np, dim3 g, const TcArgs& a, cudaStream_t s) {
  if (Np <= 64)
    launch_tc<64>(c, g, a, s);
  else
    launch_tc<96>(c, g, a, s);
}

// M = S^T X for the leaves (mode 2); the transposed-X image of the near
// field's pass (tc_p2p) must already hold this product's X.  One launch.
void tc_p2m(xrl_ctx* c, int nc, float* Mx, cudaStream_t s) {
  const Tree& t = c->tree;
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  TcArgs a;
  a.pr = p2p_pairs(c, nct, TC_PIECES, c->d.tcm_boff2.p);
  a.pr.mode = 2;
  a.pr.b0 = t.level_off[t.L];
  a.pr.ncoef = c->ncoef;
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.tcp_ximg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.tcm_p2m_img.p);
  a.out = Mx;
  a.err = c->d.tc_err.p;
  launch_tc_np(c, tc_npad(c->ncoef), dim3(nct, t.n_leaves()), a, s);
}

// one level of M2M (parents at level l from their children at l + 1): pack
// the children's multipoles, then translate; two launches
void tc_m2m(xrl_ctx* c, int l, int nc, float* Mx, cudaStream_t s) {
  const Tree& t = c->tree;
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = tc_npad(ncoef);
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  const int s0 = t.level_off[l + 1], ns = t.level_off[l + 2] - s0;
  const int nt = t.level_off[l + 1] - t.level_off[l];
  c->d.tc_aimg.ensure(c->alloc, (size_t)ns * nct * TC_PIECES * TC_ROWS * Kp);
  k_tc_pack_a<<<dim3(ns, nct), 256, 0, s>>>(nc, ncoef, Kp, s0, Mx, c->d.tc_aimg.p);
  TcArgs a;
  a.pr = m2l_pairs(c, t.level_off[l], nct, TC_PIECES, (size_t)TC_PIECES * 2 * TC_ROWS * Kp,
                   (size_t)TC_PIECES * 2 * Np * Kp);
  a.pr.src0 = s0;
  a.pr.ptr = c->d.box_child_ptr.p;
  a.pr.src = c->d.box_iota.p;
  a.pr.off = c->d.box_oct16.p;
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.tc_aimg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.tc_m2m_img.p);
  a.out = Mx;
  a.err = c->d.tc_err.p;
  launch_tc_np(c, Np, dim3(nct, nt), a, s);
}

// M2L of the FP32 pass: in = M, out = L over all target boxes [b0, b0 + nbx);
// two launches (pack, translate)
void tc_m2l(xrl_ctx* c, int nbx, int b0, int nc, const float* Mx, float* Lx, cudaStream_t s) {
  const Tree& t = c->tree;
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = tc_npad(ncoef);
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  const int src0 = t.level_off[2];
  const int nsrc = t.n_boxes() - src0;
  if (Np == 64 && c->tc_targets == 2 && c->d.m2l_gptr.n > 1 && c->d.tch_bimg.n > 0 && b0 == src0 &&
      nbx == nsrc) {
    // two sibling targets per CTA, two-piece FP16 operands
    c->d.tch_aimg.ensure(c->alloc, (size_t)nsrc * nct * TCH_PIECES * TC_ROWS * Kp);
    c->d.tch_ascale.ensure(c->alloc, (size_t)nsrc * nct * TC_ROWS);
    k_tch_pack_a<<<dim3(nsrc, nct), 256, 0, s>>>(nc, ncoef, Kp, src0, c->d.oz_dk.p, Mx, c->d.tch_aimg.p,
                                                 c->d.tch_ascale.p);
    Tc2Args g = {};
    g.mode = 0;
    g.nc = nc;
    g.nct = nct;
    g.Kp = Kp;
    g.ncoef = ncoef;
    g.src0 = src0;
    g.a_img = (size_t)TCH_PIECES * 2 * TC_ROWS * Kp;
    g.b_img = (size_t)TCH_PIECES * 2 * Np * Kp;
    g.gptr = c->d.m2l_gptr.p;
    g.gsrc = c->d.m2l_gsrc.p;
    g.gv1 = c->d.m2l_gv1.p;
    g.gv2 = c->d.m2l_gv2.p;
    g.gt1 = c->d.m2l_gt1.p;
    g.gt2 = c->d.m2l_gt2.p;
    g.ascale = c->d.tch_ascale.p;
    g.oscale = c->d.tch_oscale.p;
    g.aimg = reinterpret_cast<const char*>(c->d.tch_aimg.p);
    g.bimg = reinterpret_cast<const char*>(c->d.tch_bimg.p);
    g.out = Lx;
    g.err = c->d.tc_err.p;
    launch_tc2(c, dim3(nct, (unsigned)(c->d.m2l_gptr.n - 1)), g, s);
    return;
  }
  c->d.tc_aimg.ensure(c->alloc, (size_t)nsrc * nct * TC_PIECES * TC_ROWS * Kp);
  k_tc_pack_a<<<dim3(nsrc, nct), 256, 0, s>>>(nc, ncoef, Kp, src0, Mx, c->d.tc_aimg.p);
  TcArgs a;
  a.pr = m2l_pairs(c, b0, nct, TC_PIECES, (size_t)TC_PIECES * 2 * TC_ROWS * Kp, (size_t)TC_PIECES * 2 * Np * Kp);
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.tc_aimg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.tc_bimg.p);
  a.out = Lx;
  a.err = c->d.tc_err.p;
  launch_tc_np(c, Np, dim3(nct, nbx), a, s);
}

bool tc64_usable(const xrl_ctx* c, int nc) {
  return c->opt.tensor_cores != 0 && nc >= 64 && tc_npad(c->ncoef) <= 96 && tc_npad(c->ncoef) >= 64 &&
         c->d.tc_err.n > 0;
}

// One-time images of the FP64-accurate pass: the equilibration exponents d_k
// (from the panel moments, the P2M operator: typical size of M[k]) and the
// integer-slice images of the M2L and the 8 M2M tables.
// Largest |x| per coefficient of an [*][ncoef] (or [o][k][ncoef]) FP64 array,
// by a device reduction; the exponents are then taken on the host.
static std::vector<double> colmax(xrl_ctx* c, size_t n, const double* x, const int32_t* dk, cudaStream_t s) {
  const int ncoef = c->ncoef;
  DBuf<unsigned long long> mx;
  mx.alloc(c->alloc, ncoef);
  XRL_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long) * ncoef, s));
  if (n) {
    const unsigned nb = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 64);
    if (dk)
      k_tch_colmax<<<nb, 256, 0, s>>>(n, ncoef, dk, x, mx.p);
    else
      k_colmax_abs<<<nb, 256, 0, s>>>(n, ncoef, x, mx.p);
    count_launch(c);
  }
  std::vector<unsigned long long> h(ncoef);
  XRL_CUDA(cudaMemcpyAsync(h.data(), mx.p, sizeof(unsigned long long) * ncoef, cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaStreamSynchronize(s));
  std::vector<double> out(ncoef);
  for (int k = 0; k < ncoef; ++k) std::memcpy(&out[k], &h[k], sizeof(double));
  return out;
}

// The power-of-two equilibration exponents d_k of the FP64-accurate and the
// FP16 translations: 2^d_k is the size of the largest panel moment of index k
// (the P2M operator), i.e. the typical size of the multipole coefficient k.
static void ensure_dk(xrl_ctx* c, cudaStream_t s) {
  if (c->d.oz_dk.n != 0) return;
  const std::vector<double> mx = colmax(c, c->d.mom.n, c->d.mom.p, nullptr, s);
  std::vector<int32_t> dk(c->ncoef, 0);
  for (int k = 0; k < c->ncoef; ++k) dk[k] = mx[k] > 0.0 ? std::ilogb(mx[k]) : 0;
  c->d.oz_dk.upload(c->alloc, dk);
}

// One-time images of the FP64-accurate pass: the equilibration exponents d_k
// and the integer-slice images of the M2L and the 8 M2M tables.
static void oz_prepare(xrl_ctx* c, cudaStream_t s) {
  if (c->d.oz_bimg.n != 0) return;
  const Tree& t = c->tree;
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = tc_npad(ncoef) <= 64 ? 64 : 96;
  ensure_dk(c, s);
  const int noff = (int)(t.m2l_offsets.size() / 3);
  c->d.oz_bimg.alloc(c->alloc, (size_t)noff * OZ_S * Np * Kp);
  k_oz_pack_b<<<noff, 256, 0, s>>>(ncoef, Kp, Np, c->d.oz_dk.p, c->d.t_m2l.p, c->d.oz_bimg.p);
  c->d.oz_m2m_img.alloc(c->alloc, (size_t)8 * OZ_S * Np * Kp);
  k_oz_pack_b<<<8, 256, 0, s>>>(ncoef, Kp, Np, c->d.oz_dk.p, c->d.t_m2m.p, c->d.oz_m2m_img.p);
  count_launch(c, 2);
}

// The two-piece FP16 images of the M2L tables (64-coefficient tiles) and the
// per-coefficient output scales of the two-target M2L.
static void tch_prepare(xrl_ctx* c, int noff) {
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = 64;
  cudaStream_t s = c->stream;
  ensure_dk(c, s);
  const std::vector<double> mx = colmax(c, (size_t)noff * ncoef * ncoef, c->d.t_m2l.p, c->d.oz_dk.p, s);
  std::vector<int32_t> en(Np, 0);
  std::vector<float> osc(Np, 1.f);
  for (int n = 0; n < ncoef; ++n) {
    en[n] = mx[n] > 0.0 ? std::ilogb(mx[n]) + 1 : 0;
    osc[n] = std::ldexp(1.f, en[n] - TCH_TOP);
  }
  DBuf<int32_t> den;
  den.upload(c->alloc, en);
  c->d.tch_oscale.upload(c->alloc, osc);
  c->d.tch_bimg.alloc(c->alloc, (size_t)noff * TCH_PIECES * Np * Kp);
  k_tch_pack_b<<<noff, 256, 0, s>>>(ncoef, Kp, Np, c->d.oz_dk.p, den.p, c->d.t_m2l.p, c->d.tch_bimg.p);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaStreamSynchronize(s));   // den is released on return
}

// one level of the FP64-accurate M2M (parents at level l from their children
// at l + 1), integer slices as the M2L below: with M'[k] = 2^-d_k M[k] and
// T'[k] = 2^d_k T[k] the slices' product is T^T M exactly; two launches
void tc_m2m64(xrl_ctx* c, int l, int nc, double* Mx, cudaStream_t s) {
  const Tree& t = c->tree;
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = tc_npad(ncoef) <= 64 ? 64 : 96;
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  const int s0 = t.level_off[l + 1], ns = t.level_off[l + 2] - s0;
  const int nt = t.level_off[l + 1] - t.level_off[l];
  oz_prepare(c, s);
  c->d.oz_aimg.ensure(c->alloc, (size_t)ns * nct * OZ_S * TC_ROWS * Kp);
  k_oz_pack_a<<<dim3(ns, nct), 256, 0, s>>>(nc, ncoef, Kp, s0, c->d.oz_dk.p, Mx, c->d.oz_aimg.p);
  OzArgs a;
  a.pr = m2l_pairs(c, t.level_off[l], nct, OZ_S, (size_t)OZ_S * 2 * TC_ROWS * Kp, (size_t)OZ_S * 2 * Np * Kp);
  a.pr.src0 = s0;
  a.pr.ptr = c->d.box_child_ptr.p;
  a.pr.src = c->d.box_iota.p;
  a.pr.off = c->d.box_oct16.p;
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.oz_aimg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.oz_m2m_img.p);
  a.out = Mx;
  a.err = c->d.tc_err.p;
  launch_oz(c, Np, dim3(nct, nt), a, s);
}

// FP64-accurate M2L of the refinement residuals (in = M, out = L, FP64)
void tc_m2l64(xrl_ctx* c, int nbx, int b0, int nc, const double* Mx, double* Lx, cudaStream_t s) {
  const Tree& t = c->tree;
  const int ncoef = c->ncoef, Kp = tc_kpad(ncoef), Np = tc_npad(ncoef) <= 64 ? 64 : 96;
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  const int src0 = t.level_off[2];
  const int nsrc = t.n_boxes() - src0;
  oz_prepare(c, s);
  c->d.oz_aimg.ensure(c->alloc, (size_t)nsrc * nct * OZ_S * TC_ROWS * Kp);
  k_oz_pack_a<<<dim3(nsrc, nct), 256, 0, s>>>(nc, ncoef, Kp, src0, c->d.oz_dk.p, Mx, c->d.oz_aimg.p);
  OzArgs a;
  a.pr = m2l_pairs(c, b0, nct, OZ_S, (size_t)OZ_S * 2 * TC_ROWS * Kp, (size_t)OZ_S * 2 * Np * Kp);
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.oz_aimg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.oz_bimg.p);
  a.out = Lx;
  a.err = c->d.tc_err.p;
  launch_oz(c, Np, dim3(nct, nbx), a, s);
}

bool tcp_usable(const xrl_ctx* c, int nc) {
  return c->opt.tensor_cores != 0 && nc >= 64 && c->d.tcp_vimg.n > 0;
}

// FP32 near field Y = P_near X on the tensor cores (two launches)
void tc_p2p(xrl_ctx* c, int nc, const float* X, float* Y, cudaStream_t s) { tc_p2p_fork(c, nc, X, Y, s, s); }

void tc_p2p_fork(xrl_ctx* c, int nc, const float* X, float* Y, cudaStream_t s, cudaStream_t s2) {
  const int nl = c->tree.n_leaves();
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  c->d.tcp_ximg.ensure(c->alloc, (size_t)nct * c->tcp_sum_pc * TC_PIECES * TC_ROWS);
  k_tcp_pack_x<<<dim3(nl, nct), 256, 0, s>>>(nc, c->tcp_sum_pc, c->d.leaf_first.p, c->d.leaf_count.p, c->d.tcp_a0.p,
                                             c->d.tcp_pc.p, X, c->d.tcp_ximg.p);
  if (s2 != s) {
    XRL_CUDA(cudaEventRecord(c->ev_fork, s));
    XRL_CUDA(cudaStreamWaitEvent(s2, c->ev_fork, 0));
    s = s2;
  }
  if (c->tc_targets == 2 && c->d.p2p_gptr.n > 1) {
    Tc2Args g = {};
    g.mode = 1;
    g.nc = nc;
    g.nct = nct;
    g.sum_pc = c->tcp_sum_pc;
    g.a_row_bytes = TC_PIECES * TC_ROWS * 2;
    g.gptr = c->d.p2p_gptr.p;
    g.gsrc = c->d.p2p_gsrc.p;
    g.gv1 = c->d.p2p_gv1.p;
    g.gv2 = c->d.p2p_gv2.p;
    g.gt1 = c->d.p2p_gt1.p;
    g.gt2 = c->d.p2p_gt2.p;
    g.leaf_a0 = c->d.tcp_a0.p;
    g.leaf_pc = c->d.tcp_pc.p;
    g.leaf_f0 = c->d.leaf_first.p;
    g.leaf_n = c->d.leaf_count.p;
    g.pair_boff = c->d.tcp_boff.p;
    g.aimg = reinterpret_cast<const char*>(c->d.tcp_ximg.p);
    g.bimg = reinterpret_cast<const char*>(c->d.tcp_vimg.p);
    g.out = Y;
    g.err = c->d.tc_err.p;
    launch_tc2(c, dim3(nct, (unsigned)(c->d.p2p_gptr.n - 1)), g, s);
    return;
  }
  TcArgs a;
  a.pr = p2p_pairs(c, nct, TC_PIECES, c->d.tcp_boff.p);
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.tcp_ximg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.tcp_vimg.p);
  a.out = Y;
  a.err = c->d.tc_err.p;
  launch_tc<96>(c, dim3(nct, nl), a, s);
}

// FP64-accurate near field on the tensor cores (integer slices; two launches,
// plus the one-time packing of the near blocks)
void tc_p2p64(xrl_ctx* c, int nc, const double* X, double* Y, cudaStream_t s) {
  const int nl = c->tree.n_leaves();
  const int nct = (nc + TC_ROWS - 1) / TC_ROWS;
  if (c->d.ozp_vimg.n == 0) {
    c->d.ozp_vimg.alloc(c->alloc, (size_t)(c->ozp_img_bytes / 2));
    k_ozp_pack_v<<<(unsigned)c->d.u_src.n, 128, 0, s>>>(c->d.tcp_tgt.p, c->d.u_src.p, c->d.tcp_col.p,
                                                         c->d.leaf_count.p, c->d.tcp_pc.p, c->d.near_off.p,
                                                         c->d.near_w.p, c->d.ozp_boff.p, c->d.near_val.p,
                                                         c->d.ozp_vimg.p);
    count_launch(c);
  }
  c->d.ozp_ximg.ensure(c->alloc, (size_t)nct * c->tcp_sum_pc * OZ_S * TC_ROWS);
  k_ozp_pack_x<<<dim3(nl, nct), 256, 0, s>>>(nc, c->tcp_sum_pc, c->d.leaf_first.p, c->d.leaf_count.p, c->d.tcp_a0.p,
                                             c->d.tcp_pc.p, X, c->d.ozp_ximg.p);
  OzArgs a;
  a.pr = p2p_pairs(c, nct, OZ_S, c->d.ozp_boff.p);
  a.nc = nc;
  a.aimg = reinterpret_cast<const char*>(c->d.ozp_ximg.p);
  a.bimg = reinterpret_cast<const char*>(c->d.ozp_vimg.p);
  a.out = Y;
  a.err = c->d.tc_err.p;
  launch_oz(c, 96, dim3(nct, nl), a, s);
}

// raises XRL_ETIMEOUT if a tensor-core kernel gave up a wait since the last check
void tc_check(xrl_ctx* c, cudaStream_t s) {
  if (c->d.tc_err.n == 0) return;
  int32_t h = 0;
  XRL_CUDA(cudaMemcpyAsync(&h, c->d.tc_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaStreamSynchronize(s));
  if (h) {
    XRL_CUDA(cudaMemsetAsync(c->d.tc_err.p, 0, sizeof(int32_t), s));
    throw Error(XRL_ETIMEOUT, "a tensor-core translation kernel timed out waiting on its pipeline");
  }
}

}  // namespace xrl
