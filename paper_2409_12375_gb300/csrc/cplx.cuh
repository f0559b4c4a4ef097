// Complex FP64 helpers on double2 (device), shared by the solver files.
#pragma once
#include <cuda_runtime.h>

namespace xrl {
typedef double2 cplx;
__device__ __forceinline__ cplx cm(cplx a, cplx b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
// value of a pencil member: sum_m zs[m] a[m*stride] + j wp a[nmat*stride]
__device__ __forceinline__ cplx pencil(const double* a, size_t stride, int nmat, const cplx* zs, double wp) {
  cplx r = make_double2(0.0, wp * a[(size_t)nmat * stride]);
  for (int m = 0; m < nmat; ++m) r = cadd(r, cscale(zs[m], a[(size_t)m * stride]));
  return r;
}
}  // namespace xrl
