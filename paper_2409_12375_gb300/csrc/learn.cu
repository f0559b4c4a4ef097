// Learned initial guess for the sweep: panel features, panel-current export
// and a small per-panel MLP trained and run by this library's own kernels.
//
// The paper solves every frequency from scratch (Sec. III).  Here a sweep can
// start from a prediction: the MLP maps per-panel features (geometry, log f,
// the lowest frequency's current distribution) to the panel current
// distribution at frequency f, per unit port current; xrl_solve_guess projects
// it onto loop space and keeps it only where it lowers the FP64 residual.
//
// Network: n_in -> width (GELU) x n_hidden -> n_out.  Master weights FP32,
// forward/backward use BF16-rounded copies (round to nearest even), every
// product accumulates in FP32; loss = mean squared error; optimiser AdamW.
#include <cuda_bf16.h>

#include <cmath>
#include <random>
#include <vector>

#include "cplx.cuh"
#include "xrl_internal.hpp"

struct xrl_mlp {
  int device = 0;
  int n_in = 0, width = 0, n_hidden = 0, n_out = 0;
  int64_t n_params = 0, step = 0;
  std::vector<int> dims;                 // layer sizes n_in, width, ..., n_out
  std::vector<int64_t> woff, boff;       // offsets of W_l [in][out] and b_l [out] in the parameter vector
  xrl::DevAlloc alloc;
  xrl::DBuf<float> P, G, Mo, Vo;         // params, grads, Adam moments
  xrl::DBuf<__nv_bfloat16> Pb;           // BF16 copy of the weights (biases kept FP32)
  std::vector<xrl::DBuf<float>> act;     // per layer output activations (post-GELU), and pre-activations
  std::vector<xrl::DBuf<float>> pre;
  xrl::DBuf<float> dA, dB;               // gradient buffers [rows][width]
  xrl::DBuf<double> lossbuf;
  xrl::DBuf<uint8_t> wmask;              // 1 for weights (decayed), 0 for biases
  int64_t cap_rows = 0;
  std::string err;
};

namespace xrl {

// ---- panel current export and features ---------------------------------------------------------
// Ip[s][p][6] (caller panel order) from loop currents x[s][:]; optionally divided by the
// complex port current of the system (per unit port current)
__global__ void k_panel_currents(int N, int nsys, int nloop, int nport, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ pan_br, const double* __restrict__ pan_rho,
                                 const int32_t* __restrict__ mt_ptr, const int32_t* __restrict__ mt_col,
                                 const int8_t* __restrict__ mt_val, const int32_t* __restrict__ port_loop,
                                 const cplx* __restrict__ x, int normalize, double* __restrict__ out) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * nsys) return;
  int r = (int)(idx % N), s = (int)(idx / N);
  const cplx* xs = x + (size_t)s * nloop;
  cplx ip[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int k = 0; k < kPanEdges; ++k) {
    int b = pan_br[kPanEdges * r + k];
    if (b < 0) continue;
    cplx ie = make_double2(0, 0);
    for (int q = mt_ptr[b]; q < mt_ptr[b + 1]; ++q) ie = mt_val[q] > 0 ? cadd(ie, xs[mt_col[q]]) : csub(ie, xs[mt_col[q]]);
    for (int t = 0; t < 3; ++t) ip[t] = cadd(ip[t], cscale(ie, pan_rho[3 * kPanEdges * (size_t)r + 3 * k + t]));
  }
  cplx sc = make_double2(1.0, 0.0);
  if (normalize) {
    cplx ipt = xs[port_loop[s % nport]];
    sc = cabs2(ipt) > 0 ? cdiv(make_double2(1.0, 0.0), ipt) : make_double2(0, 0);
  }
  double* o = out + ((size_t)s * N + perm[r]) * 6;
  for (int t = 0; t < 3; ++t) {
    cplx v = cm(ip[t], sc);
    o[2 * t] = v.x;
    o[2 * t + 1] = v.y;
  }
}

// feat[(f*np + q)][p][24] for caller panel p (see xrl_panel_features in xrl.h)
__global__ void k_features(int N, int nf, int np, const int32_t* __restrict__ perm, const double* __restrict__ cen,
                           const double* __restrict__ vtx, const double* __restrict__ area, double area_mean,
                           const int32_t* __restrict__ pan_br, const int32_t* __restrict__ br_pan,
                           const int32_t* __restrict__ pan_mat, const int32_t* __restrict__ pan_cond_mat,
                           const double* __restrict__ mat_sigma, const double* __restrict__ mat_thick,
                           const double* __restrict__ freq, double f0, double lo0, double lo1, double lo2,
                           double side, const double* __restrict__ ip0, const double* __restrict__ scale,
                           float* __restrict__ feat) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * nf * np) return;
  int r = (int)(idx % N);
  int s = (int)(idx / N);
  int f = s / np, q = s % np;
  int p = perm[r];
  const double* v = vtx + 12 * (size_t)r;   // the normal from the first three vertices (panels are planar)
  double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
  double nr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double nn = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
  for (int k = 0; k < 3; ++k) nr[k] /= nn;
  // curvature proxy: mean (1 - |n . n_j|) over the panels sharing a branch with this one
  double curv = 0.0;
  int ncur = 0;
  for (int k = 0; k < kPanEdges; ++k) {
    int b = pan_br[kPanEdges * r + k];
    if (b < 0) continue;
    int o = br_pan[2 * b] == r ? br_pan[2 * b + 1] : br_pan[2 * b];
    if (o < 0) continue;
    const double* w = vtx + 12 * (size_t)o;
    double a1[3] = {w[3] - w[0], w[4] - w[1], w[5] - w[2]}, a2[3] = {w[6] - w[0], w[7] - w[1], w[8] - w[2]};
    double m[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
    double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    curv += 1.0 - fabs((m[0] * nr[0] + m[1] * nr[1] + m[2] * nr[2]) / mm);
    ++ncur;
  }
  if (ncur) curv /= ncur;
  const double fr = freq[f];
  const double lf = log10(fr);
  const int mat = pan_cond_mat[r];
  const double sig = mat_sigma[mat], thk = mat_thick[mat];
  const double delta = 1.0 / sqrt(3.14159265358979323846 * fr * 4e-7 * 3.14159265358979323846 * sig);
  const double* ip = ip0 + ((size_t)q * N + p) * 6;
  const double sq = scale[q];
  double mag = 0.0;
  for (int k = 0; k < 6; ++k) mag += ip[k] * ip[k] * sq * sq;
  float* o = feat + ((size_t)s * N + p) * 24;
  o[0] = (float)((cen[3 * (size_t)r] - lo0) / side);
  o[1] = (float)((cen[3 * (size_t)r + 1] - lo1) / side);
  o[2] = (float)((cen[3 * (size_t)r + 2] - lo2) / side);
  o[3] = (float)nr[0];
  o[4] = (float)nr[1];
  o[5] = (float)nr[2];
  o[6] = (float)(log(area[r] / area_mean) / 4.0);
  o[7] = (float)(curv * 4.0);
  o[8] = (float)((lf - 5.0) / 5.0);
  o[9] = (float)(log10(fr / f0) / 10.0);
  for (int k = 0; k < 6; ++k) o[10 + k] = (float)(ip[k] * sq);
  o[16] = (float)(log10(delta / thk) / 3.0);
  o[17] = (float)sqrt(mag);
  o[18] = pan_mat[r] < 0 ? 1.f : 0.f;
  o[19] = (float)sin(lf);
  o[20] = (float)cos(lf);
  o[21] = 1.f;
  o[22] = (float)q / (float)np;
  o[23] = 0.f;
}

// scale[q] = 1 / max_p |ip0[q][p]| (one block per port)
__global__ void k_ref_scale(int N, const double* __restrict__ ip0, double* __restrict__ scale) {
  __shared__ double sh[256];
  const int q = blockIdx.x;
  double m = 0.0;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const double* v = ip0 + ((size_t)q * N + p) * 6;
    double a = 0.0;
    for (int k = 0; k < 6; ++k) a += v[k] * v[k];
    m = fmax(m, a);
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) scale[q] = sh[0] > 0.0 ? 1.0 / sqrt(sh[0]) : 1.0;
}

void panel_currents(xrl_ctx* c, bool normalize, double* host_out) {
  XRL_CHECK(c->last_nsys > 0, XRL_ESTATE, "no solve has run on this context");
  const Topo& T = c->topo;
  const int N = c->N, nsys = c->last_nsys;
  DBuf<double> out;
  out.alloc(c->alloc, (size_t)nsys * N * 6);
  DBuf<int32_t> pl;
  pl.upload(c->alloc, c->last_port_loop);
  size_t tot = (size_t)N * nsys;
  k_panel_currents<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
      N, nsys, T.n_loops, c->last_nport, c->d.perm.p, c->d.pan_br.p, c->d.pan_rho.p, c->d.mt_ptr.p, c->d.mt_col.p,
      c->d.mt_val.p, pl.p, c->d.last_x.p, normalize ? 1 : 0, out.p);
  count_launch(c);
  XRL_CUDA(cudaGetLastError());
  XRL_CUDA(cudaMemcpyAsync(host_out, out.p, sizeof(double) * out.n, cudaMemcpyDeviceToHost, c->stream));
  XRL_CUDA(cudaStreamSynchronize(c->stream));
}

void panel_features(xrl_ctx* c, int nf, const double* freq, double f0, const double* d_ip0, float* d_feat,
                    double* h_scale, cudaStream_t s) {
  const Topo& T = c->topo;
  const int N = c->N, np = T.n_port;
  if (c->d.pan_cond_mat.n == 0) {
    std::vector<int32_t> pm(N);
    for (int p = 0; p < N; ++p) pm[c->tree.rank[p]] = T.mat_of_cond[c->cond[p]];
    c->d.pan_cond_mat.upload(c->alloc, pm);
  }
  double amean = 0.0;
  {
    std::vector<double> a = c->d.area.download();
    for (double v : a) amean += v;
    amean /= N;
  }
  DBuf<double> df, dscale;
  df.upload(c->alloc, std::vector<double>(freq, freq + nf));
  dscale.alloc(c->alloc, np);
  k_ref_scale<<<np, 256, 0, s>>>(N, d_ip0, dscale.p);
  count_launch(c);
  size_t tot = (size_t)N * nf * np;
  k_features<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      N, nf, np, c->d.perm.p, c->d.cen.p, c->d.vtx.p, c->d.area.p, amean, c->d.pan_br.p, c->d.br_pan.p,
      c->d.pan_mat.p, c->d.pan_cond_mat.p, c->d.mat_sigma.p, c->d.mat_thick.p, df.p, f0, c->tree.lo[0],
      c->tree.lo[1], c->tree.lo[2], c->tree.side, d_ip0, dscale.p, d_feat);
  count_launch(c);
  XRL_CUDA(cudaGetLastError());
  if (h_scale) XRL_CUDA(cudaMemcpyAsync(h_scale, dscale.p, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaStreamSynchronize(s));
}

// ---- MLP kernels ------------------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float a) {
  return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * __expf(-0.5f * a * a);
}

// Y[rows][out] = X[rows][in] W[in][out] + b ; optional GELU into H (A keeps the pre-activation)
// block: 64 rows x 64 outputs, 256 threads (each 4 rows x 4 outputs), K chunks of 32
__global__ void __launch_bounds__(256) k_lin_fwd(int64_t rows, int in, int out, const float* __restrict__ X,
                                                 const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                                                 float* __restrict__ A, float* __restrict__ H, int act) {
  __shared__ float Xs[32][64 + 1];
  __shared__ float Ws[32][64];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int o0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < in; k0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int rr = e / 32, kk = e % 32;
      int64_t row = r0 + rr;
      Xs[kk][rr] = (row < rows && k0 + kk < in) ? X[row * in + k0 + kk] : 0.f;
      int kk2 = e / 64, oo = e % 64;
      Ws[kk2][oo] = (k0 + kk2 < in && o0 + oo < out) ? __bfloat162float(W[(size_t)(k0 + kk2) * out + o0 + oo]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float xv[4], wv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) wv[j] = Ws[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], wv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t row = r0 + ty + 16 * i;
    if (row >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int o = o0 + tx + 16 * j;
      if (o >= out) continue;
      float a = acc[i][j] + bias[o];
      if (A) A[row * out + o] = a;
      if (H) H[row * out + o] = act ? gelu(a) : a;
    }
  }
}

// dX[rows][in] = dA[rows][out] W^T
__global__ void __launch_bounds__(256) k_lin_bwd_x(int64_t rows, int in, int out, const float* __restrict__ dA,
                                                   const __nv_bfloat16* __restrict__ W, float* __restrict__ dX) {
  __shared__ float Ds[32][64 + 1];
  __shared__ float Ws[32][64];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int i0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < out; k0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int rr = e / 32, kk = e % 32;
      int64_t row = r0 + rr;
      Ds[kk][rr] = (row < rows && k0 + kk < out) ? dA[row * out + k0 + kk] : 0.f;
      int kk2 = e / 64, ii = e % 64;
      // Ws[kk][ii] = W[i0 + ii][k0 + kk]
      Ws[kk2][ii] = (k0 + kk2 < out && i0 + ii < in) ? __bfloat162float(W[(size_t)(i0 + ii) * out + k0 + kk2]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float dv[4], wv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) dv[i] = Ds[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) wv[j] = Ws[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], wv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t row = r0 + ty + 16 * i;
    if (row >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int ii = i0 + tx + 16 * j;
      if (ii < in) dX[row * in + ii] = acc[i][j];
    }
  }
}

// dW[in][out] += X^T dA over a chunk of rows per block; db[out] += column sums of dA
__global__ void __launch_bounds__(256) k_lin_bwd_w(int64_t rows, int in, int out, const float* __restrict__ X,
                                                   const float* __restrict__ dA, float* __restrict__ dW,
                                                   float* __restrict__ db, int64_t rows_per_block) {
  __shared__ float Xs[32][64 + 1];
  __shared__ float Ds[32][64 + 1];
  const int i0 = blockIdx.y * 64, o0 = blockIdx.z * 64;
  const int64_t rb = (int64_t)blockIdx.x * rows_per_block;
  const int64_t re = rb + rows_per_block < rows ? rb + rows_per_block : rows;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  float bacc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t k0 = rb; k0 < re; k0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int kk = e / 64, cc = e % 64;
      int64_t row = k0 + kk;
      Xs[kk][cc] = (row < re && i0 + cc < in) ? X[row * in + i0 + cc] : 0.f;
      Ds[kk][cc] = (row < re && o0 + cc < out) ? dA[row * out + o0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float xv[4], dv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) dv[j] = Ds[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], dv[j], acc[i][j]);
      if (blockIdx.y == 0 && ty == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) bacc[j] += dv[j];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int ii = i0 + ty + 16 * i;
    if (ii >= in) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int o = o0 + tx + 16 * j;
      if (o < out) atomicAdd(&dW[(size_t)ii * out + o], acc[i][j]);
    }
  }
  if (blockIdx.y == 0 && ty == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int o = o0 + tx + 16 * j;
      if (o < out) atomicAdd(&db[o], bacc[j]);
    }
}

// dA = dH * gelu'(A) in place on dH
__global__ void k_gelu_bwd(int64_t n, const float* __restrict__ A, float* __restrict__ dH) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dH[i] *= gelu_d(A[i]);
}

// dY = 2 (Y - T) / n ; loss += sum (Y - T)^2 / n
__global__ void k_mse(int64_t n, const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      double* __restrict__ loss) {
  __shared__ double sh[256];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    float d = Y[i] - T[i];
    dY[i] = 2.f * d / (float)n;
    l = (double)d * d / (double)n;
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, sh[0]);
}

__global__ void k_adamw(int64_t n, float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                        float* __restrict__ V, float lr, float wd, float b1, float b2, float c1, float c2,
                        const uint8_t* __restrict__ is_weight) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g = G[i];
  float m = b1 * M[i] + (1.f - b1) * g;
  float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  float upd = (m / c1) / (sqrtf(v / c2) + 1e-8f);
  if (is_weight[i]) upd += wd * P[i];
  P[i] -= lr * upd;
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ P, __nv_bfloat16* __restrict__ B) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) B[i] = __float2bfloat16_rn(P[i]);
}

}  // namespace xrl

using namespace xrl;

namespace {

void ensure_rows(xrl_mlp* m, int64_t rows) {
  if (rows <= m->cap_rows) return;
  const size_t L = m->dims.size() - 1;
  m->act.resize(L);
  m->pre.resize(L);
  for (size_t l = 0; l < L; ++l) {
    m->act[l].alloc(m->alloc, (size_t)rows * m->dims[l + 1]);
    m->pre[l].alloc(m->alloc, (size_t)rows * m->dims[l + 1]);
  }
  int wmax = std::max(m->width, std::max(m->n_in, m->n_out));
  m->dA.alloc(m->alloc, (size_t)rows * wmax);
  m->dB.alloc(m->alloc, (size_t)rows * wmax);
  m->cap_rows = rows;
}

void forward(xrl_mlp* m, int64_t rows, const float* X, cudaStream_t s) {
  const size_t L = m->dims.size() - 1;
  const float* in = X;
  for (size_t l = 0; l < L; ++l) {
    int di = m->dims[l], dout = m->dims[l + 1];
    dim3 g((unsigned)((rows + 63) / 64), (dout + 63) / 64);
    k_lin_fwd<<<g, 256, 0, s>>>(rows, di, dout, in, m->Pb.p + m->woff[l], m->P.p + m->boff[l], m->pre[l].p,
                                m->act[l].p, l + 1 < L ? 1 : 0);
    in = m->act[l].p;
  }
}

// gradient of the mean squared error into m->G (zeroed first); returns loss
double backward(xrl_mlp* m, int64_t rows, const float* X, const float* T, cudaStream_t s) {
  const size_t L = m->dims.size() - 1;
  XRL_CUDA(cudaMemsetAsync(m->G.p, 0, sizeof(float) * m->n_params, s));
  XRL_CUDA(cudaMemsetAsync(m->lossbuf.p, 0, sizeof(double), s));
  const int64_t ny = rows * m->n_out;
  k_mse<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(ny, m->act[L - 1].p, T, m->dA.p, m->lossbuf.p);
  float* d = m->dA.p;
  float* dn = m->dB.p;
  for (size_t l = L; l-- > 0;) {
    int di = m->dims[l], dout = m->dims[l + 1];
    const float* xin = l == 0 ? X : m->act[l - 1].p;
    const int64_t rpb = 2048;
    dim3 gw((unsigned)((rows + rpb - 1) / rpb), (di + 63) / 64, (dout + 63) / 64);
    k_lin_bwd_w<<<gw, 256, 0, s>>>(rows, di, dout, xin, d, m->G.p + m->woff[l], m->G.p + m->boff[l], rpb);
    if (l > 0) {
      dim3 gx((unsigned)((rows + 63) / 64), (di + 63) / 64);
      k_lin_bwd_x<<<gx, 256, 0, s>>>(rows, di, dout, d, m->Pb.p + m->woff[l], dn);
      const int64_t nh = rows * di;
      k_gelu_bwd<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(nh, m->pre[l - 1].p, dn);
      std::swap(d, dn);
    }
  }
  XRL_CUDA(cudaGetLastError());
  double loss = 0.0;
  XRL_CUDA(cudaMemcpyAsync(&loss, m->lossbuf.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  XRL_CUDA(cudaStreamSynchronize(s));
  return loss;
}

template <class F>
xrl_status mguard(xrl_mlp* m, F&& f) {
  try {
    if (m) XRL_CUDA(cudaSetDevice(m->device));
    f();
    if (m) m->err.clear();
    return XRL_OK;
  } catch (const Error& e) {
    if (m) m->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    if (m) m->err = e.what();
    return XRL_EINVAL;
  }
}

}  // namespace

extern "C" {

xrl_status xrl_mlp_create(int32_t n_in, int32_t width, int32_t n_hidden, int32_t n_out, uint64_t seed,
                          int32_t device, xrl_mlp** out) {
  if (!out) return XRL_EINVAL;
  *out = nullptr;
  if (n_in < 1 || width < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || width > 4096 || n_out > 4096)
    return XRL_EINVAL;
  xrl_mlp* m = new xrl_mlp();
  m->device = device;
  m->n_in = n_in;
  m->width = width;
  m->n_hidden = n_hidden;
  m->n_out = n_out;
  xrl_status st = mguard(m, [&] {
    m->dims.push_back(n_in);
    for (int i = 0; i < n_hidden; ++i) m->dims.push_back(width);
    m->dims.push_back(n_out);
    int64_t off = 0;
    for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
      m->woff.push_back(off);
      off += (int64_t)m->dims[l] * m->dims[l + 1];
      m->boff.push_back(off);
      off += m->dims[l + 1];
    }
    m->n_params = off;
    // He-style uniform init, fixed seed (std::mt19937_64, portable)
    std::vector<float> h(off, 0.f);
    std::mt19937_64 rng(seed);
    for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
      double lim = std::sqrt(6.0 / m->dims[l]);
      for (int64_t k = 0; k < (int64_t)m->dims[l] * m->dims[l + 1]; ++k) {
        double u = (double)(rng() >> 11) * (1.0 / 9007199254740992.0);
        h[m->woff[l] + k] = (float)((2.0 * u - 1.0) * lim);
      }
    }
    m->P.upload(m->alloc, h);
    m->G.alloc(m->alloc, off);
    m->Mo.upload(m->alloc, std::vector<float>(off, 0.f));
    m->Vo.upload(m->alloc, std::vector<float>(off, 0.f));
    m->Pb.alloc(m->alloc, off);
    k_to_bf16<<<(unsigned)((off + 255) / 256), 256>>>(off, m->P.p, m->Pb.p);
    m->lossbuf.alloc(m->alloc, 1);
    std::vector<uint8_t> wm(off, 0);
    for (size_t l = 0; l + 1 < m->dims.size(); ++l)
      for (int64_t k = 0; k < (int64_t)m->dims[l] * m->dims[l + 1]; ++k) wm[m->woff[l] + k] = 1;
    m->wmask.upload(m->alloc, wm);
    XRL_CUDA(cudaDeviceSynchronize());
  });
  if (st != XRL_OK) {
    delete m;
    return st;
  }
  *out = m;
  return XRL_OK;
}

int64_t xrl_mlp_num_params(const xrl_mlp* m) { return m ? m->n_params : 0; }

xrl_status xrl_mlp_forward(xrl_mlp* m, int64_t rows, const float* d_x, float* d_y, void* stream) {
  if (!m) return XRL_EINVAL;
  return mguard(m, [&] {
    XRL_CHECK(rows > 0 && d_x && d_y, XRL_EINVAL, "bad forward arguments");
    cudaStream_t s = (cudaStream_t)stream;
    ensure_rows(m, rows);
    forward(m, rows, d_x, s);
    XRL_CUDA(cudaMemcpyAsync(d_y, m->act.back().p, sizeof(float) * rows * m->n_out, cudaMemcpyDeviceToDevice, s));
    XRL_CUDA(cudaGetLastError());
  });
}

xrl_status xrl_mlp_train_step(xrl_mlp* m, int64_t rows, const float* d_x, const float* d_t, float lr,
                              float weight_decay, double* loss, void* stream) {
  if (!m) return XRL_EINVAL;
  return mguard(m, [&] {
    XRL_CHECK(rows > 0 && d_x && d_t && lr > 0, XRL_EINVAL, "bad training arguments");
    cudaStream_t s = (cudaStream_t)stream;
    ensure_rows(m, rows);
    forward(m, rows, d_x, s);
    double l = backward(m, rows, d_x, d_t, s);
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    k_adamw<<<(unsigned)((m->n_params + 255) / 256), 256, 0, s>>>(m->n_params, m->P.p, m->G.p, m->Mo.p, m->Vo.p,
                                                                   lr, weight_decay, b1, b2, c1, c2,
                                                                   m->wmask.p);
    k_to_bf16<<<(unsigned)((m->n_params + 255) / 256), 256, 0, s>>>(m->n_params, m->P.p, m->Pb.p);
    XRL_CUDA(cudaGetLastError());
    if (loss) *loss = l;
  });
}

xrl_status xrl_mlp_gradients(xrl_mlp* m, int64_t rows, const float* d_x, const float* d_t, float* h_grads,
                             double* loss) {
  if (!m) return XRL_EINVAL;
  return mguard(m, [&] {
    XRL_CHECK(rows > 0 && d_x && d_t && h_grads, XRL_EINVAL, "bad gradient arguments");
    ensure_rows(m, rows);
    forward(m, rows, d_x, nullptr);
    double l = backward(m, rows, d_x, d_t, nullptr);
    XRL_CUDA(cudaMemcpy(h_grads, m->G.p, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
    if (loss) *loss = l;
  });
}

xrl_status xrl_mlp_get_params(const xrl_mlp* m, float* h) {
  if (!m || !h) return XRL_EINVAL;
  return mguard(const_cast<xrl_mlp*>(m), [&] {
    XRL_CUDA(cudaMemcpy(h, m->P.p, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  });
}

xrl_status xrl_mlp_set_params(xrl_mlp* m, const float* h) {
  if (!m || !h) return XRL_EINVAL;
  return mguard(m, [&] {
    XRL_CUDA(cudaMemcpy(m->P.p, h, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
    k_to_bf16<<<(unsigned)((m->n_params + 255) / 256), 256>>>(m->n_params, m->P.p, m->Pb.p);
    XRL_CUDA(cudaDeviceSynchronize());
  });
}

const char* xrl_mlp_last_error(const xrl_mlp* m) { return m ? m->err.c_str() : "null mlp"; }

void xrl_mlp_destroy(xrl_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  delete m;
}

}  // extern "C"
