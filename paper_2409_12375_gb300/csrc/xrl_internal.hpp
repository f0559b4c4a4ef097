// Internal state of an xrl context and helpers shared by the library's
// translation units.  Not part of the public ABI (see include/xrl.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <map>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/xrl.h"

namespace xrl {

// ---- errors ---------------------------------------------------------------
struct Error : std::runtime_error {
  xrl_status code;
  Error(xrl_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define XRL_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::xrl::Error(e_ == cudaErrorMemoryAllocation ? XRL_ENOMEM : XRL_ECUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

#define XRL_CHECK(cond, code, msg)                 \
  do {                                             \
    if (!(cond)) throw ::xrl::Error((code), (msg)); \
  } while (0)

// ---- device memory with a high-water mark -----------------------------------
// Freed blocks are kept, by size, and handed out again for a request of the
// same size: a sweep allocates the same work arrays every time, and a
// cudaMalloc per array per chunk left the GPU idle.  A block may still be in
// use by kernels in flight when it is freed, so the first reuse after a free
// synchronises the device, as cudaFree itself would have.  The cache is
// released when an allocation fails, at every setup and when the context is
// destroyed.  `peak` counts cached blocks too (they hold device memory).
// A launch error still pending when an allocation is made is raised here, so
// that the retry below cannot clear it.
struct DevAlloc {
  int64_t cur = 0, peak = 0, cached = 0;
  bool dirty = false;   // a block was freed since the last synchronisation
  std::multimap<size_t, void*> cache;
  void* get(size_t bytes) {
    if (bytes == 0) return nullptr;
    const cudaError_t pend = cudaGetLastError();
    if (pend != cudaSuccess) throw Error(XRL_ECUDA, std::string("pending CUDA error: ") + cudaGetErrorString(pend));
    auto it = cache.find(bytes);
    if (it != cache.end()) {
      if (dirty) {
        XRL_CUDA(cudaDeviceSynchronize());
        dirty = false;
      }
      void* p = it->second;
      cache.erase(it);
      cached -= (int64_t)bytes;
      cur += (int64_t)bytes;
      return p;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaErrorMemoryAllocation && !cache.empty()) {
      cudaGetLastError();
      trim();
      e = cudaMalloc(&p, bytes);
    }
    if (e != cudaSuccess)
      throw Error(e == cudaErrorMemoryAllocation ? XRL_ENOMEM : XRL_ECUDA,
                  std::string("cudaMalloc of ") + std::to_string(bytes >> 20) + " MiB with " +
                      std::to_string(cur >> 20) + " MiB held: " + cudaGetErrorString(e));
    cur += (int64_t)bytes;
    if (cur + cached > peak) peak = cur + cached;
    return p;
  }
  void put(void* p, size_t bytes) {
    if (!p) return;
    cur -= (int64_t)bytes;
    cache.emplace(bytes, p);
    cached += (int64_t)bytes;
    dirty = true;
  }
  void trim() {
    for (auto& kv : cache) cudaFree(kv.second);
    cache.clear();
    cached = 0;
    dirty = false;
  }
  ~DevAlloc() { trim(); }
};

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DevAlloc* a = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), a(o.a) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n; a = o.a;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (a && p) a->put(p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
  void alloc(DevAlloc& al, size_t count) {
    release();
    a = &al;
    n = count;
    p = static_cast<T*>(al.get(count * sizeof(T)));
  }
  void upload(DevAlloc& al, const std::vector<T>& h) {
    alloc(al, h.size());
    if (!h.empty()) {
      // A pageable copy may return before its DMA lands, and the library's
      // streams do not wait on the legacy stream: wait for it here.
      XRL_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
      XRL_CUDA(cudaStreamSynchronize(cudaStreamLegacy));
    }
  }
  void ensure(DevAlloc& al, size_t count) {
    if (n < count) alloc(al, count);
  }
  std::vector<T> download() const {
    std::vector<T> h(n);
    if (n) {
      // the writer may be a kernel on a non-blocking stream
      XRL_CUDA(cudaDeviceSynchronize());
      XRL_CUDA(cudaMemcpy(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost));
    }
    return h;
  }
};

// ---- quadrature rule table (shared specification with the CPU checker) -------
// Class boundaries in q = |c_k - c_l| / (r_k + r_l) and rule orders.
constexpr double kQNear = 1.5, kQSemi = 3.0, kQFar = 10.0;
constexpr int kEdgeN = 10, kEdgeK = 3, kVertN = 10, kVertK = 3;
constexpr int kNearQ = 8, kSemiQ = 5, kMidQ = 4, kFarQ = 3;

// Panels are triangles or rectangles (parallelograms): at most four edges, and a
// rectangle (v0, v1, v2, v3) is integrated as its triangles (v0, v1, v2), (v0, v2, v3).
constexpr int kPanEdges = 4;

// Host geometry of caller panel p (vertex ids pan[4p..4p+3], -1 in slot 3 for a triangle):
// vertex count, vertex-mean centroid (the centroid of a triangle or a parallelogram) and area.
inline int panel_nv(const std::vector<int32_t>& pan, int p) { return pan[4 * (size_t)p + 3] >= 0 ? 4 : 3; }
void panel_centroid_host(const std::vector<double>& xyz, const std::vector<int32_t>& pan, int p, double c[3]);
double panel_area_host(const std::vector<double>& xyz, const std::vector<int32_t>& pan, int p);

// ---- host-side setup products -------------------------------------------------
struct Tree {
  int L = 0;                                   // leaf level; levels 0..L
  double lo[3] = {0, 0, 0}, side = 0;          // root cube
  std::vector<uint64_t> key;                   // per caller panel (level-21 Morton key)
  std::vector<int32_t> perm;                   // Morton rank -> caller panel
  std::vector<int32_t> rank;                   // caller panel -> Morton rank
  std::vector<int32_t> level_off;              // first global box id of each level (size L+2)
  std::vector<uint64_t> box_key;               // global box id -> key at its level
  std::vector<int32_t> parent;                 // global box id -> parent global id (-1 root)
  std::vector<int32_t> octant;                 // child position in parent (0..7)
  std::vector<int32_t> leaf_first, leaf_count; // leaf-local index -> Morton panel range
  std::vector<int32_t> leaf_of;                // Morton rank -> leaf-local index
  // V-list per target box (global ids), all levels >= 2 concatenated in box order
  std::vector<int64_t> v_ptr;                  // size n_boxes+1
  std::vector<int32_t> v_src;                  // global source box
  std::vector<int16_t> v_off;                  // index into m2l_offsets
  std::vector<int32_t> m2l_offsets;            // distinct (target - source) offsets, 3 ints each
  // U-list per leaf (leaf-local ids)
  std::vector<int64_t> u_ptr;
  std::vector<int32_t> u_src;
  int n_boxes() const { return (int)box_key.size(); }
  int n_leaves() const { return (int)leaf_first.size(); }
};

struct Topo {
  int n_live = 0, n_term = 0, n_nodes = 0, n_cb = 0, n_branch = 0, n_port = 0;
  int n_loops = 0, n_vertex_loops = 0, n_global_loops = 0;
  std::vector<int32_t> live_of_panel;           // caller panel -> live index or -1
  std::vector<int32_t> br_tail, br_head;        // node ids (live index or n_live + terminal)
  std::vector<int32_t> br_pan[2];               // caller panel of tail / head side (-1 if terminal)
  std::vector<double> br_rho[2];                // signed rho (3 per branch): +rho tail, -rho head
  std::vector<int64_t> m_ptr;                   // loop CSR
  std::vector<int32_t> m_col;
  std::vector<int8_t> m_val;
  std::vector<int64_t> mt_ptr;                  // branch CSR (transpose)
  std::vector<int32_t> mt_col;
  std::vector<int8_t> mt_val;
  // Q pencil: Q(f) = sum_m Z_s^m(f) QA_m + j omega mu0/4pi QP (CSR over loops)
  int n_mat = 0;
  std::vector<int32_t> mat_of_cond;             // conductor -> material
  std::vector<double> mat_sigma, mat_thick;
  std::vector<int64_t> q_ptr;
  std::vector<int32_t> q_col;
  std::vector<double> q_val;                    // [nnz][n_mat + 1], last = P part
  // banded direct form of Q (exact preconditioner): vertex loops in reverse
  // Cuthill-McKee order form a band of half-width `band`; the global loops
  // (homology and ports, numbered last) form a dense border.
  int n_band = 0, band = 0, n_border = 0;
  std::vector<int32_t> band_perm;               // band position -> loop index
  std::vector<double> band_val;                 // [(n_mat+1)][n_band][band+1], column j = i - band + k
  std::vector<double> border_vg;                // [(n_mat+1)][n_band][n_border]
  std::vector<double> border_gg;                // [(n_mat+1)][n_border][n_border]
};

// ---- device-resident state ------------------------------------------------------
struct Dev {
  // Morton-ordered panel data
  DBuf<double> vtx;        // [N][12] vertices (caller vertex order; a triangle's 4th is unused)
  DBuf<double> cen;        // [N][3]
  DBuf<double> area;       // [N]
  DBuf<double> radius;     // [N]
  DBuf<int32_t> tri;       // [N][4] vertex ids (-1 in the 4th slot: triangle)
  DBuf<int32_t> cidx;      // [N] caller index
  DBuf<int32_t> perm;      // [N] Morton rank -> caller
  DBuf<uint64_t> keys;     // [N] per caller panel
  DBuf<int32_t> leaf_first, leaf_count, leaf_box;   // per leaf
  DBuf<int32_t> u_ptr32, u_src;                      // U-list (leaf-local)
  DBuf<int64_t> near_off;                            // per leaf: offset of its value block
  DBuf<int32_t> near_w;                              // per leaf: block width
  DBuf<double> near_val;                             // values
  DBuf<float> near_val32;                            // FP32 copy (mixed precision)
  DBuf<float2> near_hl;                              // double-float (hi, lo) split, made on first use
  DBuf<float2> x_hl;                                 // double-float split of an FP64 product's input
  DBuf<int64_t> near_col_off;                         // per leaf: offset into near_src
  DBuf<int32_t> near_src;                             // per leaf: Morton index of each near column
  DBuf<double> mom;                                  // [N][ncoef] P2M moments (leaf-scaled)
  DBuf<float> mom32;
  DBuf<float> mom32w;      // FP32 moments with the L2P weights folded in (k_l2p_weights)
  DBuf<float2> mom_hl, momw_hl;   // double-float splits of the moments and of the weighted moments
  DBuf<double> t_m2m, t_l2l, t_m2l;                  // translation matrices (transposed)
  DBuf<float> t_m2m32, t_l2l32, t_m2l32;
  DBuf<int32_t> box_parent, box_oct, box_child_ptr, box_child;  // tree arrays (global ids)
  DBuf<int32_t> box_iota;   // 0..n_boxes (list pointers / sources of the list-form M2M, L2L)
  DBuf<int16_t> box_oct16;  // octant as a translation index
  DBuf<uint16_t> tc_bimg;   // packed 3-piece BF16 images of the M2L tables (tensor-core path)
  DBuf<uint16_t> tc_aimg;   // packed 3-piece BF16 images of the FP32 multipoles, per product
  DBuf<uint16_t> tch_bimg;  // two-piece FP16 images of the M2L tables (two-target M2L)
  DBuf<uint16_t> tch_aimg;  // two-piece FP16 images of the FP32 multipoles, per product
  DBuf<float> tch_ascale;   // their row scales 2^(e_A - 14), per (box, tile, row)
  DBuf<float> tch_oscale;   // output scales 2^(e_n - 14) per coefficient
  // M2L and near field by sibling pairs (k_xlate_tc2): per group its two
  // targets and the merged list (source, entry of t1 or -1, entry of t2 or -1)
  DBuf<int32_t> m2l_gptr, m2l_gsrc, m2l_gt1, m2l_gt2, m2l_gv1, m2l_gv2;
  DBuf<int32_t> p2p_gptr, p2p_gsrc, p2p_gt1, p2p_gt2, p2p_gv1, p2p_gv2;
  DBuf<int32_t> tc_err;     // set by a tensor-core kernel that timed out
  DBuf<uint16_t> oz_bimg;   // integer-slice BF16 images of the M2L tables (FP64-accurate path)
  DBuf<uint16_t> oz_aimg;   // integer-slice BF16 images of the FP64 multipoles, per product
  DBuf<uint16_t> oz_m2m_img;   // integer-slice BF16 images of the 8 M2M tables
  DBuf<int32_t> oz_dk;      // power-of-two equilibration exponents per coefficient index
  // near field on the tensor cores: leaves padded to 16 panels
  DBuf<int32_t> tcp_a0, tcp_pc;         // per leaf: padded panel offset and count
  DBuf<int32_t> tcp_tgt, tcp_col;       // per U-list pair: target leaf, first near column of the source
  DBuf<int64_t> tcp_boff, ozp_boff;     // per U-list pair: byte offset of its near-block image
  DBuf<uint16_t> tcp_vimg, ozp_vimg;    // near-block images (3 BF16 pieces; 5 integer slices)
  DBuf<uint16_t> tcp_ximg, ozp_ximg;    // transposed-X images, per product
  DBuf<uint16_t> tc_m2m_img;   // BF16-piece images of the 8 M2M tables
  DBuf<int64_t> tcm_boff2;      // per leaf: byte offset of its P2M moment image
  DBuf<uint16_t> tcm_p2m_img;   // leaf moment images (coefficients x panels)
  DBuf<int32_t> v_ptr32, v_src;
  DBuf<int32_t> op_ptr, op_tgt, op_src;               // V-list pairs grouped by M2L offset
  DBuf<int16_t> v_off;
  DBuf<int32_t> lvl_boxes;                            // per level: global ids of its boxes (same as range)
  // FMM work buffers (resized to the column count)
  DBuf<double> X, Y, Mexp, Lexp;
  DBuf<float> X32, Y32, M32, L32;
  // operator data
  DBuf<int32_t> pan_br;      // [N][kPanEdges] branch ids per Morton panel (-1 none)
  DBuf<double> pan_rho;      // [N][kPanEdges][3] signed rho per (panel, slot)
  DBuf<int32_t> pan_mat;     // [N] material id (-1 terminal)
  DBuf<int32_t> pan_cond_mat;  // [N] material id of every panel (features)
  DBuf<int32_t> br_pan;      // [B][2] Morton panel (-1 terminal)
  DBuf<double> br_rho;       // [B][2][3]
  DBuf<int32_t> m_ptr, m_col, mt_ptr, mt_col;
  DBuf<int32_t> m_long;     // loop rows longer than the warp-per-row reduce takes
  DBuf<double2> m_long_part; // their segment partial sums
  DBuf<int8_t> m_val, mt_val;
  DBuf<int32_t> q_ptr, q_col;
  DBuf<double> q_val;
  DBuf<double> mat_sigma, mat_thick;
  DBuf<int32_t> band_perm;
  DBuf<double> band_val, border_vg, border_gg;
  // solver work
  DBuf<double> work;         // generic scratch for the solver
  DBuf<double2> last_x;      // loop currents of the last solve [nsys][n_loops]
};

// Multigrid hierarchy of the preconditioner pencil (amg.cu): per level the
// pencil [nnz][n_mat + 1] over its unknowns and the transfer to the next level.
struct AmgLevel {
  int n = 0, nc = 0;
  int64_t nnz = 0;
  bool coarsest = false;
  DBuf<int32_t> ptr, col;
  DBuf<double> pen;
  DBuf<int64_t> dpos;                      // position of each row's diagonal (-1 none)
  DBuf<int32_t> p_ptr, p_col, r_ptr, r_col;
  DBuf<float> p_val, r_val;
};
// a CSR pencil block of Q (A_vg, A_gv, A_gg of the Schur elimination)
struct AmgBlock {
  int n = 0;
  int64_t nnz = 0;
  DBuf<int32_t> ptr, col;
  DBuf<double> pen;
};
struct AmgHier {
  std::vector<AmgLevel> lv;   // hierarchy of A_vv (or of all of Q when ng = 0)
  int W = 0;
  int nv = 0, ng = 0;         // vertex loops (multigrid) and global loops (Schur complement)
  AmgBlock vg, gv, gg;
  bool ready = false;
};
struct AmgLevelWork {
  DBuf<float2> vals, dinv, x, b, r, aug;
};
struct AmgWork {
  int nf = 0, cap = 0;        // frequencies; systems the level buffers hold
  std::vector<AmgLevelWork> lv;
  DBuf<float2> bsave, xacc;   // right-hand side and summed correction of repeated V-cycles
  // Schur elimination of the global loops: block values per frequency, the
  // inverted complement [nf][ng][2 ng], and apply buffers
  DBuf<float2> vg_vals, gv_vals, gg_vals, saug, u, tg, zg;
  DBuf<int32_t> err;
};

// Phase profiler: CUDA event pairs on the launching stream plus algorithmic work.
enum Phase { PH_P2P = 0, PH_P2M, PH_M2M, PH_M2L, PH_L2L, PH_L2P, PH_OPER, PH_PREC, PH_KRYLOV, PH_P2P64, PH_M2L64,
             PH_COUNT };
struct Prof {
  bool on = false;
  struct Rec {
    cudaEvent_t a, b;
    int phase;
  };
  std::vector<Rec> pending;
  double ms[PH_COUNT] = {0}, flops[PH_COUNT] = {0}, bytes[PH_COUNT] = {0};
  int64_t launches[PH_COUNT] = {0};
  int64_t total_launches = 0;
  // while a CUDA graph is being captured: its event pairs and work, read back after every replay
  bool capturing = false;
  struct GRec {
    cudaEvent_t a, b;
    int phase, launches;
    double flops, bytes;
  };
  std::vector<GRec> graph_recs;
  int64_t graph_launches = 0;
};

}  // namespace xrl

struct xrl_ctx {
  xrl_options opt;
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t stream2 = nullptr;              // the FP32 near field runs here beside the far field
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  xrl::DevAlloc alloc;
  // inputs
  std::vector<double> xyz;
  std::vector<int32_t> pan, cond;   // pan [N][4] vertex ids, -1 in the 4th slot for a triangle
  std::vector<double> sigma, thick;
  std::vector<std::vector<int32_t>> port_src, port_sink;
  bool have_mesh = false, have_cond = false, ready = false;
  int N = 0, ncoef = 0, p = 0, max_leaf = 0;
  int max_off_pairs = 0;                // most V-list pairs of one M2L offset
  bool df64_m2l = false;   // FP64 M2L on the FP32 pipes (set inside mixed-precision solves)
  int tcp_sum_pc = 0;                   // padded panels of all leaves (tensor-core near field)
  int tc_targets = 2;                   // targets per CTA of the FP32 tensor-core M2L / near field (autotuned)
  int64_t tcp_img_bytes = 0, ozp_img_bytes = 0;
  int last_nsys = 0, last_nport = 0;
  std::vector<int32_t> last_port_loop;
  xrl::Tree tree;
  xrl::Topo topo;
  xrl::Dev d;
  xrl::AmgHier amg;
  xrl_stats stats;
  xrl::Prof prof;
  std::vector<double> gl_nodes;   // host GL tables for the rule table (set in setup)
};

// ---- translation-unit entry points (internal) --------------------------------------
namespace xrl {
// profiling helpers (api.cu): begin returns an event recorded on s (or null)
cudaEvent_t prof_begin(xrl_ctx* c, cudaStream_t s);
void prof_end(xrl_ctx* c, cudaStream_t s, cudaEvent_t a, int phase, int launches, double flops, double bytes);
void prof_graph_replayed(xrl_ctx* c);   // after a replay of the captured graph has completed
void prof_graph_release(xrl_ctx* c);
inline void count_launch(xrl_ctx* c, int n = 1) {
  if (c->prof.capturing)
    c->prof.graph_launches += n;
  else
    c->prof.total_launches += n;
}
// tree.cpp
void build_tree(xrl_ctx* c, const std::vector<uint64_t>& keys_by_caller);
uint64_t morton_key(uint32_t ix, uint32_t iy, uint32_t iz);
void morton_decode(uint64_t key, uint32_t* ix, uint32_t* iy, uint32_t* iz);
// topology.cpp
void build_topology(xrl_ctx* c);
// p12 = NULL: diagonal-of-P pencil (eq. 10); else the diagonal-of-L pencil with p12[b] the
// P entry between the tail and head panels of conductor branch b (0 where one side is a terminal)
void build_precond_pattern(xrl_ctx* c, const std::vector<double>& p_diag_caller,
                           const std::vector<double>* p12 = nullptr);
void build_band(xrl_ctx* c);
// harmonics.cpp
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
void build_translations(int p, const std::vector<int32_t>& offsets, std::vector<double>& m2m,
                        std::vector<double>& l2l, std::vector<double>& m2l);
// geom.cu
void launch_geometry(xrl_ctx* c);              // computes panel data + keys (caller order) on device
void launch_near_fill(xrl_ctx* c);             // near-field blocks (rule table)
void launch_moments(xrl_ctx* c);               // P2M/L2P moment table
void launch_direct(xrl_ctx* c, int ncols, const double* x, double* y, cudaStream_t s);
// rows [nrows] Morton ranks; Y [nrows][nc]
void launch_direct_rows(xrl_ctx* c, int nrows, const int32_t* rows, int nc, const double* X, double* Y,
                        cudaStream_t s);
std::vector<double> pair_entries(xrl_ctx* c, const std::vector<int32_t>& k_caller,
                                 const std::vector<int32_t>& l_caller);   // P entries of panel pairs
void upload_rule_tables(xrl_ctx* c);
// fmm.cu
void fmm_prepare(xrl_ctx* c);                  // upload tree and operators
void fmm_apply(xrl_ctx* c, int ncols, const double* X, double* Y, cudaStream_t s);      // Morton [N][nc]
void fmm_apply32(xrl_ctx* c, int ncols, const float* X, float* Y, cudaStream_t s);
void fmm_apply_into(xrl_ctx* c, int ncols, const double* X, double* Y, double* Mx, double* Lx, cudaStream_t s);
void launch_to_morton(const xrl_ctx* c, int ncols, const double* x_user, double* X, cudaStream_t s);
void launch_from_morton(const xrl_ctx* c, int ncols, const double* Y, double* y_user, cudaStream_t s);
void launch_to_morton32(const xrl_ctx* c, int ncols, const float* x_user, float* X, cudaStream_t s);
void launch_from_morton32(const xrl_ctx* c, int ncols, const float* Y, float* y_user, cudaStream_t s);
// tc.cu: tensor-core (tcgen05) M2L of the FP32 products
bool tc_usable(const xrl_ctx* c, int ncols);
void tc_prepare(xrl_ctx* c);
void tc_m2l(xrl_ctx* c, int nbx, int b0, int ncols, const float* M, float* L, cudaStream_t s);
void tc_check(xrl_ctx* c, cudaStream_t s);
bool tc64_usable(const xrl_ctx* c, int ncols);
bool tcp_usable(const xrl_ctx* c, int ncols);
void tc_p2p(xrl_ctx* c, int ncols, const float* X, float* Y, cudaStream_t s);
// pack X on s, then the near field on s2 after a fork event (joined by the caller)
void tc_p2p_fork(xrl_ctx* c, int ncols, const float* X, float* Y, cudaStream_t s, cudaStream_t s2);
void tc_p2p64(xrl_ctx* c, int ncols, const double* X, double* Y, cudaStream_t s);
bool tcm_usable(const xrl_ctx* c, int ncols);
void tc_p2m(xrl_ctx* c, int ncols, float* M, cudaStream_t s);
void tc_m2m(xrl_ctx* c, int level, int ncols, float* M, cudaStream_t s);
void tc_m2m64(xrl_ctx* c, int level, int ncols, double* M, cudaStream_t s);   // FP64-accurate, integer slices
void tc_m2l64(xrl_ctx* c, int nbx, int b0, int ncols, const double* M, double* L, cudaStream_t s);
// solve.cu
void solver_prepare(xrl_ctx* c);
void run_solve(xrl_ctx* c, int nf, const double* f, double* R, double* L, const float* shape = nullptr,
               int* accepted = nullptr, double* guess_res = nullptr, bool from_prev = false);
void panel_currents(xrl_ctx* c, bool normalize, double* host_out);
void panel_features(xrl_ctx* c, int nf, const double* freq, double f0, const double* d_ip0, float* d_feat,
                    double* h_scale, cudaStream_t s);
void apply_operator_host(xrl_ctx* c, int nsys, const double* f, const double* v, double* w, int mode);
// precond.cu
bool band_usable(const xrl_ctx* c);
bool band_fits(int band, int n_border);   // within the banded solver's limits
void band_prepare(xrl_ctx* c);
// Factor and work arrays of the banded preconditioner for nf frequencies,
// partitioned into P blocks of m rows (see precond.cu).
struct BandWork {
  int nf = 0, P = 1, m = 0;
  bool mixed = false;
  DBuf<double2> fac, facT, Wb, Sinv, Vsp, Wsp, R, scr, hb, part;
  DBuf<float2> fac32, facT32, Vsp32, Wsp32, R32, scr32, hb32, Wb32;
};
void band_alloc(xrl_ctx* c, BandWork& bw, int nf, int nsys, bool mixed);
void band_factor(xrl_ctx* c, BandWork& bw, const double2* zs, const double* wp, cudaStream_t s);
void band_apply(xrl_ctx* c, BandWork& bw, int nsys, int nport, const double2* zs, const double* wp,
                const double2* v, double2* z, const int* active, cudaStream_t s);
// amg.cu: multigrid V-cycle for Q^-1 where the band form is not usable
void amg_prepare(xrl_ctx* c);
void amg_factor(xrl_ctx* c, AmgWork& w, int nf, int nsys, const double2* zsf, const double* wpf, cudaStream_t s);
void amg_apply(xrl_ctx* c, AmgWork& w, int nsys, int nport, const double2* v, double2* z, cudaStream_t s);
void amg_check(xrl_ctx* c, AmgWork& w, cudaStream_t s);
}  // namespace xrl
