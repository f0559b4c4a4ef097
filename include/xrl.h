/*
 * xrl.h -- C ABI of the GB300 (sm_103a) library for broadband resistance /
 * inductance extraction with an FMM-accelerated surface integral equation,
 * following Wang, Liu, Gu, Jia, Yucel, "XRL: An FMM-Accelerated SIE Simulator
 * for Resistance and Inductance Extraction of Complicated 3-D Geometries"
 * (arXiv 2409.12375).
 *
 * Problem statement (Sec. II-A, eq. 1-3; Sec. III, port definition): the
 * caller gives closed triangulated conductor surfaces, a conductivity and an
 * ESI thickness per conductor, ports (a source and a sink terminal patch of
 * panels each) and a list of frequencies; the library returns per-frequency
 * port resistance and inductance matrices.  The raw panel potential product
 * y = P x (the quantity the paper accelerates with the FMM, Sec. II-C) is
 * exported too.
 *
 * Conventions for every call:
 *  - Units are SI (metres, S/m, Hz, ohm, henry).  P has units 1/m.
 *  - Panels are addressed in the caller's order (the order of `tri`);
 *    reordering (Morton order) is internal.
 *  - Ownership: the caller owns every buffer it passes.  Host inputs are
 *    copied before the call returns; no caller pointer is retained.
 *    Device pointers (the *_device calls) are borrowed for the duration of
 *    the call's work on the given stream only.
 *  - Errors: calls return an xrl_status; no exception crosses the ABI and the
 *    library never aborts.  xrl_last_error(ctx) gives a message for the last
 *    failing call on that context.  On error no output buffer is written.
 *  - Threading: one context is used by one host thread at a time.
 */
#ifndef XRL_H
#define XRL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xrl_ctx xrl_ctx; /* opaque, owned by the library */

typedef enum {
  XRL_OK = 0,
  XRL_EINVAL = 1,   /* bad argument (null pointer, size out of range, NaN) */
  XRL_ETOPO = 2,    /* mesh is not a closed 2-manifold, terminals touch, port spans two conductors */
  XRL_ENOMEM = 3,   /* device or host allocation failed */
  XRL_ECUDA = 4,    /* a CUDA runtime call failed (message has the CUDA error string) */
  XRL_ENOCONV = 5,  /* an iterative solve did not reach its tolerance in the allowed iterations */
  XRL_ETIMEOUT = 6, /* a bounded device-side wait gave up */
  XRL_ESTATE = 7    /* call out of order (e.g. solve before setup) */
} xrl_status;

typedef struct {
  int32_t fmm_order;   /* expansion order p of the solid-harmonic FMM (2..12), default 8 */
  int32_t leaf_target; /* mean panels per non-empty leaf used to pick the tree depth, default 32
                          (with mac_theta = 0 the depth is also capped so that leaf sides are >= 2x
                          the largest panel radius) */
  int32_t precision;   /* 0: FP64 everywhere (CUDA-core FP64 kernels); 1: mixed (FP32 FMM/near field
                          inside FP64 refinement); 2: FP64-accurate products throughout on the tensor
                          cores and FP32 pipes (the integer-slice and double-float kernels of mode 1's
                          residuals), no FP32 inner iterations */
  int32_t precond;     /* 0: none; 1: diagonal-of-P preconditioner of eq. 10 applied exactly (banded
                          LDL^T of the RCM-ordered vertex loops + Schur border); 2: eq. 10 applied
                          inexactly by Jacobi-preconditioned
                          COCG; 3: the diagonal-of-L preconditioner of Sec. II-D / Table IV,
                          Z_s + j omega L_d (loop-space surface impedance of eq. 8 kept whole, L_d the
                          diagonal of the branch-branch inductance sum_t A_t mu0/4pi P A_t^T), applied
                          like 1; 4: eq. 10 applied by one smoothed-aggregation multigrid V-cycle
                          (FP32).  1 and 3 take the multigrid V-cycle of their own matrix where the
                          band form is not usable (band wider than 63 or more than 16 global loops,
                          as on planes with many holes) */
  int32_t restart;     /* FGMRES restart length m, default 50 (Sec. III uses restart 50) */
  int32_t max_iters;   /* total outer iterations per solve, default 500 */
  int32_t inner_iters; /* max inner COCG iterations per preconditioner apply, default 60 */
  int32_t warm_start;  /* 0: zero initial guess; 1: with rhs_chunk, every frequency of a chunk starts
                          from the previous chunk's last-frequency solution of the same port, scaled
                          per system by the complex factor minimising the FP64 residual and kept only
                          where it lowers ||b - A x0|| by more than 1 % (the first chunk starts at 0) */
  double tol;          /* relative residual ||b - Ax|| / ||b|| per system, default 1e-8 */
  double inner_tol;    /* inner COCG relative residual, default 1e-3 */
  int32_t device;      /* CUDA device ordinal, default 0 */
  int32_t separation;  /* with mac_theta = 0: well-separatedness ws of the octree (1 or 2), leaves
                          within ws cells are near field; default 2 (see xrl_export_lists) */
  int32_t use_graphs;  /* 1 (default): the inner operator of every Arnoldi step is replayed from a
                          CUDA graph captured once per solve; 0: plain launches */
  int32_t tensor_cores; /* 1 (default): for n_cols >= 64 the FP32 products of the mixed mode run
                           their near field, P2M, M2M and M2L on the tcgen05 tensor cores (three
                           BF16 pieces, six products, ~FP32 accuracy) and the FP64-accurate
                           residuals their near field, M2M and M2L in 7-bit integer slices
                           (exact FP32 accumulation); 0: CUDA-core kernels only */
  double mac_theta;    /* > 0: two boxes of one octree level are far enough apart for the expansions
                          when rho_t + rho_s <= mac_theta |c_t - c_s| (c = box centre, rho = largest
                          distance from it to a vertex of the box's panels), the near field holds the
                          rest, and the depth has no leaf-size cap; must be < 1.  0 (default): the
                          cell-distance rule of `separation` with its leaf-size cap (see
                          xrl_export_lists) */
  int32_t mg_cycles;   /* V-cycles per multigrid preconditioner application (1..8), default 3 */
  int32_t rhs_chunk;   /* 0 (default): all (frequency, port) systems of xrl_solve form one multi-RHS
                          block; > 0: the frequencies are solved in consecutive chunks of at most
                          max(1, rhs_chunk / n_ports) frequencies (all ports of a frequency in one
                          chunk), which bounds the Krylov basis to (2 restart + 1) x n_loops x chunk
                          complex values */
} xrl_options;

/* Fill `opt` with the defaults listed above. */
void xrl_default_options(xrl_options* opt);

/* Create a context on opt->device (NULL opt = defaults).  *out receives the
 * handle; destroy it with xrl_destroy.  Returns XRL_ECUDA when no usable
 * GPU is present. */
xrl_status xrl_create(const xrl_options* opt, xrl_ctx** out);

/* Conductor surface mesh of triangles.  xyz: [n_vert][3] vertex coordinates
 * in metres; tri: [n_tri][3] vertex indices (any orientation); cond_id:
 * [n_tri] conductor index per panel (0-based, NULL = all 0).  Each edge must
 * be shared by exactly two panels; this is checked in xrl_setup (XRL_ETOPO).
 * The arrays are copied; the caller keeps ownership. */
xrl_status xrl_set_mesh(xrl_ctx* ctx, int64_t n_vert, const double* xyz, int64_t n_tri,
                        const int32_t* tri, const int32_t* cond_id);

/* Hybrid triangle/rectangle mesh (Sec. II-A, Figs. 1-2: currents on
 * "triangular and rectangular supports").  pan: [n_panels][4] vertex indices
 * in cyclic order; a triangle has -1 in its 4th slot.  A 4-vertex panel must be
 * a parallelogram (|v0 + v2 - v1 - v3| <= 1e-9 |v2 - v0|, else XRL_EINVAL): its
 * centroid is the vertex mean, its current a pulse (Sec. II-A, eq. 4) and its
 * integrals the sums over its triangles (v0, v1, v2) and (v0, v2, v3).  Its
 * four edges are branches of the PEEC graph (Algorithm 1); the diagonal is not.
 * Other arguments and errors as xrl_set_mesh; a repeated vertex in a panel is
 * XRL_ETOPO. */
xrl_status xrl_set_mesh_panels(xrl_ctx* ctx, int64_t n_vert, const double* xyz, int64_t n_panels,
                               const int32_t* pan, const int32_t* cond_id);

/* Material of each conductor: sigma [n_cond] in S/m and the thickness
 * varsigma [n_cond] in metres of the double-plane ESI model, eq. 3
 * (R_DC = 2/(sigma*varsigma), R_RF = sqrt(pi*mu0/sigma)). */
xrl_status xrl_set_conductors(xrl_ctx* ctx, int32_t n_cond, const double* sigma,
                              const double* thickness);

/* Add a port (Sec. III-B: source and sink terminals as in Q3D): the source
 * and sink terminal patches are lists of panel indices.  Each patch is
 * collapsed into one equipotential node carrying no surface current; an
 * ideal external branch with a 1 V source joins sink to source.  Patches of
 * different ports may coincide (a shared sink).  *port_id receives the
 * port's index (0-based, in call order). */
xrl_status xrl_add_port(xrl_ctx* ctx, int64_t n_src, const int32_t* src_panels, int64_t n_sink,
                        const int32_t* sink_panels, int32_t* port_id);

/* Geometry-dependent setup, once per mesh: panel geometry and Morton order,
 * octree and interaction lists, PEEC branches and the centroid-midpoint
 * matrices A_1..A_3 (Algorithm 1), a loop basis M (Sec. II-B), the
 * frequency-independent near-field block of P (Sec. II-C, filled once,
 * Sec. II-D) and the FMM operators. */
xrl_status xrl_setup(xrl_ctx* ctx);

/* y = P x for n_cols columns, HOST buffers, x and y laid out [n_cols][n_tri]
 * in caller panel order.  P_kl = (1/(A_k A_l)) int_k int_l 1/|r - r'| (eq. 6
 * with the centroid-midpoint normalisation), evaluated by the FMM of
 * Sec. II-C (near field by quadrature, far field by expansions of order p).
 * Copies in and out inside the call; synchronous. */
xrl_status xrl_fmm_mvm(xrl_ctx* ctx, int32_t n_cols, const double* x, double* y);

/* Same product on DEVICE buffers d_x, d_y ([n_cols][n_tri], FP64) enqueued on
 * `stream` (a cudaStream_t, NULL = the context's stream).  Asynchronous with
 * respect to the host; d_x and d_y must stay valid until the stream reaches
 * the end of this work.  d_x and d_y must not overlap. */
xrl_status xrl_fmm_mvm_device(xrl_ctx* ctx, int32_t n_cols, const double* d_x, double* d_y,
                              void* stream);

/* The FP32 product of the mixed-precision solver's inner iterations (Sec.
 * II-C evaluated in FP32: near field, P2M, M2M and M2L on the tensor cores
 * when opt.tensor_cores and n_cols >= 64, the near field on a second stream
 * of the context beside the far field; L2L and L2P FP32): y = P x on DEVICE
 * buffers d_x, d_y ([n_cols][n_tri], float32) enqueued on `stream` (NULL =
 * the context's stream).  Relative accuracy ~1e-6 (FP32 rounding plus the
 * order-p truncation).  Synchronises the stream on return to check the
 * tensor-core kernels' wait status (XRL_ETIMEOUT if one gave up). */
xrl_status xrl_fmm_mvm32_device(xrl_ctx* ctx, int32_t n_cols, const float* d_x, float* d_y, void* stream);

/* Same product as xrl_fmm_mvm_device, for callers that must not allocate GPU
 * memory: a real-time loop where a cudaMalloc could stall or fail, or a host
 * framework whose own allocator owns the device memory budget.  This call
 * allocates nothing: its working buffers (the Morton-ordered copies of x and
 * y and the multipole/local expansions, 2 N n_cols + 2 n_boxes (p+1)^2 n_cols
 * doubles) live in one fixed device array of XRL_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that the library declares statically; every GPU the library is
 * loaded on holds that array until the process exits.  Sizes that do not
 * fit return XRL_EINVAL (nothing is launched).  It always runs the plain
 * FP64 kernels (also in a precision = 1 context), which read only what
 * xrl_setup built.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, no allocation), so make that first
 * call before any stream capture.  All calls share the one array: two calls
 * whose work overlaps on the GPU (different streams, or different contexts
 * on the same device) race and corrupt each other's results, so serialise
 * them.  The array keeps the last call's contents; nothing in it needs to
 * start at zero.  Profiling (xrl_set_profiling) is not recorded for this
 * call.  The caller's current device is restored on return.  The paper has
 * no counterpart: this is an interface variant only.  d_x and d_y as for
 * xrl_fmm_mvm_device. */
#define XRL_NOALLOC_SCRATCH_BYTES (32u << 20)
xrl_status xrl_fmm_mvm_device_noalloc(xrl_ctx* ctx, int32_t n_cols, const double* d_x, double* d_y,
                                      void* stream);

/* Reference product y = P x by direct O(N^2) summation on the GPU, every
 * entry evaluated with the same quadrature rule table as the near field
 * (device buffers, layout as xrl_fmm_mvm_device). */
xrl_status xrl_direct_mvm_device(xrl_ctx* ctx, int32_t n_cols, const double* d_x, double* d_y,
                                 void* stream);

typedef struct {
  int32_t n_panels, n_live, n_branches, n_loops, n_ports, n_leaves, n_levels, n_boxes;
  int64_t near_nnz;      /* stored near-field entries */
  int32_t n_vertex_loops, n_global_loops;
  int32_t total_iters;   /* outer FGMRES iterations of the last solve (max over systems) */
  int32_t total_inner;   /* inner COCG iterations of the last solve */
  int32_t n_mvm;         /* operator applications (FMM products) in the last solve */
  double max_rel_res;    /* largest final true relative residual of the last solve */
  double setup_ms, solve_ms, mvm_ms; /* wall times of the last setup / solve / fmm_mvm */
  int64_t peak_device_bytes;         /* high-water mark of the library's device allocations */
  int64_t near_nnz_padded;  /* near-field entries of the tensor-core near blocks (leaves padded to
                               16 panels); 0 when that path is off */
  double precond_setup_ms;  /* host + device time of the last setup spent building the preconditioner
                               pencil (P entries, loop pattern, band ordering and band values) */
  int32_t tc_targets_per_cta; /* targets per CTA of the FP32 tensor-core M2L and near field (2: sibling
                                 pairs share a CTA where the coefficients / padded leaves are <= 64;
                                 1: one each), as xrl_autotune chose it; 2 before any autotune */
  double setup_phase_ms[6]; /* the last setup's host wall time by phase: 0 PEEC topology and loops,
                               1 panel geometry, Morton order and octree, 2 near-field fill, 3 moments
                               and translation operators (incl. tensor-core images), 4 preconditioner
                               pencil and band, 5 solver operator data */
  int32_t mg_levels;        /* levels of the multigrid hierarchy of Q (0: none built) */
  int32_t mg_coarse_n;      /* unknowns of its coarsest level */
  int64_t device_bytes;     /* device memory the context's buffers hold now */
  int64_t cached_device_bytes; /* freed blocks the context keeps for reuse (released when an
                                  allocation fails, at every setup and at destroy) */
} xrl_stats;

/* FMM autotuner: tries leaf_target in {16, 32, 64} x fmm_order in {4, 6, 7, 8}
 * (with the context's separation rule), re-running xrl_setup for each.  A candidate is admissible
 * when its FP64 product matches the FP64 direct sum (xrl_direct_mvm_device) on
 * two seeded random columns to mvm_tol (relative 2-norm; above 32,768 panels
 * the norm is taken over 1024 spread rows, whose direct sums are computed).  Each admissible
 * candidate's product at n_cols columns is timed with CUDA events in the
 * precision the solver's products use (FP32 if `precision` = 1, the
 * FP64-accurate tensor-core product if 2, else FP64); in FP32 each candidate
 * is timed with one and with two sibling targets per tensor-core CTA and
 * keeps the faster (xrl_stats.tc_targets_per_cta).  Among the candidates
 * within 3% of the fastest time, the one with the smallest product error is
 * kept (so that timing noise does not flip the choice).  The context ends set
 * up with it, and its options are updated.  Outputs (host, may be NULL): the
 * chosen leaf_target, fmm_order, its product time in ms, and its error.
 * XRL_ENOCONV if no candidate meets mvm_tol (the context is left set up with
 * the most accurate one). */
xrl_status xrl_autotune(xrl_ctx* ctx, int32_t n_cols, double mvm_tol, int32_t precision, int32_t* leaf_target,
                        int32_t* fmm_order, double* product_ms, double* product_err);

/* Counters and timings of the context (valid after setup). */
xrl_status xrl_get_stats(const xrl_ctx* ctx, xrl_stats* out);

/* Broadband sweep (Sec. II-D, Sec. III): for each frequency f in freq_hz
 * [n_freq] (f > 0), all ports are excited one at a time and the loop system
 * of eq. 7-8 is solved by right-preconditioned flexible GMRES with the FMM
 * product; all (frequency, port) systems form one multi-RHS block, or blocks
 * of opt.rhs_chunk systems (then xrl_stats.total_iters sums the blocks'
 * iteration counts).  Output:
 * R, L [n_freq][n_ports][n_ports], R = Re Z_port (ohm), L = Im Z_port / omega
 * (henry), Z_port = Y^-1 with Y the short-circuit port admittance.  Returns
 * XRL_ENOCONV (outputs still written) if some system did not reach opt.tol. */
xrl_status xrl_solve(xrl_ctx* ctx, int32_t n_freq, const double* freq_hz, double* R, double* L);

/* Loop-space operator for parity checks: w_s = Z(f_s) v_s for n_sys systems,
 * Z(f) = M [sum_t A_t (diag(Z_s(f)/A) + j omega mu0/4pi P) A_t^T] M^T (eq. 8),
 * with P applied by the FMM in FP64 accuracy, computed as the solver's
 * residuals compute it (opt.precision = 1: double-float arithmetic on the
 * FP32 pipes for n_sys >= 6).  Host buffers: freq [n_sys]; v, w
 * [n_sys][n_loops] complex as interleaved (re, im) doubles. */
xrl_status xrl_apply_operator(xrl_ctx* ctx, int32_t n_sys, const double* freq, const double* v,
                              double* w);

/* Preconditioner action for parity checks: w_s = Q(f_s) v_s with Q of eq. 10
 * (opt.precond = 1 or 2) or the diagonal-of-L Q_L (opt.precond = 3), the
 * sparse matrix itself, not its inverse; layout as xrl_apply_operator. */
xrl_status xrl_apply_precond_matrix(xrl_ctx* ctx, int32_t n_sys, const double* freq,
                                    const double* v, double* w);

/* Preconditioner solve for parity checks: w_s = Q(f_s)^-1 v_s by the banded
 * LDL^T + Schur border factorisation (XRL_EINVAL if the band form is not
 * usable for this mesh); layout as xrl_apply_operator. */
xrl_status xrl_apply_precond_inverse(xrl_ctx* ctx, int32_t n_sys, const double* freq, const double* v,
                                     double* w);

/* Export of setup products for checks (host buffers sized from xrl_get_stats):
 *  tree:   keys [n_panels] Morton keys (caller order), perm [n_panels] Morton
 *          rank -> caller index, leaf_of [n_panels] leaf index per Morton rank;
 *  branch: tail, head [n_branches] (panel index, or -1-terminal for a
 *          terminal node; port branches last: tail = -1-sink, head = -1-source);
 *  loops:  CSR of M: row_ptr [n_loops+1], col [nnz], val [nnz] (+1/-1);
 *          pass col = val = NULL to get nnz in row_ptr[n_loops]. */
xrl_status xrl_export_tree(const xrl_ctx* ctx, uint64_t* keys, int32_t* perm, int32_t* leaf_of);
xrl_status xrl_export_branches(const xrl_ctx* ctx, int32_t* tail, int32_t* head);
xrl_status xrl_export_loops(const xrl_ctx* ctx, int64_t* row_ptr, int32_t* col, int8_t* val);

/* Interaction lists of the octree (uniform depth).  With mac_theta > 0 two
 * boxes of one level are well separated when rho_t + rho_s <= mac_theta
 * |c_t - c_s| (c = centre of the box's cell, rho = largest distance from c to
 * a vertex of the box's panels); at level 1 every pair is near, at level
 * l >= 2 the candidates of a box are the children of its parent's near
 * boxes, split into the V-list (well separated) and the near list, and the
 * leaf level's near lists are the U-lists (near field).  With mac_theta = 0:
 * U-list = leaves within `separation` cells in every direction, V-list =
 * children of the parent's near boxes that are not near the box.  Output,
 * for level l in [2, n_levels): box counts, Morton keys of the occupied boxes
 * and the V-list (multipole-to-local) pairs as CSR over target boxes, and for
 * the leaf level the U-list as CSR.  Sizes via the counts query (pass NULL
 * arrays). */
xrl_status xrl_export_lists(const xrl_ctx* ctx, int32_t level, int32_t* n_boxes, uint64_t* box_keys,
                            int64_t* v_ptr, int32_t* v_src, int64_t* u_ptr, int32_t* u_src);

/* ---- learned initial guess -------------------------------------------------
 * Not part of the paper: a per-panel network predicts the panel current
 * distribution of a sweep from its lowest frequency, and the prediction is
 * used only as the FGMRES starting point, judged by the FP64 residual. */

/* Panel currents of the last xrl_solve: Ip [n_sys][n_panels][6] (caller
 * panel order, system s = freq index * n_ports + port), entries
 * (Re, Im) of I_x, I_y, I_z with I_p = J * area (A m).  normalize != 0
 * divides each system by its complex port current (per unit port current). */
xrl_status xrl_get_panel_currents(xrl_ctx* ctx, int32_t normalize, double* Ip);

/* Per-panel features for the network, DEVICE buffers: d_ip0 [n_ports][n_panels][6]
 * (FP64, per unit port current at the reference frequency f0, caller order),
 * d_feat [n_freq * n_ports][n_panels][24] (FP32, caller order).  The reference
 * currents of port q enter scaled by scale[q] = 1 / max_p |I_p| (written to
 * the host array `scale` [n_ports] when not NULL; training targets use the
 * same scale).  Features:
 * 0-2 centroid in the root cube, 3-5 unit normal, 6 log(A / mean A)/4,
 * 7 4 x mean (1 - |n . n_j|) over edge neighbours, 8 (log10 f - 5)/5,
 * 9 log10(f/f0)/10, 10-15 the reference currents, 16 log10(skin depth /
 * ESI thickness)/3, 17 |reference current|, 18 terminal flag, 19-20
 * sin/cos(log10 f), 21 one, 22 port / n_ports, 23 zero.  Synchronous. */
xrl_status xrl_panel_features(xrl_ctx* ctx, int32_t n_freq, const double* freq_hz, double f0,
                              const double* d_ip0, float* d_feat, double* scale, void* stream);

/* xrl_solve starting from predicted panel current SHAPES d_shape
 * [n_freq * n_ports][n_panels][6] (device, FP32, caller order): each is
 * projected onto loop space by weighted least squares (weights 1/area, the
 * resistive energy norm; solved with the banded factorisation of the pencil
 * at Z_s = 1), scaled by the complex factor minimising the FP64 residual, and
 * kept only where it lowers ||b - A x0|| by more than 1 % (else x0 = 0).
 * accepted [n_sys] and guess_res [n_sys] (||b - A x0|| / ||b||) are host
 * outputs (may be NULL).  Needs precond = 1 with a usable band. */
xrl_status xrl_solve_guess(xrl_ctx* ctx, int32_t n_freq, const double* freq_hz, const float* d_shape, double* R,
                           double* L, int32_t* accepted, double* guess_res);

typedef struct xrl_mlp xrl_mlp; /* opaque network: n_in -> width (GELU) x n_hidden -> n_out */

/* Create a network on `device`; weights He-uniform from `seed`.  Parameters
 * (FP32 master copy) are laid out per layer l: W_l [in_l][out_l] row-major,
 * then b_l [out_l].  Forward and backward use the weights rounded to BF16
 * (nearest even) and accumulate in FP32. */
xrl_status xrl_mlp_create(int32_t n_in, int32_t width, int32_t n_hidden, int32_t n_out, uint64_t seed,
                          int32_t device, xrl_mlp** out);
int64_t xrl_mlp_num_params(const xrl_mlp* mlp);
/* d_y [rows][n_out] = network(d_x [rows][n_in]); device buffers, enqueued on stream. */
xrl_status xrl_mlp_forward(xrl_mlp* mlp, int64_t rows, const float* d_x, float* d_y, void* stream);
/* One AdamW step (beta 0.9 / 0.999, eps 1e-8; weight decay on weights only)
 * on the mean squared error of d_x against targets d_t [rows][n_out]; *loss
 * receives the loss before the step.  Synchronises the stream. */
xrl_status xrl_mlp_train_step(xrl_mlp* mlp, int64_t rows, const float* d_x, const float* d_t, float lr,
                              float weight_decay, double* loss, void* stream);
/* Gradient of the mean squared error w.r.t. the parameters into h_grads
 * (host, parameter layout); no update. */
xrl_status xrl_mlp_gradients(xrl_mlp* mlp, int64_t rows, const float* d_x, const float* d_t, float* h_grads,
                             double* loss);
xrl_status xrl_mlp_get_params(const xrl_mlp* mlp, float* h_params);
xrl_status xrl_mlp_set_params(xrl_mlp* mlp, const float* h_params);
const char* xrl_mlp_last_error(const xrl_mlp* mlp);
void xrl_mlp_destroy(xrl_mlp* mlp);

/* Per-phase device timing, recorded with CUDA events on the stream each
 * phase's kernels run on, while profiling is switched on (xrl_set_profiling).
 * phase: 0 P2P near field (FP32), 1 P2M, 2 M2M, 3 M2L (FP32), 4 L2L, 5 L2P,
 * 6 operator gather/scatter, 7 preconditioner (factor and solves), 8
 * Arnoldi/FGMRES updates, 9 P2P near field (FP64), 10 M2L (FP64: native, or
 * double-float on the FP32 pipes inside mixed-precision solves).
 * ms = summed event time, launches = kernel launches, flops / bytes =
 * algorithmic work (not counters) summed over those launches.  Reading
 * synchronises the context's stream.  xrl_kernel_launches returns every
 * kernel launch of the library on this context since creation. */
xrl_status xrl_set_profiling(xrl_ctx* ctx, int32_t on);
xrl_status xrl_get_profile(xrl_ctx* ctx, int32_t phase, double* ms, int64_t* launches, double* flops,
                           double* bytes);
xrl_status xrl_reset_profile(xrl_ctx* ctx);
int64_t xrl_kernel_launches(const xrl_ctx* ctx);

/* The cudaStream_t (as void*) on which the context enqueues its own work
 * (setup, xrl_fmm_mvm, xrl_solve); NULL for a NULL context. */
void* xrl_get_stream(const xrl_ctx* ctx);

/* Last error message of this context ("" if none).  Valid until the next call. */
const char* xrl_last_error(const xrl_ctx* ctx);

/* Release every resource of the context (NULL is ignored). */
void xrl_destroy(xrl_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* XRL_H */
