/*
 * rbf.h -- C ABI of the GB300 (sm_103a) band-limited FMM for radial basis
 * function interpolation, after Zhao & Stoll, "A Fast Multipole Method based
 * on Band-limited Approximations for Radial Basis Functions" (arXiv 1606.07652).
 *
 * The library computes u = A lambda with A_ij = Phi(x_i - x_j) (Eq. (1)) by the
 * paper's FMM: a near field summed point to point over neighbour leaves and a
 * far field carried by exponential (band-limited Fourier quadrature)
 * expansions, Eqs. (35)-(38), (43)-(48), (54).  It also solves A lambda = u
 * with GMRES driven by that product (Sec. 1).
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers unless the name ends in _host.  The caller
 *    owns every pointer it passes; the library never frees them.
 *  - The library owns rbf_tree and everything hanging off it (sorted points,
 *    lists, coefficient tables, expansion workspace); rbf_tree_free releases it.
 *  - Every call returns an int: RBF_OK (0) or a negative RBF_E* code; no C++
 *    exception crosses the ABI.  rbf_last_error() gives a message for the last
 *    failure on the calling thread.
 *  - Work is enqueued on `stream` (a cudaStream_t, or NULL for the legacy
 *    default stream).  Calls that return results in host memory synchronise
 *    that stream before they return; the others are asynchronous.
 *  - Vectors lambda and u are in the caller's original point order; the
 *    Morton permutation is internal.  Several right-hand sides are stored
 *    column-major with a leading dimension (ld >= N).
 *  - A tree is not thread-safe: calls on one tree must not overlap in time.
 */
#ifndef RBF_H
#define RBF_H

#include <stdint.h>

#if defined(__GNUC__)
#define RBF_API __attribute__((visibility("default")))
#else
#define RBF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define RBF_OK 0
#define RBF_EINVAL (-1)   /* bad argument (null pointer, size, parameter range) */
#define RBF_ENOMEM (-2)   /* device allocation failed */
#define RBF_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define RBF_ENOCONV (-4)  /* iterative solve stopped before reaching rtol */
#define RBF_ETIMEOUT (-5) /* a bounded device-side wait ran out */
#define RBF_ENOTSUP (-6)  /* combination not supported by this build */

#define RBF_MAX_DIM 6
#define RBF_MAX_DEPTH 10

/* Radial kernels of the tables "Global functions" and "Compactly supported
 * functions" (Sec. 2.2) in shape-parameter form: Gaussian
 * Phi(r) = exp(-(eps r)^2); inverse multiquadric Phi(r) = 1/sqrt(1 + (eps r)^2);
 * multiquadric Phi(r) = sqrt(1 + (eps r)^2); Wendland
 * Phi(r) = (1 - eps r)_+^3 (3 eps r + 1) (Phi_{2,1}, support radius 1/eps; the
 * compact kernel of the numerical examples, Sec. 5).  All have Phi(0) = 1.
 * The multiquadric grows with r and needs the taper (window_alpha > 0). */
typedef enum { RBF_GAUSSIAN = 0, RBF_IMQ = 1, RBF_MQ = 2, RBF_WENDLAND = 3 } rbf_kernel;

/* Arithmetic of the matrix-vector product.  Inputs and outputs of
 * rbf_fmm_matvec are FP64 in both cases. */
typedef enum { RBF_FP64 = 0, RBF_FP32 = 1 } rbf_precision;

/* Parameters of the band-limited expansion (Sec. 3.2, "Low-rank representation").
 *  M            quadrature nodes per dimension (even, 2..64).  The nodes are
 *               xi_k = k * 2pi/L, k = -M/2..M/2, with half weight at +-M/2,
 *               so the band limit is sigma = pi M / L.  M = 0: no far field;
 *               the product is the near field alone (far kernel K = 0), which
 *               is within max_far |Phi| (rbf_kernel_error) of the exact product:
 *               for kernels that vanish beyond one leaf width (narrow
 *               Gaussians, compact supports).  The other fields are then
 *               ignored except grid, which must be RBF_GRID_SHARED.
 *  period_L     period of the sampled kernel; must exceed the root side (twice
 *               the root side when window_alpha > 0).  Far offsets have
 *               components below `side`, so Phi(L - side) bounds the image error.
 *  window_alpha steepness of the erfc taper applied to slowly decaying kernels
 *               before periodisation (0 = no taper).  The taper is flat on
 *               |t| <= side and falls to ~0 at |t| = L - side.
 *  csample      1: C(xi) from samples of Phi on the lattice h Z^d, h = L/M
 *               (Eq. (M2Loperator), the paper's kernel-independent route);
 *               0: closed-form Gaussian transform (validation, Gaussian only).
 *  grid         RBF_GRID_SHARED (0): one frequency grid on every level; M2M and
 *               L2L are exact diagonal shifts (interpolation P = I in Eqs. (43)
 *               and (48)).
 *               RBF_GRID_NESTED (1): the scale-invariant grids of Sec. 4.1.1:
 *               the same M on every level, xi_{l-1} = xi_l / 2 (level l uses
 *               period L * 2^(2-l) and coefficients sampled at that scale,
 *               flat taper radius side * 2^(2-l)); M2M interpolates and L2L
 *               anterpolates in xi with local Lagrange stencils (Eqs. (43),
 *               (47), (48), (51)).  Needs d <= 3, csample = 1,
 *               window_alpha > 0 and M >= 2 lagrange_K; single right-hand-side
 *               kernels only (several columns run one after another).
 *  lagrange_K   points of the Lagrange stencil of the nested grids (even,
 *               2..16; 0 = 8).  Ignored on the shared grid. */
#define RBF_GRID_SHARED 0
#define RBF_GRID_NESTED 1
typedef struct {
    int M;
    double period_L;
    double window_alpha;
    int csample;
    int grid;
    int lagrange_K;
} rbf_fmm_params;

typedef struct rbf_tree rbf_tree;

/* Summary of a built tree (host struct). */
typedef struct {
    int64_t N;
    int d;
    int depth;                 /* D: leaves are the level-D boxes */
    double lo[RBF_MAX_DIM];    /* root cube [lo, lo + side]^d */
    double side;
    int64_t n_leaf;            /* non-empty leaves */
    int64_t n_near;            /* entries of all near lists */
    int64_t max_leaf_points;   /* largest leaf */
    int64_t n_box[RBF_MAX_DEPTH + 1]; /* non-empty boxes per level */
} rbf_tree_info;

/* Build the Morton tree of the centres (Sec. 1, "hierarchical tree
 * partitioning"; groups G_b and neighbour lists N_a of Eq. (38)).
 *  X        device, [N][d] row-major FP64, caller's order.
 *  N        number of centres, 1 <= N < 2^31.
 *  d        dimension, 1..RBF_MAX_DIM.
 *  lo_host  host array of d doubles, the root cube's lower corner, or NULL to
 *           use the bounding box of X (then `side` is ignored and set to the
 *           largest extent).
 *  side     root cube edge (> 0) when lo_host is given.
 *  depth    D, 0..RBF_MAX_DEPTH with d*D <= 63; depth < 0 picks
 *           round(log_{2^d}(N/32)) clamped to [2, RBF_MAX_DEPTH].
 *  out      receives the new tree (NULL on failure).
 * Box coordinates are k_t = min(max(floor(((x_t-lo_t)/side)*2^D), 0), 2^D-1)
 * in FP64; Morton keys put dimension 0 in bit 0; the sort is stable by
 * (key, original index).  Synchronises `stream`. */
RBF_API int rbf_tree_build(const double *X, int64_t N, int d, const double *lo_host, double side, int depth,
                   void *stream, rbf_tree **out);

/* Fill *info_host.  No device work. */
RBF_API int rbf_tree_get_info(const rbf_tree *t, rbf_tree_info *info_host);

/* Copy the tree to host arrays for bit-exact checks; any pointer may be NULL.
 *  perm[N]            sorted position -> original index
 *  keys[N]            Morton keys of the sorted points
 *  leaf_key[n_leaf]   Morton keys of the non-empty leaves, ascending
 *  leaf_off[n_leaf+1] first sorted point of each leaf
 *  near_off[n_leaf+1], near_idx[n_near]  CSR near lists N_a (compact leaf ids,
 *                     ascending; leaves at Chebyshev index distance <= 1,
 *                     self included).  Synchronises `stream`. */
RBF_API int rbf_tree_export(const rbf_tree *t, int64_t *perm, uint64_t *keys, uint64_t *leaf_key,
                    int64_t *leaf_off, int64_t *near_off, int64_t *near_idx, void *stream);

/* Interaction lists IL_l of the MLFMM coupling step (Sec. 4.1, Eq. (45)) for one
 * level 2 <= l <= D: level-l boxes whose parents are within Chebyshev distance
 * 1 of the parent of a and which are at distance >= 2 from a.  Built on the
 * device on first request.  box_key[n_box[l]] (ascending Morton keys of the
 * non-empty level-l boxes), il_off[n_box[l]+1], il_idx[*n_il_host] (compact
 * level-l ids, ascending).  Pass il_idx = NULL to query *n_il_host first.
 * Synchronises `stream`. */
RBF_API int rbf_tree_export_level(rbf_tree *t, int level, uint64_t *box_key, int64_t *il_off,
                          int64_t *il_idx, int64_t *n_il_host, void *stream);

/* u = A lambda by the band-limited FMM (Eqs. (38), (54)):
 *   u_i = sum_{j in near leaves} lambda_j Phi(x_i - x_j)
 *       + sum_{other j} lambda_j K(x_i - x_j),
 *   K(r) = sum_xi omega(xi) C(xi) e^{i xi . r}   (Eq. (35)).
 * Passes: near field, P2M at the leaves (Eq. (P2M)), M2M upsweep (Eq. (43),
 * one shared grid), coupling (Eq. (45)), downsweep to the leaves (Eq. (48)),
 * L2P (Eq. (46)).
 *  lambda   device FP64, N x nrhs column-major, leading dimension ld_lambda.
 *  u        device FP64, N x nrhs column-major, leading dimension ld_u; written.
 *  prec     RBF_FP64 or RBF_FP32 arithmetic for every pass.
 *  params   expansion parameters (see rbf_fmm_params); NULL = defaults
 *           (M=32, L=4 side, alpha=0 for the Gaussian and 4.5 for the other
 *           kernels, csample=1, shared grid).
 * Coefficient tables and expansion workspace are built on first use and kept
 * in the tree until the parameters change.  Asynchronous.
 * With RBF_FP32 and nrhs >= RBF_MULTI_RHS_MIN the columns go through the far
 * field G at a time (G <= 16, bounded by min(64 GB, half the free device
 * memory) of expansion workspace): P2M and L2P of the G columns are complex
 * matrix products on the tensor cores (three-term split TF32 operands, FP32
 * accumulation), the translations run per column.  Check
 * rbf_check_device_waits after such calls when a bounded device wait must be
 * ruled out. */
#define RBF_MULTI_RHS_MIN 4
RBF_API int rbf_fmm_matvec(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *params,
                   rbf_precision prec, const double *lambda, int64_t ld_lambda, double *u,
                   int64_t ld_u, int nrhs, void *stream);

/* Synchronises the device and reports whether a bounded wait inside a
 * tensor-core kernel gave up since the previous call (RBF_ETIMEOUT, with the
 * kernel's results left incomplete) or not (RBF_OK).  Clears the record. */
RBF_API int rbf_check_device_waits(void);

/* Same product with host buffers: copies lambda_host to the device, runs
 * rbf_fmm_matvec, copies u back.  Synchronises `stream`. */
RBF_API int rbf_fmm_matvec_host(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *params,
                        rbf_precision prec, const double *lambda_host, double *u_host, int nrhs,
                        void *stream);

/* Plain O(N^2) sum of Eq. (1) in FP64 at selected targets (error checks):
 *  X [N][d] row-major, lambda [N], targets [nt] (indices into X), u [nt].
 *  A target index outside [0, N) gives NaN in its entry of u. */
RBF_API int rbf_direct_sum(const double *X, int64_t N, int d, rbf_kernel kernel, double eps,
                   const double *lambda, const int64_t *targets, int64_t nt, double *u, void *stream);

/* Solver options for rbf_interp_solve (Sec. 1: GMRES with the FMM product).
 *  restart_m   Krylov dimension per restart (1..200).
 *  max_iters   total inner iterations over all restarts and refinements; each
 *              refinement step may use max(restart_m, max_iters / max_refine).
 *  max_refine  outer FP64 refinement steps (>= 1).
 *  rtol        target ||u - A lambda||_2 / ||u||_2, measured with the FP64 FMM.
 *  inner_prec  arithmetic of the matvec inside GMRES (RBF_FP64 or RBF_FP32).
 *  precond     0: none (the diagonal of A is Phi(0) = 1, so the diagonal
 *              preconditioner is the identity); 1: learned sparse approximate
 *              inverse (built with rbf_precond_build).  With precond = 1 the
 *              first correction step is a trial: one GMRES cycle of restart_m
 *              iterations with P; if its inner solve does not converge within
 *              that cycle, one plain cycle from the same iterate follows and
 *              the iterate with the smaller FP64 residual is kept (P is
 *              dropped, used_fallback = 1, when the plain cycle wins).  A P
 *              that does not help therefore costs at most one cycle.  Later
 *              steps also drop P when a preconditioned step fails to halve
 *              the FP64 residual.
 *  history_host  optional (NULL: none): host array of 4 * history_cap
 *              doubles that receives the residual history (rbf_solve_report).
 *  history_cap   its capacity in entries. */
typedef struct {
    int restart_m;
    int max_iters;
    int max_refine;
    double rtol;
    rbf_precision inner_prec;
    int precond;
    double *history_host;
    int history_cap;
} rbf_solve_opts;

/* Per-solve report (host struct).  When rbf_solve_opts::history_host is set,
 * the solve appends one entry (inner iterations so far, seconds since the
 * start, relative residual, kind) at every FP64 true residual (kind
 * RBF_HIST_FP64: ||u - A64 lambda|| / ||u||) and at every GMRES restart
 * (kind RBF_HIST_INNER: the residual of the inner correction equation, with
 * the inner-precision product, over ||u||), stops at history_cap entries and
 * reports the count in history_len. */
#define RBF_HIST_FP64 0
#define RBF_HIST_INNER 1
typedef struct {
    int iters;            /* inner GMRES iterations, all restarts */
    int refinements;      /* correction steps taken (GMRES calls) */
    int used_fallback;    /* 1 when the learned preconditioner was dropped */
    double rel_resid;     /* final ||u - A64 lambda|| / ||u|| */
    double seconds;       /* wall time of the solve */
    int matvecs_inner;    /* products in inner arithmetic */
    int matvecs_fp64;     /* FP64 products for true residuals */
    int history_len;      /* residual-history entries written */
} rbf_solve_report;

/* Solve A lambda = u (one right-hand side at a time, nrhs columns) with
 * restarted, right-preconditioned GMRES (two-pass classical Gram-Schmidt,
 * Givens rotations; FP64 basis) inside an FP64 iterative-refinement loop:
 * r = u - A64 lambda, GMRES on A delta = r with the inner-precision matvec,
 * lambda += delta, until ||r||/||u|| <= rtol.  lambda holds the initial guess
 * on entry (zero it for a cold start) and the solution on return.
 * u, lambda: device FP64 N x nrhs, leading dimension N.  rep_host may be NULL.
 * Returns RBF_ENOCONV (lambda still holds the best iterate) when the budget
 * runs out.  Synchronises `stream`. */
RBF_API int rbf_interp_solve(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *params,
                     const double *u, double *lambda, int nrhs, const rbf_solve_opts *opts,
                     rbf_solve_report *rep_host, void *stream);

/* Per-pass device timing.  While enabled, every product on the tree records a
 * pair of CUDA events around each pass, on the stream the pass runs on.
 * Pass ids: RBF_PASS_P2P near field, RBF_PASS_P2M, RBF_PASS_M2M upsweep,
 * RBF_PASS_M2L coupling + downsweep, RBF_PASS_L2P, RBF_PASS_PERM gather of
 * lambda and scatter of u.  rbf_profile(t, 1) enables and clears,
 * rbf_profile(t, 0) disables.  rbf_profile_read synchronises on the recorded
 * events and returns, per pass, the summed milliseconds and the number of
 * kernel launches since the last clear (host arrays of RBF_PASS_COUNT). */
#define RBF_PASS_P2P 0
#define RBF_PASS_P2M 1
#define RBF_PASS_M2M 2
#define RBF_PASS_M2L 3
#define RBF_PASS_L2P 4
#define RBF_PASS_PERM 5
#define RBF_PASS_COUNT 6
RBF_API int rbf_profile(rbf_tree *t, int enable);
/* Launch shape of the FP32 P2M that the tree's FP32 plan measured when it was
 * created (both shapes run twice on the tree, the faster kept; the shapes give
 * the same bits): *shape_host = 1 dense (five CTAs of up to 192 threads per SM),
 * 2 wide (four of up to 256), 0 chosen by rule (no FP32 plan yet, fewer than
 * 16,384 points, column segments wider than 36, nested grids or no far field). */
RBF_API int rbf_p2m_launch_shape(const rbf_tree *t, int *shape_host);
RBF_API int rbf_profile_read(rbf_tree *t, double *ms_host, int64_t *launches_host);

/* Measured peak rate of one arithmetic unit of the current device (the
 * denominators of roofline fractions; the paper has no counterpart).  A grid
 * of 32 warps per SM runs independent dependency chains of one instruction:
 *  RBF_PROBE_FFMA   FP32 fused multiply-add, in flop/s (2 per FMA)
 *  RBF_PROBE_DFMA   FP64 fused multiply-add, in flop/s
 *  RBF_PROBE_EX2    ex2.approx.f32 on the multi-function unit, results/s
 *  RBF_PROBE_RSQRT  rsqrt.approx.f32 on the multi-function unit, results/s
 * seconds (0, 10]: length of the timed launch (after a short calibration).
 * rate_host: the measured rate.  Synchronises `stream`; allocates a small
 * output buffer for the duration of the call. */
#define RBF_PROBE_FFMA 0
#define RBF_PROBE_DFMA 1
#define RBF_PROBE_EX2 2
#define RBF_PROBE_RSQRT 3
RBF_API int rbf_peak_probe(int kind, double seconds, double *rate_host, void *stream);

/* Morton order of the centres without any device allocation.  The paper has
 * no counterpart; this entry point exists for callers that must not call
 * cudaMalloc at call time: code whose device memory is owned by another
 * allocator (a framework's memory pool that already holds the free memory),
 * and latency-critical loops that re-sort moving centres every step, where
 * cudaMalloc/cudaFree would add allocation latency and may synchronise the
 * whole device.
 * It computes exactly what rbf_tree_build stores as keys and perm (same box
 * coordinates, Morton keys and stable (key, index) radix sort), with every
 * temporary buffer (the second key/index buffer, digit histograms, scan
 * partial sums) in one file-scope device arena of fixed size (54,528,000
 * bytes, 52 MiB), which every GPU that loads the library holds until the
 * process exits.
 *  X         device [N][d] row-major FP64, caller's order.
 *  N         1 .. 4,194,304 (= 2^22, the arena's limit); larger N returns
 *            RBF_EINVAL with a message.
 *  d, depth  as rbf_tree_build (depth >= 0, d*depth <= 63).
 *  lo_host   host array of d doubles (root cube corner), read during the
 *            call and passed to the device by value; side > 0.
 *  perm      device int32[N], written: sorted position -> original index.
 *  keys      device uint64[N], written: Morton keys in sorted order.
 * Asynchronous on `stream`; it allocates no memory and calls no allocating
 * library routine.  The first call in each CUDA context of a device (the
 * primary context, and again after a cudaDeviceReset) looks up the arena's
 * device address with that device current (cudaGetSymbolAddress) and caches
 * it for that context; make that first call before any stream capture.
 * Every call shares the one arena, and each region of it
 * is fully rewritten before it is read, so the previous call's contents never
 * leak into a result; calls that overlap in time on the GPU (different
 * streams or threads) race on the arena and must be serialised by the caller. */
RBF_API int rbf_morton_order_noalloc(const double *X, int64_t N, int d, const double *lo_host,
                                     double side, int depth, int32_t *perm, uint64_t *keys,
                                     void *stream);

/* ---------------------------------------------------------------------------
 * Learned approximate-cardinal preconditioner for rbf_interp_solve.
 * Column i of P carries weights on the RBF_KNN nearest centres S_i of centre i
 * (itself first), approximating its local cardinal function: sum_{j in S_i}
 * w_j Phi(x_k - x_j) = delta_{ik} on S_i.  A small MLP maps eps-scaled
 * neighbour offsets to the direction of those weights; each column is then
 * scaled so that it is exactly cardinal at its own centre.  The network is
 * trained on exact FP64 local solves.  The paper has no preconditioner: this
 * is an extension of its Krylov solve (Sec. 1).
 * ------------------------------------------------------------------------- */
#define RBF_KNN 32

/* k-nearest neighbours of every centre (RBF_KNN of them, itself included),
 * ascending squared distance sum_t (x_t - y_t)^2 in FP64, ties by original
 * index.  idx_host: host int64[N][RBF_KNN], original indices.  Computed on
 * the device once per tree (rings of leaves until the k-th distance is
 * certified) and kept.  Synchronises `stream`. */
RBF_API int rbf_knn(rbf_tree *t, int64_t *idx_host, void *stream);

/* Exact local cardinal coefficients c = (A_S + delta I)^-1 e_1 on S = the
 * neighbours of each listed centre (original indices centres_host[nc]), with
 * A_S[j][k] = Phi(x_j - x_k) and delta = delta_rel * ||A_S||_F; FP64 Cholesky,
 * one warp per centre.  A failed factorisation yields NaN.  c_host: host
 * double[nc][RBF_KNN].  Synchronises `stream`. */
RBF_API int rbf_cardinal_weights(rbf_tree *t, rbf_kernel kernel, double eps, double delta_rel,
                                 const int64_t *centres_host, int64_t nc, double *c_host,
                                 void *stream);

/* Network input of each listed centre: eps (x_j - x_i) for its neighbours j in
 * distance order, flattened (RBF_KNN * d floats).  F: device float[nc][32 d]. */
RBF_API int rbf_precond_features(rbf_tree *t, double eps, const int64_t *centres_host, int64_t nc,
                                 float *F, void *stream);

/* The network: d_in -> width -> width -> width -> d_out, ReLU on the hidden
 * layers, FP32 master weights with BF16 copies for the tensor-core GEMMs
 * (mma.sync BF16, FP32 accumulation).  Parameters are flattened layer by layer
 * as W_l (out x in, row-major) then b_l.  Initial weights: He-normal from a
 * counter-based generator (SplitMix64 + Box-Muller) seeded by `seed`, zero
 * biases. */
typedef struct rbf_mlp rbf_mlp;
RBF_API int rbf_mlp_create(int d_in, int width, int d_out, uint64_t seed, rbf_mlp **out);
RBF_API int rbf_mlp_num_params(const rbf_mlp *net, int64_t *count);
RBF_API int rbf_mlp_get_params(const rbf_mlp *net, float *host);
/* Sets the FP32 master weights (and their BF16 copies) and resets Adam. */
RBF_API int rbf_mlp_set_params(rbf_mlp *net, const float *host);
/* Y[B][d_out] = network(X[B][d_in]); device FP32 arrays. */
RBF_API int rbf_mlp_forward(rbf_mlp *net, const float *X, int64_t B, float *Y, void *stream);
/* Gradient of mean((Y - T)^2) with respect to the flattened parameters into
 * grad (device float[num_params]); *loss_host (may be NULL) gets the loss. */
RBF_API int rbf_mlp_gradient(rbf_mlp *net, const float *X, const float *T, int64_t B, float *grad,
                             float *loss_host, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that loss. */
RBF_API int rbf_mlp_train_step(rbf_mlp *net, const float *X, const float *T, int64_t B, float lr,
                               float *loss_host, void *stream);
RBF_API void rbf_mlp_free(rbf_mlp *net);
/* Checkpoint: write the network (sizes, FP32 parameters, Adam moments and step)
 * to `path` as a flat little-endian binary with the header "RBFMLP01"; load it
 * into a new network (*out; NULL on failure).  A loaded network continues
 * training exactly where the saved one stopped.  RBF_EINVAL on an unreadable,
 * truncated or foreign file.  Synchronise the device. */
RBF_API int rbf_mlp_save(const rbf_mlp *net, const char *path);
RBF_API int rbf_mlp_load(const char *path, rbf_mlp **out);

typedef struct {
    int n_train;      /* training centres, evenly spaced in Morton order */
    int epochs;
    int batch;
    float lr;         /* Adam step size */
    double delta_rel; /* regularisation of the local solves */
} rbf_train_opts;

typedef struct {
    float loss_first, loss_last; /* first and last mini-batch loss */
    int steps;
    double seconds;
} rbf_train_report;

/* Train `net` (shape 32 d -> 32) on this tree's centres: exact local cardinal
 * solves give targets c / max|c|; every step runs on the device.  Synchronises. */
RBF_API int rbf_precond_train(rbf_tree *t, rbf_kernel kernel, double eps, rbf_mlp *net,
                              const rbf_train_opts *opts, rbf_train_report *rep_host, void *stream);

/* Build P for this tree from the network (net != NULL) or from exact local
 * solves (net == NULL), then attach it: rbf_interp_solve uses it when
 * opts.precond == 1.  Synchronises. */
RBF_API int rbf_precond_build(rbf_tree *t, rbf_kernel kernel, double eps, rbf_mlp *net,
                              double delta_rel, void *stream);

/* z = P y (device FP64 vectors in the caller's order).  Synchronises. */
RBF_API int rbf_precond_apply(rbf_tree *t, const double *y, double *z, void *stream);

/* ---------------------------------------------------------------------------
 * Autotuning and batches of independent problems.
 * ------------------------------------------------------------------------- */

/* Largest |K(r) - Phi(r)| over 1024 sampled far offsets (w_D <= |r|_inf <= side,
 * w_D = side / 2^depth) for the given expansion parameters; K is the far
 * kernel of Eq. (35) built exactly as rbf_fmm_matvec builds it (FP64).  This
 * is the per-pair error that the scaled Lemma, Eq. (33), multiplies by
 * sum |lambda_j|.  Always the shared grid's kernel (params->grid is ignored).
 * Synchronises the device. */
RBF_API int rbf_kernel_error(rbf_kernel kernel, double eps, int d, const rbf_fmm_params *params,
                             double side, int depth, double *max_err_host);

/* Pick the tree depth (about 32 points per leaf for d >= 3, 64 for d <= 2,
 * depth >= 2), the period and taper (Gaussian: no taper, Phi(L - side) <
 * tol / 100; Wendland: no taper, L just above side + 1/eps so that the support
 * never wraps; inverse multiquadric and multiquadric: L = 4 side,
 * alpha = 4.5) and the smallest even M in [8, 64] whose measured far-kernel
 * error (rbf_kernel_error) is <= tol (64 when none is); M = 0 (no far field)
 * when max |Phi| over the far offsets of that depth is already <= tol.
 * *err_out (may be NULL) receives the achieved error. */
RBF_API int rbf_autotune(rbf_kernel kernel, double eps, int d, int64_t N, double side, double tol,
                         rbf_fmm_params *params_out, int *depth_out, double *err_out);

/* Unit costs of the FP32 products on the current GPU, in seconds, measured by
 * rbf_cost_calibrate: a pair of the batched direct sum (4 right-hand sides per
 * pair), a near-field pair of the FMM, a (point, mode) of P2M + L2P, a (leaf,
 * mode) of M2M + M2L (both per right-hand side), and what one FMM column costs
 * beyond its passes inside a CUDA graph (gathers, scatters, launch gaps). */
typedef struct {
    double direct_pair_s;
    double near_pair_s;
    double point_mode_s;
    double leaf_mode_s;
    double column_fixed_s;
} rbf_cost_model;

/* Measure the cost model on synthetic problems (64 direct sums of 8192 3-D
 * points; one 3-D FMM product of 65,536 points, M = 12, 4 columns, its passes
 * timed by CUDA events and its graph replay timed whole).  The result is also
 * kept as the current device's model for rbf_batch_create.  Synchronises;
 * allocates about 60 MB while it runs.  Takes a fraction of a second. */
RBF_API int rbf_cost_calibrate(rbf_cost_model *model_out, void *stream);

/* The cheapest way to apply A to nrhs columns of one problem under the cost
 * model, among: the direct sum of Eq. (1) (d <= 4; exact; *depth_out = 0,
 * params M = 0), the near field alone (M = 0, where |Phi| <= tol beyond one
 * leaf, Eq. (38) without its far part) at the autotuner's depth D or D - 1,
 * and the FMM with the autotuner's expansion order at D or D - 1 (the order is
 * searched only when the FMM's cheapest order, M = 8, could beat the best
 * candidate so far).  Near pairs and occupied leaves are estimated for
 * uniform points.  *err_out (may be NULL) gets the far-kernel error of the
 * choice (0 for the direct sum); *pred_s_out (may be NULL) its predicted
 * seconds per product. */
RBF_API int rbf_autotune_cost(rbf_kernel kernel, double eps, int d, int64_t N, int nrhs,
                              double side, double tol, const rbf_cost_model *model,
                              rbf_fmm_params *params_out, int *depth_out, double *err_out,
                              double *pred_s_out);

/* One problem of a batch: centres X (device [N][d] FP64, in [0,1]^d), kernel,
 * shape parameter, and the number of right-hand sides. */
typedef struct {
    const double *X;
    int64_t N;
    int d;
    rbf_kernel kernel;
    double eps;
    int nrhs;
} rbf_problem;

typedef struct rbf_batch rbf_batch;

/* How rbf_batch_create_opts picks each problem's product. */
#define RBF_BATCH_AUTO 0   /* rbf_autotune_cost: direct sum, near field alone or FMM */
#define RBF_BATCH_FMM 1    /* rbf_autotune for every problem (a tree each) */
#define RBF_BATCH_DIRECT 2 /* the direct sum for every problem with d <= 4 */
typedef struct {
    double tol_kernel;            /* far-kernel tolerance of the autotuner (> 0) */
    int choice;                   /* RBF_BATCH_* */
    const rbf_cost_model *model;  /* NULL: the current device's model, measured on first use */
} rbf_batch_opts;

/* Statistics of a batch: problems by product kind, the direct sum's work items,
 * kernel nodes of the product graph and of the GMRES step graph (0 until
 * built), wall time of the creation (autotuning, trees, coordinate records),
 * and the cost model's predicted milliseconds of one batch product. */
typedef struct {
    int n_direct, n_near_only, n_fmm;
    int direct_items;
    int product_nodes, step_nodes;
    double setup_s;
    double predicted_ms;
    rbf_cost_model model;
    double direct_pairs;  /* pair evaluations of the direct launch (N^2 per group of 4 columns) */
} rbf_batch_stats;

/* Choose every problem's product (opts->choice) and build what it needs: a
 * tree (root [0,1]^d) for FMM and near-field problems, 16-byte coordinate
 * records and a work list for the direct sums.  Vectors of a batch are packed:
 * problem p's right-hand side r occupies [off[p] + r N_p, off[p] + (r+1) N_p)
 * of a device array of `total` doubles (rbf_batch_layout).  The problem array
 * may be freed after the call; the centres must stay alive.  Synchronises. */
RBF_API int rbf_batch_create_opts(const rbf_problem *problems_host, int n_problems,
                                  const rbf_batch_opts *opts, void *stream, rbf_batch **out);
/* rbf_batch_create_opts with choice RBF_BATCH_AUTO and the device's model. */
RBF_API int rbf_batch_create(const rbf_problem *problems_host, int n_problems, double tol_kernel,
                             void *stream, rbf_batch **out);
/* Host arrays of n_problems entries (any may be NULL); depth 0 and M 0 mark a
 * problem summed directly (one leaf holding every centre: all pairs are near). */
RBF_API int rbf_batch_layout(const rbf_batch *b, int64_t *off_host, int *depth_host, int *M_host,
                             int64_t *total_host);
RBF_API int rbf_batch_get_stats(const rbf_batch *b, rbf_batch_stats *stats_out);
/* Device time of the two parts of a batch product, each run alone `reps` times
 * (after one run outside the timing) with CUDA events on `stream`: the direct
 * launch and the tree problems' products (enqueued over the batch's streams).
 * Either part may be empty (0 ms).  Writes the batch's product buffer;
 * synchronises. */
RBF_API int rbf_batch_time_parts(rbf_batch *b, rbf_precision prec, int reps, double *direct_ms_host,
                                 double *trees_ms_host, void *stream);
/* u = A lambda for every problem and right-hand side (packed device arrays).
 * The first call per precision runs the products once (allocating plans) and
 * captures them into one CUDA graph: the direct sums as one persistent launch
 * on `stream`, the other problems' products over several streams; every later
 * call is a copy into the batch's own buffer, one graph launch and a copy out.
 * Asynchronous after the first call. */
RBF_API int rbf_batch_matvec(rbf_batch *b, rbf_precision prec, const double *lambda_packed,
                             double *u_packed, void *stream);
/* Restarted GMRES(m) on every system (problem, right-hand side) in lockstep,
 * entirely on the device: one CUDA graph launch per step holds all products,
 * the two classical Gram-Schmidt passes (batched dot products and updates),
 * the norm, every system's Givens rotations and least-squares residual, and
 * v_{j+1}; the column index j lives in device memory, so one graph serves
 * every step.  A second graph per restart solves the triangular systems,
 * updates lambda and recomputes the true residual.  The host reads one flag
 * (any system active) per step.  u_packed, lambda_packed: device arrays laid
 * out like the batch buffers (lambda holds the initial guess).
 * rel_resid_host[n_systems] (may be NULL) gets ||u - A lambda|| / ||u|| per
 * system for the product in `prec` (the residual of the last restart);
 * *step_ms_host the mean device time of a step (CUDA events around each step
 * graph).  No iterative refinement in batch mode.  Allocates (m + 1) packed
 * vectors; synchronises. */
RBF_API int rbf_batch_solve(rbf_batch *b, const double *u_packed, double *lambda_packed,
                            int restart_m, int max_iters, double rtol, rbf_precision prec,
                            double *rel_resid_host, int *iters_host, double *step_ms_host,
                            void *stream);
RBF_API void rbf_batch_free(rbf_batch *b);

/* ---------------------------------------------------------------------------
 * Evaluation at new points: s(y) = sum_j lambda_j Phi(y - x_j) (Eq. (1) with
 * targets that are not centres, e.g. the interpolant after the solve).
 * ------------------------------------------------------------------------- */
typedef struct rbf_eval rbf_eval;

/* Prepare the evaluation of the centres of tree t at nt new points Y (device,
 * [nt][d] row-major FP64, copied; the tree is only read).  One tree over the
 * centres and the new points together is built with t's root cube and depth,
 * so the product runs the same passes (near field over neighbour leaves, far
 * field through the expansions) with zero coefficients on the new points.
 * Every point of Y must lie in t's root cube [lo, lo + side]^d (RBF_EINVAL
 * otherwise: the far-field approximation holds only inside it).  nt >= 1.
 * *out receives the handle (NULL on failure).  Synchronises `stream`. */
RBF_API int rbf_eval_create(const rbf_tree *t, const double *Y, int64_t nt, void *stream,
                            rbf_eval **out);

/* s = the FMM evaluation at the new points for nrhs coefficient columns.
 * lambda: device FP64, N x nrhs in t's original centre order, leading dimension
 * ld_lambda >= N; s: device FP64, nt x nrhs, leading dimension ld_s >= nt.
 * Kernel, eps, params and precision as in rbf_fmm_matvec.  Asynchronous. */
RBF_API int rbf_eval_apply(rbf_eval *e, rbf_kernel kernel, double eps, const rbf_fmm_params *params,
                           rbf_precision prec, const double *lambda, int64_t ld_lambda, double *s,
                           int64_t ld_s, int nrhs, void *stream);

/* Release an evaluation handle (not the source tree).  NULL is accepted. */
RBF_API void rbf_eval_free(rbf_eval *e);

/* Release a tree and everything it owns.  NULL is accepted. */
RBF_API void rbf_tree_free(rbf_tree *t);

/* Self-test of the failure path of the bounded device waits: one thread waits,
 * with the same try-wait loop and backoff as the tensor-core kernels, on an
 * mbarrier that nothing arrives on, and gives up after `seconds` (0 < seconds
 * <= 2) of SM clock.  *gave_up_host = 1 when the wait gave up (the expected
 * outcome); the device status bit it sets makes the next
 * rbf_check_device_waits return RBF_ETIMEOUT (and clear it).  No fault, no
 * hang: the kernel returns.  Synchronises `stream`. */
RBF_API int rbf_selftest_bounded_wait(double seconds, int *gave_up_host, void *stream);

/* Message for a status code, and the detail of the last failure on this thread. */
RBF_API const char *rbf_strerror(int code);
RBF_API const char *rbf_last_error(void);

/* Library version, "major.minor.patch". */
RBF_API const char *rbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBF_H */
