// rbf_internal.cuh -- internal types and helpers of the sm_103a library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/rbf.h"

// ---------------------------------------------------------------- errors --
void rbf_set_error(const char *fmt, ...);

#define RBF_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            rbf_set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
            return RBF_ECUDA;                                                               \
        }                                                                                   \
    } while (0)

#define RBF_LAUNCH_CHECK() RBF_CUDA_TRY(cudaGetLastError())

#define RBF_TRY(expr)               \
    do {                            \
        int _s = (expr);            \
        if (_s != RBF_OK) return _s; \
    } while (0)

#define RBF_REQUIRE(cond, ...)            \
    do {                                  \
        if (!(cond)) {                    \
            rbf_set_error(__VA_ARGS__);   \
            return RBF_EINVAL;            \
        }                                 \
    } while (0)

int rbf_malloc(void **p, size_t bytes);
template <typename T>
inline int rbf_alloc(T **p, size_t count)
{
    return rbf_malloc(reinterpret_cast<void **>(p), count * sizeof(T));
}
void rbf_free(void *p);

// --------------------------------------------------------------- complex --
template <typename R>
struct cplx_t;
template <>
struct cplx_t<float> {
    using type = float2;
};
template <>
struct cplx_t<double> {
    using type = double2;
};
template <typename R>
using cplx = typename cplx_t<R>::type;

template <typename C>
__device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// acc += a * b
template <typename C>
__device__ __forceinline__ void cmac(C &acc, C a, C b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
template <typename C>
__device__ __forceinline__ C cconj(C a)
{
    a.y = -a.y;
    return a;
}

// Phi at (eps r)^2 = e2r2 in FP64, any kernel (rbf_kernel)
__host__ __device__ inline double rbf_phi64(int kernel, double e2r2)
{
    if (kernel == RBF_GAUSSIAN) return exp(-e2r2);
    if (kernel == RBF_MQ) return sqrt(1.0 + e2r2);
    if (kernel == RBF_WENDLAND) {
        const double q = sqrt(e2r2), t = q < 1.0 ? 1.0 - q : 0.0;
        return t * t * t * (3.0 * q + 1.0);
    }
    return 1.0 / sqrt(1.0 + e2r2);
}

// FP32 Phi through the special-function unit's approximations (ex2, rsqrt) with
// denormals flushed: the reciprocal square root's argument is >= 1 and a flushed
// exponential is below 2^-126 of the largest term
#ifndef RBF_PHI_APPROX
#define RBF_PHI_APPROX 1
#endif
// Phi in the product's arithmetic, the kernel fixed at compile time, from
// s = c0 + |e (x_i - x_j)|^2 with the coordinates pre-scaled by e (e = eps, or
// eps sqrt(log2 e) for the FP32 Gaussian, which goes through exp2) and c0 = 1 for
// the multiquadric and its inverse, 0 otherwise: exp(-s), 1/sqrt(s), sqrt(s) or
// (1 - q)_+^3 (3 q + 1) with q = sqrt(s).  Folding eps^2 into the coordinates and
// the "1 +" into the sum saves an instruction per pair.
template <int KER>
__device__ __forceinline__ constexpr float phi_c0()
{
    return KER == RBF_IMQ || KER == RBF_MQ ? 1.0f : 0.0f;
}
template <int KER>
__device__ __forceinline__ float phi_s(float x)
{
#if RBF_PHI_APPROX
    if (KER == RBF_GAUSSIAN) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
        return y;
    }
    if (KER == RBF_IMQ) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
#endif
    if (KER == RBF_GAUSSIAN) return exp2f(-x);
    if (KER == RBF_IMQ) return rsqrtf(x);
    if (KER == RBF_MQ) return sqrtf(x);
    const float q = sqrtf(x);
    const float t = fmaxf(1.0f - q, 0.0f);
    return t * t * t * fmaf(3.0f, q, 1.0f);
}
template <int KER>
__device__ __forceinline__ double phi_s(double x)
{
    if (KER == RBF_GAUSSIAN) return exp(-x);
    if (KER == RBF_IMQ) return rsqrt(x);
    if (KER == RBF_MQ) return sqrt(x);
    const double q = sqrt(x);
    const double t = fmax(1.0 - q, 0.0);
    return t * t * t * fma(3.0, q, 1.0);
}

__device__ __forceinline__ void sincos_r(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double *s, double *c) { sincos(x, s, c); }

// ----------------------------------------------------------------- tree ---
struct rbf_level {
    int32_t nbox = 0;
    uint64_t *key = nullptr;       // [nbox] ascending Morton keys at this level
    int32_t *parent = nullptr;     // [nbox] compact id at level-1 (levels >= 1)
    int32_t *child_off = nullptr;  // [nbox+1] children range at level+1 (levels < D)
    int32_t *il_off = nullptr;     // [nbox+1] interaction lists (levels >= 2, lazy)
    int32_t *il_idx = nullptr;
    int64_t n_il = -1;
};

struct rbf_plan;  // expansion tables + workspace, one per precision

// Per-pass event timing (rbf_profile); events are recorded only while enabled.
struct rbf_prof {
    bool on = false;
    std::vector<cudaEvent_t> start[RBF_PASS_COUNT], stop[RBF_PASS_COUNT];
    int64_t launches[RBF_PASS_COUNT] = {0};
};

// learned / exact approximate-cardinal preconditioner P (sorted order)
struct rbf_precond_data {
    int32_t *nbr = nullptr;      // [N][RBF_KNN] sorted ids of the nearest centres, nearest first
    double *W = nullptr;         // [N][RBF_KNN] weights of column i on nbr[i][k]
    int32_t *row_off = nullptr;  // [N+1] rows of P: entries row_off[j] .. row_off[j+1]-1
    int32_t *ent = nullptr;      // [N*RBF_KNN] entry ids (i*RBF_KNN + k) by row, columns ascending
    bool ready = false;
    int kernel = -1;
    double eps = 0.0;
};

#ifndef RBF_PENCIL_Z
#define RBF_PENCIL_Z 8
#endif

struct rbf_tree {
    int64_t N = 0;
    int d = 0, D = 0;
    double lo[RBF_MAX_DIM] = {0};
    double side = 1.0;
    // sorted points
    uint64_t *keys = nullptr;   // [N]
    int32_t *perm = nullptr;    // [N] sorted -> original
    double *xs64 = nullptr;     // SoA [d][N]
    float *xs32 = nullptr;      // SoA [d][N]
    // leaves = level-D boxes
    int32_t *leaf_off = nullptr;    // [nleaf+1]
    int32_t *near_off = nullptr;    // [nleaf+1]
    int32_t *near_idx = nullptr;    // [n_near]
    int64_t n_near = 0;
    int32_t max_leaf = 0;
    int32_t *nb4 = nullptr;         // [nbox(D-1)][4^d] leaf ids around each parent (d <= 3)
    // pencils of the 3-D coupling (D >= 3): 2 x 2 x RBF_PENCIL_Z leaves each, the
    // leaf ids of the 4 x 4 neighbourhood of its planes z0 - 1 .. z0 + RBF_PENCIL_Z
    int32_t npz = 0;
    int4 *pz_seg = nullptr;         // [npz] (X, Y, Zs): leaves 2X..2X+1, 2Y..2Y+1, Zs Z ..
    int32_t *pz_nb = nullptr;       // [npz][(RBF_PENCIL_Z + 2) * 16]
    rbf_level lev[RBF_MAX_DEPTH + 1];
    rbf_plan *plan[2] = {nullptr, nullptr};  // indexed by rbf_precision
    rbf_prof prof;
    rbf_precond_data pc;
    // generic device scratch for solver/host-API copies
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int32_t nleaf() const { return lev[D].nbox; }
    const uint64_t *leaf_key() const { return lev[D].key; }
};

// Records a start event now and a stop event when it goes out of scope, when
// profiling is on; `launches` kernels are counted for the pass.
struct rbf_pass_timer {
    rbf_tree *t;
    int pass;
    cudaStream_t s;
    rbf_pass_timer(rbf_tree *t_, int pass_, cudaStream_t s_, int launches = 1);
    ~rbf_pass_timer();
};

// tree.cu
int rbf_scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_host,
                           cudaStream_t s);
int rbf_build_il(rbf_tree *t, int level, cudaStream_t s);
void rbf_prof_release(rbf_tree *t);
void rbf_precond_release(rbf_tree *t);
int rbf_precond_apply_sorted(const rbf_tree *t, const double *y, double *z, cudaStream_t s);

// --------------------------------------------------------------- plan -----
// Half-spectrum layout of an expansion: dimension 0 keeps k0 = 0..M/2,
// dimensions 1..d-1 keep k = -M/2..M/2.  The flattened mode index has
// dimension 0 slowest and dimension d-1 fastest:
//     m = ((k0 * n1 + k1') * n1 + k2') ...,  k_t' = k_t + M/2.
// A "row" is (k0, ..., k_{d-2}), a "column" is k_{d-1}.
struct rbf_plan {
    int prec = -1;
    int kernel = -1;
    double eps = 0, L = 0, alpha = 0;
    int M = 0, csample = -1;
    int n0 = 0, n1 = 0;        // values of k0, of k_t (t >= 1)
    int nrow = 0, ncol = 0;    // rows x cols = modes (ncol = n1, or n0 when d == 1)
    int64_t nmode = 0;
    int64_t mstride = 0;       // per-box stride of an expansion array (multiple of 4)
    void *omegaC = nullptr;    // [nmode] real: half-spectrum weight * omega * C
    void *xi = nullptr;        // [n1] real: xi_k, k = -M/2..M/2
    void *root_ph = nullptr;   // [d][2^D][n1] complex: e^{i xi_k (c_a,t - c_0,t)}
    void *shift_ph = nullptr;  // [D+1][n1] complex: e^{-i xi_k w_l / 2}, w_l = side / 2^l
                               // (the square of row D is the leaf-neighbour phase e^{-i xi_k w_D})
    void *V[RBF_MAX_DEPTH + 1] = {nullptr};  // expansions per level
    void *Lleaf = nullptr;     // local expansions at the leaves
    void *Vzero = nullptr;     // [mstride] zeros: the expansion of an absent box
    void *lam_s = nullptr;     // [N] gathered lambda
    void *u_near = nullptr;    // [N]
    void *u_far = nullptr;     // [N]
    size_t bytes = 0;
    // multi-right-hand-side workspace (FP32 plans only), grown on demand:
    // mr_G columns at a time, each with its own leaf and local expansions
    int mr_G = 0;
    float2 *mr_V = nullptr;    // [mr_G][nleaf][mstride]
    float2 *mr_L = nullptr;    // [mr_G][nleaf][mstride]
    float *mr_lam = nullptr;   // [mr_G][N]
    float *mr_un = nullptr;    // [mr_G][N]
    float *mr_uf = nullptr;    // [mr_G][N]
    float2 *mr_E = nullptr;    // [N][even_up(n0 + (d-1) n1)] point phase tables of P2M
    float *mr_Lt = nullptr;    // [N][16] coefficients of a group, point-major
    // nested (scale-invariant) grids of Sec. 4.1.1 (grid == RBF_GRID_NESTED), nested.cu
    int grid = RBF_GRID_SHARED;
    int lagK = 0, lagKT = 0;   // taps of the interpolation and of its transpose
    int p2m_shape = 0;         // FP32 P2M launch shape measured at creation (0: by rule)
    void *nest_wc[RBF_MAX_DEPTH + 1] = {nullptr};  // [nmode] omega_l C_l, levels 2..D
    void *nest_xi = nullptr;   // [n1] nodes of the leaf grid
    void *nest_ph = nullptr;   // [15][n1] complex translation phases (level independent)
    int32_t *lag_fidx = nullptr;  // [n1][lagK] child node of each tap (k + M/2)
    void *lag_fw = nullptr;       // [n1][lagK] interpolation weights
    int32_t *lag_tidx = nullptr;  // [n1][lagKT] parent node of each transposed tap
    void *lag_tw = nullptr;       // [n1][lagKT] transposed weights (0 in padding)
    int32_t *nest_nbr[RBF_MAX_DEPTH + 1] = {nullptr};  // [nbox_l][3^d] neighbours, levels 1..D-1
    int32_t *nest_nb4[RBF_MAX_DEPTH + 1] = {nullptr};  // [nbox_{l-1}][4^d] level-l boxes around
                                                       // each parent's children, levels 2..D
    void *nest_Vt[RBF_MAX_DEPTH + 1] = {nullptr};  // parents on their children's grid, 1..D-1
    void *nest_L[RBF_MAX_DEPTH + 1] = {nullptr};   // local expansions, levels 2..D-1 (D: Lleaf)
    void *nest_tmp[2] = {nullptr, nullptr};        // [nleaf][mstride] pass buffers
};

int rbf_plan_get(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *p, int prec,
                 cudaStream_t s, rbf_plan **out);
void rbf_plan_free(rbf_plan *p);
// omegaC of one grid (period L, taper flat on |t| <= R_in) into dst ([nmode], FP64 or FP32)
int rbf_make_omegaC(int prec, int d, int kernel, double eps, int M, double L, double alpha,
                    double R_in, int csample, int64_t nmode, void *dst, cudaStream_t s);
// nested grids (nested.cu): tables and per-level workspace; free; the far field
int rbf_nested_build(rbf_tree *t, rbf_plan *p, cudaStream_t s);
void rbf_nested_free(rbf_plan *p);
template <typename R>
int rbf_run_far_nested(rbf_tree *t, const rbf_plan *p, const R *lam_s, R *u_far, cudaStream_t s);

// Far-field and near-field passes (expansions.cu, p2p.cu)
template <typename R>
int rbf_run_p2p(rbf_tree *t, int kernel, double eps, const R *lam_s, R *u, cudaStream_t s);
template <typename R>
int rbf_run_far(rbf_tree *t, const rbf_plan *p, const R *lam_s, R *u_far, cudaStream_t s);
// FP32 near field of G <= 16 columns at once (lam_s, u: [G][N])
int rbf_run_p2p_multi(rbf_tree *t, int kernel, double eps, const float *lam_s, int G, float *u,
                      cudaStream_t s);
// P2M and L2P of one column on explicit leaf arrays (CUDA cores)
template <typename R>
int rbf_run_p2m(rbf_tree *t, const rbf_plan *p, const R *lam_s, cplx<R> *V, cudaStream_t s);
template <typename R>
int rbf_run_l2p(rbf_tree *t, const rbf_plan *p, const cplx<R> *L, R *u_far, cudaStream_t s);
// the translation passes on explicit leaf arrays (V[0..D-1] of the plan are scratch)
template <typename R>
int rbf_run_m2m(rbf_tree *t, const rbf_plan *p, const cplx<R> *VD, cudaStream_t s);
template <typename R>
int rbf_run_m2l(rbf_tree *t, const rbf_plan *p, const cplx<R> *VD, cplx<R> *L, cudaStream_t s);
// FP32 far field of G right-hand sides at once: P2M and L2P on the tensor cores
// (far_mrhs.cu); lam_s and u_far are [G][N], V and L are [G][nleaf][mstride]
int rbf_run_far_multi(rbf_tree *t, rbf_plan *p, const float *lam_s, int G, float2 *V, float2 *L,
                      float *u_far, cudaStream_t s);
// nonzero when the plan's columns per mode row fit a tensor-core tile
int rbf_far_multi_supported(const rbf_plan *p);
int rbf_tune_p2m_shape(rbf_tree *t, rbf_plan *p, cudaStream_t s);
// nonzero when a bounded device-side wait of a tensor-core kernel gave up
int rbf_tc_fetch_status(int *flags_host);

// Internal product on sorted-order device vectors (FP64 in/out, any arithmetic);
// used by the matvec entry point and the solver.
int rbf_matvec_sorted64(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *p,
                        int prec, const double *lam_sorted, double *u_sorted, cudaStream_t s);

void rbf_default_params(rbf_kernel kernel, double side, rbf_fmm_params *p);

// ------------------------------------------------- batched direct sums ---
// The problems of a batch whose plain sum (Eq. (1)) is cheaper than their FMM:
// one persistent launch over a work list of (problem, column group, target
// tile) items (batch_direct.cu).
struct rbf_direct_set {
    int np = 0;
    int nitems = 0, nitems64 = 0;  // FP32 items, then FP64 items (half-size tiles)
    int4 *items = nullptr;
    int *ctr = nullptr;            // [2] work-queue counters, zeroed before each launch
    int64_t *N = nullptr, *off = nullptr, *xoff = nullptr;  // per direct problem
    int *nrhs = nullptr, *ker = nullptr, *dim = nullptr;
    double *eps = nullptr;
    double *x64 = nullptr;         // [points][4] coordinates, zero-padded
    float4 *x32 = nullptr;
    int grid32 = 0, grid64 = 0;    // resident CTAs
};
int rbf_direct_set_build(rbf_direct_set *ds, const rbf_problem *probs, const int64_t *off,
                         const std::vector<int> &which, cudaStream_t s);
int rbf_direct_set_run(const rbf_direct_set *ds, int prec, const double *lam, double *u,
                       cudaStream_t s);
void rbf_direct_set_free(rbf_direct_set *ds);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
