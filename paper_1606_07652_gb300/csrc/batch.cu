// batch.cu -- many independent interpolation problems of uneven size at once,
// the autotuner that picks each problem's tree depth and expansion order, and
// the cost model that decides, per problem, between the plain sum of Eq. (1),
// the near field alone and the full FMM.
//
// Problems whose direct sum is cheapest are summed together by one persistent
// launch over a work list (batch_direct.cu); every other problem keeps its own
// tree and autotuned plan and runs its product on one of several streams.  One
// CUDA graph holds a whole GMRES step of all systems (problem, right-hand
// side): the products, the batched CGS2 reductions and updates, and the Givens
// rotations of every system's Hessenberg column, all on the device with the
// column index j in device memory, so the same graph is replayed for every
// step; a second graph holds the restart (back substitution, update of lambda,
// true residual).  The host reads one flag per step (any system active).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "rbf_internal.cuh"

namespace {

__host__ __device__ inline uint64_t mix64(uint64_t x)
{
    // SplitMix64 finaliser (Steele, Lea, Flood 2014)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

constexpr int KE_T = 256;  // threads per sample of the kernel-error evaluation

// |K(r) - Phi(r)| at sampled far offsets r (w <= |r|_inf <= side), with
// K(r) = Re sum_{half spectrum} omegaC e^{i xi.r}: one CTA per sample, its
// threads stride over the modes, a fixed-order tree reduction in shared memory.
__global__ void __launch_bounds__(KE_T) k_kernel_error(int d, int M, int64_t nmode, const double *xi,
                                                       const double *omegaC, int kernel, double eps,
                                                       double w, double side, uint64_t seed,
                                                       double *err)
{
    const int q = blockIdx.x;
    double r[RBF_MAX_DIM];
    double linf = 0.0, r2 = 0.0;
    for (int t = 0; t < d; ++t) {
        const uint64_t h = mix64(seed ^ ((uint64_t)q * 131 + t));
        r[t] = (2.0 * ((h >> 11) * (1.0 / 9007199254740992.0)) - 1.0) * side;
        linf = fmax(linf, fabs(r[t]));
    }
    // push the offset out of the near zone along its largest component; with no
    // far field (M = 0, K = 0) the first sample is the nearest far offset itself
    if (M == 0 && q == 0) {
        for (int t = 0; t < d; ++t) r[t] = t == 0 ? w : 0.0;
    } else if (linf < w) {
        int tm = 0;
        for (int t = 1; t < d; ++t)
            if (fabs(r[t]) > fabs(r[tm])) tm = t;
        r[tm] = r[tm] >= 0 ? w + (side - w) * 0.5 : -(w + (side - w) * 0.5);
    }
    for (int t = 0; t < d; ++t) r2 += r[t] * r[t];
    const int n1 = M + 1;
    double K = 0.0;
    for (int64_t m = threadIdx.x; m < nmode; m += KE_T) {
        int64_t rr = m;
        double ph = 0.0;
        for (int t = d - 1; t >= 1; --t) {
            ph += xi[rr % n1] * r[t];
            rr /= n1;
        }
        ph += xi[rr + M / 2] * r[0];
        K += omegaC[m] * cos(ph);
    }
    __shared__ double sh[KE_T];
    sh[threadIdx.x] = K;
    __syncthreads();
    for (int o = KE_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) err[q] = fabs(sh[0] - rbf_phi64(kernel, eps * eps * r2));
}

constexpr int BRED_T = 256;
constexpr int GM_BB = 8;  // blocks per (system, basis vector) in the reductions

// Device state of the lockstep batched GMRES(m): systems s = (problem,
// right-hand side) own the segments [soff[s], soff[s] + slen[s]) of the packed
// vectors; H is stored per system as [ks][m] (row k, column j).
struct Gm {
    int nsys, m, ks;
    int64_t total;
    const int64_t *soff, *slen;
    const int *sys_of;
    double *V;      // [(m + 1)][total] Krylov basis
    double *part;   // [nsys][ks][GM_BB] partial dot products
    double *hcur;   // [nsys][ks] this pass's projections
    double *hacc;   // [nsys][ks] both passes (the Hessenberg column)
    double *H;      // [nsys][ks][m]
    double *cs, *sn;  // [nsys][m] Givens rotations
    double *g;      // [nsys][ks] rotated right-hand side
    double *y;      // [nsys][ks] least-squares solution at restart
    double *beta, *bnorm, *scale;  // [nsys]
    int *act, *ny;  // [nsys] active flag, columns of the current cycle
    int *j;         // [1] current column
    int *any;       // [1] some system still active
    double rtol;
};

// part[s][k][b] = block b's share of V_k[s] . w[s] for k <= j (active systems);
// k = -1 (kk == 0 with self) takes w . w into slot 0
__global__ void k_gdots(const Gm g, const double *w, int self)
{
    const int s = blockIdx.z, k = blockIdx.y, b = blockIdx.x;
    const int jj = self ? 0 : *g.j;
    if (k > jj) return;
    __shared__ double sh[BRED_T];
    double acc = 0.0;
    if (g.act[s]) {
        const double *v = self ? w + g.soff[s] : g.V + (int64_t)k * g.total + g.soff[s];
        const double *x = w + g.soff[s];
        for (int64_t i = (int64_t)b * BRED_T + threadIdx.x; i < g.slen[s];
             i += (int64_t)GM_BB * BRED_T)
            acc = fma(v[i], x[i], acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = BRED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g.part[((int64_t)s * g.ks + k) * GM_BB + b] = sh[0];
}

// hcur[s][k] = sum_b part; hacc = hcur (pass 0) or hacc + hcur (pass 1)
__global__ void k_gdots_final(const Gm g, int pass)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)g.nsys * g.ks) return;
    const int k = (int)(q % g.ks);
    if (k > *g.j) return;
    double s = 0.0;
    for (int b = 0; b < GM_BB; ++b) s += g.part[q * GM_BB + b];
    g.hcur[q] = s;
    g.hacc[q] = pass ? g.hacc[q] + s : s;
}

// w -= sum_{k <= j} V_k hcur[s][k]  (active systems)
__global__ void k_gsub(const Gm g, double *w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.total) return;
    const int s = g.sys_of[i];
    if (!g.act[s]) return;
    const int jj = *g.j;
    double a = w[i];
    for (int k = 0; k <= jj; ++k) a = fma(-g.V[(int64_t)k * g.total + i], g.hcur[(int64_t)s * g.ks + k], a);
    w[i] = a;
}

// lam = V_j; clears the step's "any active" flag
__global__ void k_gcopy_vj(const Gm g, double *lam)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *g.any = 0;
    if (i < g.total) lam[i] = g.V[(int64_t)(*g.j) * g.total + i];
}

// one thread per system: the new Hessenberg column (hacc, ||w|| from part slot
// 0), the earlier rotations applied to it, a new rotation that zeroes its
// subdiagonal, the rotated right-hand side g and the residual estimate |g_{j+1}|
__global__ void k_givens(const Gm g)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.nsys) return;
    if (!g.act[q]) {
        g.scale[q] = 0.0;
        return;
    }
    const int j = *g.j, ks = g.ks, m = g.m;
    double wn = 0.0;
    for (int b = 0; b < GM_BB; ++b) wn += g.part[(int64_t)q * ks * GM_BB + b];
    const double hn = sqrt(fmax(wn, 0.0));
    double *h = g.hacc + (int64_t)q * ks;
    const double *c = g.cs + (int64_t)q * m, *sn = g.sn + (int64_t)q * m;
    double hk = h[0];
    for (int k = 0; k < j; ++k) {
        const double hk1 = h[k + 1];
        const double a = c[k] * hk + sn[k] * hk1;
        const double bb = -sn[k] * hk + c[k] * hk1;
        g.H[((int64_t)q * ks + k) * m + j] = a;
        hk = bb;
    }
    // h[j] is now hk, h[j+1] = hn
    const double den = hypot(hk, hn);
    const double cj = den > 0 ? hk / den : 1.0, sj = den > 0 ? hn / den : 0.0;
    g.cs[(int64_t)q * m + j] = cj;
    g.sn[(int64_t)q * m + j] = sj;
    g.H[((int64_t)q * ks + j) * m + j] = den;
    double *gq = g.g + (int64_t)q * ks;
    gq[j + 1] = -sj * gq[j];
    gq[j] = cj * gq[j];
    const double res = fabs(gq[j + 1]);
    g.ny[q] = j + 1;
    g.scale[q] = hn > 0 ? 1.0 / hn : 0.0;
    if (res <= g.rtol * g.bnorm[q] || hn == 0.0 || !(res == res)) g.act[q] = 0;
    else atomicOr(g.any, 1);
}

// V_{j+1} = w / ||w|| per system (zero for inactive systems)
__global__ void k_gnext(const Gm g, const double *w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.total) return;
    g.V[(int64_t)(*g.j + 1) * g.total + i] = g.scale[g.sys_of[i]] * w[i];
}

__global__ void k_ginc(const Gm g)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *g.j += 1;
}

// restart: y = R^{-1} g over the system's ny columns (back substitution)
__global__ void k_gtri(const Gm g)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.nsys) return;
    const int n = g.ny[q], ks = g.ks, m = g.m;
    const double *H = g.H + (int64_t)q * ks * m;
    const double *gq = g.g + (int64_t)q * ks;
    double *y = g.y + (int64_t)q * ks;
    for (int k = n - 1; k >= 0; --k) {
        double v = gq[k];
        for (int c = k + 1; c < n; ++c) v -= H[(int64_t)k * m + c] * y[c];
        const double dkk = H[(int64_t)k * m + k];
        y[k] = dkk != 0.0 ? v / dkk : 0.0;
    }
}

// x += sum_{k < ny[s]} V_k y[s][k]
__global__ void k_gadd(const Gm g, double *x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.total) return;
    const int s = g.sys_of[i];
    const int n = g.ny[s];
    double a = x[i];
    for (int k = 0; k < n; ++k) a = fma(g.V[(int64_t)k * g.total + i], g.y[(int64_t)s * g.ks + k], a);
    x[i] = a;
}

// V_0 = u - A x (the product output in au); resets j and the flag of the cycle
__global__ void k_gresid(const Gm g, const double *u, const double *au)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *g.j = 0;
        *g.any = 0;
    }
    if (i < g.total) g.V[i] = u[i] - au[i];
}

// every system active for a norm pass
__global__ void k_gactivate(const Gm g)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < g.nsys) g.act[q] = 1;
}

// ||u|| per system from part slot 0 (1 where u = 0)
__global__ void k_gbnorm(const Gm g)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.nsys) return;
    double s = 0.0;
    for (int b = 0; b < GM_BB; ++b) s += g.part[(int64_t)q * g.ks * GM_BB + b];
    const double n = sqrt(fmax(s, 0.0));
    g.bnorm[q] = n > 0 ? n : 1.0;
}

// start of a cycle: beta = ||r|| (part slot 0), g = beta e_1, active systems,
// scale = 1 / beta (j and the flag were reset by k_gresid)
__global__ void k_gstart(const Gm g)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.nsys) return;
    double s = 0.0;
    for (int b = 0; b < GM_BB; ++b) s += g.part[(int64_t)q * g.ks * GM_BB + b];
    const double beta = sqrt(fmax(s, 0.0));
    g.beta[q] = beta;
    double *gq = g.g + (int64_t)q * g.ks;
    for (int k = 0; k < g.ks; ++k) gq[k] = 0.0;
    gq[0] = beta;
    g.ny[q] = 0;
    const int a = beta > g.rtol * g.bnorm[q] && beta == beta && beta < INFINITY;
    g.act[q] = a;
    g.scale[q] = a ? 1.0 / beta : 0.0;
    if (a) atomicOr(g.any, 1);
}

// V_0 *= scale per system
__global__ void k_gscale0(const Gm g)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.total) g.V[i] *= g.scale[g.sys_of[i]];
}

}  // namespace

// ------------------------------------------------------------- autotuner ---
extern "C" int rbf_kernel_error(rbf_kernel kernel, double eps, int d, const rbf_fmm_params *p,
                                double side, int depth, double *max_err_host)
{
    RBF_REQUIRE(p && max_err_host, "rbf_kernel_error: NULL argument");
    RBF_REQUIRE(d >= 1 && d <= RBF_MAX_DIM && depth >= 1 && depth <= RBF_MAX_DEPTH && side > 0.0,
                "rbf_kernel_error: bad sizes");
    // a tree with no points: only its dimension, side and depth matter for the tables
    rbf_tree t;
    t.N = 0;
    t.d = d;
    t.D = depth;
    t.side = side;
    // the far kernel K of the shared grid
    rbf_fmm_params q = *p;
    q.grid = RBF_GRID_SHARED;
    rbf_plan *pl = nullptr;
    int st = rbf_plan_get(&t, kernel, eps, &q, RBF_FP64, 0, &pl);
    if (st != RBF_OK) {
        t.plan[0] = nullptr;
        return st;
    }
    const int ns = 1024;
    double *err = nullptr;
    st = rbf_alloc(&err, ns);
    if (st == RBF_OK) {
        const double w = side / (double)(1 << depth);
        k_kernel_error<<<ns, KE_T>>>(d, pl->M, pl->nmode, (const double *)pl->xi,
                                     (const double *)pl->omegaC, kernel, eps, w, side, 0x5EEDull,
                                     err);
        std::vector<double> h(ns);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(h.data(), err, ns * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rbf_set_error("rbf_kernel_error: CUDA failure");
            st = RBF_ECUDA;
        } else {
            *max_err_host = *std::max_element(h.begin(), h.end());
        }
    }
    rbf_free(err);
    rbf_plan_free(pl);
    t.plan[0] = nullptr;
    return st;
}

namespace {

// depth: about 32 points per leaf in 3-D and up, 64 in 1-D/2-D, at least 2 levels
int auto_depth(int d, int64_t N)
{
    const double per_leaf = d >= 3 ? 32.0 : 64.0;
    int D = (int)std::lround(std::log(std::max(1.0, (double)N / per_leaf)) / std::log((double)(1 << d)));
    D = std::max(2, std::min(D, RBF_MAX_DEPTH));
    while (d * D > 63) --D;
    return D;
}

// period and taper: the Gaussian needs Phi(L - side) below tol; the Wendland
// function needs its support 1/eps inside L - side; the (inverse) multiquadric a
// taper between side and L - side
rbf_fmm_params auto_period(rbf_kernel kernel, double eps, double side, double tol)
{
    rbf_fmm_params p{};
    p.csample = 1;
    if (kernel == RBF_GAUSSIAN) {
        p.window_alpha = 0.0;
        p.period_L = side + std::sqrt(std::max(0.0, -std::log(0.01 * tol))) / eps;
        p.period_L = std::max(p.period_L, 1.25 * side);
    } else if (kernel == RBF_WENDLAND) {
        p.window_alpha = 0.0;
        p.period_L = std::max(side + 1.0 / eps, 1.25 * side) * 1.0000001;
    } else {
        p.window_alpha = 4.5;
        p.period_L = 4.0 * side;
    }
    return p;
}

// the even M in [8, 64] at which the kernel's Fourier transform has decayed to
// tol at the band edge pi M / L (Gaussian: exp(-xi^2 / (4 eps^2)); inverse
// multiquadric: ~exp(-xi / eps); the Wendland function's transform decays only
// algebraically: 16)
int predicted_M(rbf_kernel kernel, double eps, double L, double tol)
{
    const double lt = std::log(1.0 / tol);
    const double pred = kernel == RBF_GAUSSIAN ? 2.0 * eps * L * std::sqrt(lt) / M_PI
                        : kernel == RBF_WENDLAND ? 16.0
                                                 : eps * L * lt / M_PI;
    const int M0 = 2 * (int)std::lround(pred / 2.0);
    return std::max(8, std::min(64, M0));
}

// expansion order at depth D: the smallest even M in [8, 64] whose measured
// far-kernel error meets tol (the error falls with M), else 64.  The search
// starts from predicted_M and steps by 2.
int search_M(rbf_kernel kernel, double eps, int d, int D, double side, double tol,
             rbf_fmm_params *p, int *M_out, double *err_out)
{
    auto error_at = [&](int M, double *e) -> int {
        p->M = M;
        return rbf_kernel_error(kernel, eps, d, p, side, D, e);
    };
    const int M0 = predicted_M(kernel, eps, p->period_L, tol);
    double err = INFINITY;
    RBF_TRY(error_at(M0, &err));
    int Mbest = M0;
    if (err <= tol) {
        while (Mbest > 8) {
            double e = INFINITY;
            RBF_TRY(error_at(Mbest - 2, &e));
            if (e > tol) break;
            Mbest -= 2;
            err = e;
        }
    } else {
        while (Mbest < 64 && err > tol) {
            Mbest += 2;
            RBF_TRY(error_at(Mbest, &err));
        }
    }
    p->M = Mbest;
    *M_out = Mbest;
    *err_out = err;
    return RBF_OK;
}

}  // namespace

extern "C" int rbf_autotune(rbf_kernel kernel, double eps, int d, int64_t N, double side, double tol,
                            rbf_fmm_params *out, int *depth_out, double *err_out)
{
    RBF_REQUIRE(out && depth_out, "rbf_autotune: NULL argument");
    RBF_REQUIRE(eps > 0.0 && side > 0.0 && tol > 0.0 && N >= 1 && d >= 1 && d <= RBF_MAX_DIM,
                "rbf_autotune: bad arguments");
    const int D = auto_depth(d, N);
    rbf_fmm_params p = auto_period(kernel, eps, side, tol);
    // no far field at all when the kernel is within tol beyond one leaf width
    // (K = 0 is then a far kernel within tol: narrow Gaussians, compact supports)
    double e0 = INFINITY;
    p.M = 0;
    RBF_TRY(rbf_kernel_error(kernel, eps, d, &p, side, D, &e0));
    if (e0 <= tol) {
        *out = p;
        *depth_out = D;
        if (err_out) *err_out = e0;
        return RBF_OK;
    }
    int M = 0;
    double err = INFINITY;
    RBF_TRY(search_M(kernel, eps, d, D, side, tol, &p, &M, &err));
    *out = p;
    *depth_out = D;
    if (err_out) *err_out = err;
    return RBF_OK;
}

// ------------------------------------------------------------ cost model ---
namespace {

// near pairs of N uniform points at depth D: a box of S = 2^D per dimension has
// (3 S - 2) / S neighbours per dimension on average (the faces have two)
double near_pairs_est(double N, int d, int D)
{
    const double S = std::ldexp(1.0, D);
    return N * N * std::pow(std::min(1.0, (3.0 * S - 2.0) / (S * S)), d);
}

// occupied leaves of N uniform points among 2^{dD}
double leaves_est(double N, int d, int D)
{
    const double B = std::ldexp(1.0, d * D);
    return B * (1.0 - std::exp(-N / B));
}

double nmode_of(int d, int M)
{
    return M == 0 ? 0.0 : (M / 2 + 1) * std::pow((double)(M + 1), d - 1);
}

double cost_direct(const rbf_cost_model &c, double N, int nrhs)
{
    return c.direct_pair_s * N * N * ((nrhs + 3) / 4);
}

double cost_fmm(const rbf_cost_model &c, double N, int d, int D, int M, int nrhs)
{
    const double t = c.near_pair_s * near_pairs_est(N, d, D) * std::max(1.0, nrhs / 4.0);
    if (M == 0) return t + c.column_fixed_s;
    const double nm = nmode_of(d, M);
    return t + nrhs * (c.point_mode_s * N * nm + c.leaf_mode_s * leaves_est(N, d, D) * nm +
                       c.column_fixed_s);
}

// seeded uniform points in [0,1)^d and N(0,1)-like coefficients (sum of
// uniforms), host side, for the calibration problems
void synth(uint64_t seed, int64_t n, int d, std::vector<double> &X)
{
    X.resize((size_t)n * d);
    for (int64_t i = 0; i < n * d; ++i)
        X[i] = (double)(mix64(seed * 0x100000001B3ull + (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
}

struct DevBuf {
    double *p = nullptr;
    ~DevBuf() { rbf_free(p); }
};

int calibrate(rbf_cost_model *c, cudaStream_t s)
{
    cudaEvent_t e0, e1;
    RBF_CUDA_TRY(cudaEventCreate(&e0));
    RBF_CUDA_TRY(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    // (1) the batched direct sum: 64 problems of 8192 points, 3-D, 4 columns
    {
        const int np = 64, d = 3, nr = 4;
        const int64_t n = 8192;
        std::vector<double> X;
        synth(11, n * np, d, X);
        DevBuf Xd, lam, u;
        RBF_TRY(rbf_alloc(&Xd.p, X.size()));
        RBF_TRY(rbf_alloc(&lam.p, (size_t)n * np * nr));
        RBF_TRY(rbf_alloc(&u.p, (size_t)n * np * nr));
        RBF_CUDA_TRY(cudaMemcpyAsync(Xd.p, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        std::vector<double> L;
        synth(12, n * np * nr, 1, L);
        RBF_CUDA_TRY(cudaMemcpyAsync(lam.p, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        std::vector<rbf_problem> pr(np);
        std::vector<int64_t> off(np);
        std::vector<int> which(np);
        for (int k = 0; k < np; ++k) {
            pr[k] = rbf_problem{Xd.p + (size_t)k * n * d, n, d, RBF_IMQ, 2.0, nr};
            off[k] = (int64_t)k * n * nr;
            which[k] = k;
        }
        rbf_direct_set ds;
        int st = rbf_direct_set_build(&ds, pr.data(), off.data(), which, s);
        float ms = 0.f;
        if (st == RBF_OK) st = rbf_direct_set_run(&ds, RBF_FP32, lam.p, u.p, s);
        if (st == RBF_OK && cudaEventRecord(e0, s) != cudaSuccess) st = RBF_ECUDA;
        for (int r = 0; r < 3 && st == RBF_OK; ++r) st = rbf_direct_set_run(&ds, RBF_FP32, lam.p, u.p, s);
        if (st == RBF_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = RBF_ECUDA;
        rbf_direct_set_free(&ds);
        if (st != RBF_OK) return st;
        c->direct_pair_s = ms * 1e-3 / 3.0 / ((double)np * n * n);
    }
    // (2) one FMM product: 65,536 points, 3-D, IMQ eps = 2, M = 12, 4 columns
    {
        const int d = 3, nr = 4, M = 12;
        const int64_t n = 65536;
        const int D = auto_depth(d, n);
        std::vector<double> X, L;
        synth(13, n, d, X);
        synth(14, n * nr, 1, L);
        DevBuf Xd, lam, u;
        RBF_TRY(rbf_alloc(&Xd.p, X.size()));
        RBF_TRY(rbf_alloc(&lam.p, (size_t)n * nr));
        RBF_TRY(rbf_alloc(&u.p, (size_t)n * nr));
        RBF_CUDA_TRY(cudaMemcpyAsync(Xd.p, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        RBF_CUDA_TRY(cudaMemcpyAsync(lam.p, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        const double lo[3] = {0.0, 0.0, 0.0};
        rbf_tree *t = nullptr;
        RBF_TRY(rbf_tree_build(Xd.p, n, d, lo, 1.0, D, s, &t));
        rbf_fmm_params p = auto_period(RBF_IMQ, 2.0, 1.0, 1e-6);
        p.M = M;
        auto prod = [&](cudaStream_t q) {
            return rbf_fmm_matvec(t, RBF_IMQ, 2.0, &p, RBF_FP32, lam.p, n, u.p, n, nr, q);
        };
        int st = prod(s);  // plans and workspace
        double pass[RBF_PASS_COUNT] = {0};
        int64_t nl[RBF_PASS_COUNT] = {0};
        const int runs = 2;
        if (st == RBF_OK) st = rbf_profile(t, 1);
        for (int r = 0; r < runs && st == RBF_OK; ++r) st = prod(s);
        if (st == RBF_OK) st = rbf_profile_read(t, pass, nl);
        if (st == RBF_OK) st = rbf_profile(t, 0);
        // the same product captured in a graph, as the batch runs it
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        float ms = 0.f;
        if (st == RBF_OK) {
            cudaStream_t cs;
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
                st = RBF_ECUDA;
            } else {
                if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = RBF_ECUDA;
                else {
                    st = prod(cs);
                    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && st == RBF_OK) st = RBF_ECUDA;
                }
                cudaStreamDestroy(cs);
            }
        }
        if (st == RBF_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = RBF_ECUDA;
        if (st == RBF_OK && cudaGraphLaunch(ge, s) != cudaSuccess) st = RBF_ECUDA;
        if (st == RBF_OK && cudaEventRecord(e0, s) != cudaSuccess) st = RBF_ECUDA;
        for (int r = 0; r < 3 && st == RBF_OK; ++r)
            if (cudaGraphLaunch(ge, s) != cudaSuccess) st = RBF_ECUDA;
        if (st == RBF_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = RBF_ECUDA;
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        rbf_tree_free(t);
        if (st != RBF_OK) return st;
        const double nm = nmode_of(d, M), nd = (double)n;
        const double sec = 1e-3 / runs;
        c->near_pair_s = pass[RBF_PASS_P2P] * sec / near_pairs_est(nd, d, D);
        c->point_mode_s = (pass[RBF_PASS_P2M] + pass[RBF_PASS_L2P]) * sec / (nd * nm * nr);
        c->leaf_mode_s = (pass[RBF_PASS_M2M] + pass[RBF_PASS_M2L]) * sec / (leaves_est(nd, d, D) * nm * nr);
        double passes = 0.0;
        for (int k = 0; k < RBF_PASS_COUNT; ++k)
            if (k != RBF_PASS_PERM) passes += pass[k] * sec;
        const double tg = ms * 1e-3 / 3.0;
        // what the graph spends beyond the passes' own work: gathers, scatters,
        // launch gaps; at least 4 microseconds per column
        c->column_fixed_s = std::max(4e-6, (tg - passes) / nr);
    }
    return RBF_OK;
}

rbf_cost_model g_model[64];
bool g_model_ok[64] = {false};

}  // namespace

extern "C" int rbf_cost_calibrate(rbf_cost_model *out, void *stream)
{
    RBF_REQUIRE(out != nullptr, "rbf_cost_calibrate: NULL argument");
    rbf_cost_model c{};
    RBF_TRY(calibrate(&c, (cudaStream_t)stream));
    int dev = 0;
    RBF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64) {
        g_model[dev] = c;
        g_model_ok[dev] = true;
    }
    *out = c;
    return RBF_OK;
}

// the model of the current device, measured on first use
static int current_model(rbf_cost_model *out, cudaStream_t s)
{
    int dev = 0;
    RBF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && g_model_ok[dev]) {
        *out = g_model[dev];
        return RBF_OK;
    }
    return rbf_cost_calibrate(out, s);
}

extern "C" int rbf_autotune_cost(rbf_kernel kernel, double eps, int d, int64_t N, int nrhs,
                                 double side, double tol, const rbf_cost_model *model,
                                 rbf_fmm_params *params_out, int *depth_out, double *err_out,
                                 double *pred_s_out)
{
    RBF_REQUIRE(model && params_out && depth_out, "rbf_autotune_cost: NULL argument");
    RBF_REQUIRE(eps > 0.0 && side > 0.0 && tol > 0.0 && N >= 1 && d >= 1 && d <= RBF_MAX_DIM &&
                    nrhs >= 1,
                "rbf_autotune_cost: bad arguments");
    const rbf_cost_model &c = *model;
    const double n = (double)N;
    const int Dr = auto_depth(d, N);
    rbf_fmm_params p = auto_period(kernel, eps, side, tol);
    bool have = false;
    double best = INFINITY, besterr = 0.0;
    int bestD = 0, bestM = 0;
    // the direct sum: exact, one batched launch (d <= 4)
    if (d <= 4) {
        best = cost_direct(c, n, nrhs);
        have = true;
    }
    const int cand[2] = {Dr - 1, Dr};
    // the near field alone, where the kernel is within tol beyond one leaf
    for (int D : cand) {
        if (D < 2) continue;
        const double t = cost_fmm(c, n, d, D, 0, nrhs);
        if (have && t >= best) continue;
        double e = INFINITY;
        p.M = 0;
        RBF_TRY(rbf_kernel_error(kernel, eps, d, &p, side, D, &e));
        if (e <= tol) {
            best = t;
            bestD = D;
            bestM = 0;
            besterr = e;
            have = true;
        }
    }
    // the FMM, searched only if it could win at an order 10 below the predicted
    // one (the measured order has always been within a few of the prediction);
    // the order found at Dr also meets tol at Dr - 1 (its far offsets are a subset)
    const int Mlb = std::max(8, predicted_M(kernel, eps, p.period_L, tol) - 10);
    double lb = INFINITY;
    for (int D : cand)
        if (D >= 2) lb = std::min(lb, cost_fmm(c, n, d, D, Mlb, nrhs));
    if (!have || lb < best) {
        int M = 0;
        double e = INFINITY;
        RBF_TRY(search_M(kernel, eps, d, Dr, side, tol, &p, &M, &e));
        if (e <= tol || !have) {
            for (int D : cand) {
                if (D < 2) continue;
                const double t = cost_fmm(c, n, d, D, M, nrhs);
                if (!have || t < best) {
                    best = t;
                    bestD = D;
                    bestM = M;
                    besterr = e;
                    have = true;
                }
            }
        }
    }
    p.M = bestM;
    *params_out = p;
    *depth_out = bestD;
    if (err_out) *err_out = besterr;
    if (pred_s_out) *pred_s_out = best;
    return RBF_OK;
}

// ---------------------------------------------------------------- batches ---
struct rbf_batch {
    int np = 0;
    std::vector<rbf_problem> probs;
    std::vector<rbf_tree *> trees;  // nullptr for the problems summed directly
    std::vector<rbf_fmm_params> params;
    std::vector<int> depth;         // 0: direct sum
    std::vector<int64_t> off;       // packed offset of problem p (all its right-hand sides)
    std::vector<int> tree_probs;    // problems with a tree (FMM or near field alone)
    int64_t total = 0;
    double *lam = nullptr, *u = nullptr;  // packed product buffers
    rbf_direct_set direct;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_prec = -1;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    rbf_batch_stats stats{};
};

static void batch_release(rbf_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->events) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto t : b->trees)
        if (t) rbf_tree_free(t);
    rbf_direct_set_free(&b->direct);
    rbf_free(b->lam);
    rbf_free(b->u);
    delete b;
}

extern "C" void rbf_batch_free(rbf_batch *b)
{
    if (b) batch_release(b);
}

static int kernel_nodes(cudaGraph_t g, int *out)
{
    size_t n = 0;
    RBF_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) RBF_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &n));
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        RBF_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
        if (ty == cudaGraphNodeTypeKernel) ++k;
    }
    *out = k;
    return RBF_OK;
}

extern "C" int rbf_batch_create_opts(const rbf_problem *probs, int np, const rbf_batch_opts *opts,
                                     void *stream, rbf_batch **out)
{
    RBF_REQUIRE(out && probs && opts && np >= 1, "rbf_batch_create: bad arguments");
    RBF_REQUIRE(opts->tol_kernel > 0.0, "rbf_batch_create: tol_kernel must be > 0");
    RBF_REQUIRE(opts->choice >= RBF_BATCH_AUTO && opts->choice <= RBF_BATCH_DIRECT,
                "rbf_batch_create: unknown choice %d", opts->choice);
    *out = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    for (int p = 0; p < np; ++p) {
        const rbf_problem &q = probs[p];
        RBF_REQUIRE(q.X && q.N >= 1 && q.d >= 1 && q.d <= RBF_MAX_DIM && q.nrhs >= 1 && q.eps > 0.0 &&
                        q.kernel >= RBF_GAUSSIAN && q.kernel <= RBF_WENDLAND,
                    "rbf_batch_create: problem %d is malformed", p);
    }
    rbf_cost_model model{};
    bool have_model = false;
    if (opts->model) {
        model = *opts->model;
        have_model = true;
    } else if (opts->choice == RBF_BATCH_AUTO) {
        RBF_TRY(current_model(&model, s));
        have_model = true;
    }
    rbf_batch *b = new rbf_batch();
    b->np = np;
    b->probs.assign(probs, probs + np);
    b->stats.model = model;
    std::vector<int> direct;
    int st = RBF_OK;
    for (int p = 0; p < np && st == RBF_OK; ++p) {
        const rbf_problem &q = probs[p];
        rbf_fmm_params prm{};
        int D = 0;
        double err = 0.0, pred = 0.0;
        if (opts->choice == RBF_BATCH_DIRECT && q.d <= 4) {
            D = 0;
            if (have_model) pred = cost_direct(model, (double)q.N, q.nrhs);
        } else if (opts->choice == RBF_BATCH_AUTO) {
            st = rbf_autotune_cost(q.kernel, q.eps, q.d, q.N, q.nrhs, 1.0, opts->tol_kernel, &model,
                                   &prm, &D, &err, &pred);
        } else {
            st = rbf_autotune(q.kernel, q.eps, q.d, q.N, 1.0, opts->tol_kernel, &prm, &D, &err);
            if (st == RBF_OK && have_model) pred = cost_fmm(model, (double)q.N, q.d, D, prm.M, q.nrhs);
        }
        if (st != RBF_OK) break;
        rbf_tree *t = nullptr;
        if (D == 0) {
            direct.push_back(p);
            ++b->stats.n_direct;
            b->stats.direct_pairs += (double)q.N * (double)q.N * ((q.nrhs + 3) / 4);
        } else {
            std::vector<double> lo(q.d, 0.0);
            st = rbf_tree_build(q.X, q.N, q.d, lo.data(), 1.0, D, stream, &t);
            if (st != RBF_OK) break;
            b->tree_probs.push_back(p);
            if (prm.M == 0) ++b->stats.n_near_only;
            else ++b->stats.n_fmm;
        }
        b->trees.push_back(t);
        b->params.push_back(prm);
        b->depth.push_back(D);
        b->off.push_back(b->total);
        b->total += q.N * q.nrhs;
        b->stats.predicted_ms += pred * 1e3;
    }
    if (st == RBF_OK) st = rbf_alloc(&b->lam, std::max<int64_t>(b->total, 1));
    if (st == RBF_OK) st = rbf_alloc(&b->u, std::max<int64_t>(b->total, 1));
    if (st == RBF_OK && cudaMemsetAsync(b->lam, 0, b->total * sizeof(double), s) != cudaSuccess)
        st = RBF_ECUDA;
    if (st == RBF_OK) st = rbf_direct_set_build(&b->direct, probs, b->off.data(), direct, s);
    b->stats.direct_items = b->direct.nitems;
    if (st == RBF_OK) {
        const int ns = std::min((int)b->tree_probs.size(), 16);
        for (int q = 0; q < ns && st == RBF_OK; ++q) {
            cudaStream_t sq;
            if (cudaStreamCreateWithFlags(&sq, cudaStreamNonBlocking) != cudaSuccess) st = RBF_ECUDA;
            else b->streams.push_back(sq);
        }
        for (int q = 0; q < ns + 1 && st == RBF_OK; ++q) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = RBF_ECUDA;
            else b->events.push_back(e);
        }
    }
    if (st == RBF_OK && cudaStreamSynchronize(s) != cudaSuccess) st = RBF_ECUDA;
    if (st != RBF_OK) {
        batch_release(b);
        return st;
    }
    b->stats.setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = b;
    return RBF_OK;
}

extern "C" int rbf_batch_create(const rbf_problem *probs, int np, double tol_kernel, void *stream,
                                rbf_batch **out)
{
    rbf_batch_opts o{};
    o.tol_kernel = tol_kernel;
    o.choice = RBF_BATCH_AUTO;
    o.model = nullptr;
    return rbf_batch_create_opts(probs, np, &o, stream, out);
}

extern "C" int rbf_batch_layout(const rbf_batch *b, int64_t *off_host, int *depth_host, int *M_host,
                                int64_t *total_host)
{
    RBF_REQUIRE(b != nullptr, "rbf_batch_layout: batch is NULL");
    for (int p = 0; p < b->np; ++p) {
        if (off_host) off_host[p] = b->off[p];
        if (depth_host) depth_host[p] = b->depth[p];
        if (M_host) M_host[p] = b->params[p].M;
    }
    if (total_host) *total_host = b->total;
    return RBF_OK;
}

extern "C" int rbf_batch_get_stats(const rbf_batch *b, rbf_batch_stats *out)
{
    RBF_REQUIRE(b && out, "rbf_batch_get_stats: NULL argument");
    *out = b->stats;
    return RBF_OK;
}

// all products: the direct sums in one persistent launch on s, the other
// problems one stream per slot, in the order they are enqueued
static int batch_enqueue(rbf_batch *b, int prec, cudaStream_t s)
{
    const int ns = (int)b->streams.size();
    if (ns > 0) {
        RBF_CUDA_TRY(cudaEventRecord(b->events[ns], s));
        for (int q = 0; q < ns; ++q) RBF_CUDA_TRY(cudaStreamWaitEvent(b->streams[q], b->events[ns], 0));
    }
    RBF_TRY(rbf_direct_set_run(&b->direct, prec, b->lam, b->u, s));
    for (size_t k = 0; k < b->tree_probs.size(); ++k) {
        const int p = b->tree_probs[k];
        const rbf_problem &q = b->probs[p];
        cudaStream_t sq = b->streams[k % ns];
        RBF_TRY(rbf_fmm_matvec(b->trees[p], q.kernel, q.eps, &b->params[p], (rbf_precision)prec,
                               b->lam + b->off[p], q.N, b->u + b->off[p], q.N, q.nrhs, sq));
    }
    for (int q = 0; q < ns; ++q) {
        RBF_CUDA_TRY(cudaEventRecord(b->events[q], b->streams[q]));
        RBF_CUDA_TRY(cudaStreamWaitEvent(s, b->events[q], 0));
    }
    return RBF_OK;
}

extern "C" int rbf_batch_time_parts(rbf_batch *b, rbf_precision prec, int reps, double *direct_ms,
                                    double *trees_ms, void *stream)
{
    RBF_REQUIRE(b && direct_ms && trees_ms && reps >= 1, "rbf_batch_time_parts: bad arguments");
    RBF_REQUIRE(prec == RBF_FP32 || prec == RBF_FP64, "rbf_batch_time_parts: precision");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    RBF_CUDA_TRY(cudaEventCreate(&e0));
    RBF_CUDA_TRY(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    // the tree problems alone: the direct set hidden for the duration
    rbf_direct_set saved = b->direct;
    b->direct.np = 0;
    auto trees = [&]() { return batch_enqueue(b, prec, s); };
    int st = trees();
    float ms = 0.f;
    if (st == RBF_OK && cudaEventRecord(e0, s) != cudaSuccess) st = RBF_ECUDA;
    for (int r = 0; r < reps && st == RBF_OK; ++r) st = trees();
    if (st == RBF_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = RBF_ECUDA;
    b->direct = saved;
    RBF_TRY(st);
    *trees_ms = b->tree_probs.empty() ? 0.0 : (double)ms / reps;
    RBF_TRY(rbf_direct_set_run(&b->direct, prec, b->lam, b->u, s));
    RBF_CUDA_TRY(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) RBF_TRY(rbf_direct_set_run(&b->direct, prec, b->lam, b->u, s));
    RBF_CUDA_TRY(cudaEventRecord(e1, s));
    RBF_CUDA_TRY(cudaEventSynchronize(e1));
    RBF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *direct_ms = b->direct.np == 0 ? 0.0 : (double)ms / reps;
    return RBF_OK;
}

// capture fn(cs) into a graph and instantiate it
template <typename F>
static int capture(F fn, cudaGraph_t *g_out, cudaGraphExec_t *e_out)
{
    cudaStream_t cs;
    RBF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const cudaError_t eb = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (eb != cudaSuccess) cudaStreamDestroy(cs);
    RBF_CUDA_TRY(eb);
    const int st = fn(cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != RBF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    RBF_CUDA_TRY(e);
    const cudaError_t ei = cudaGraphInstantiate(e_out, g, 0);
    if (ei != cudaSuccess) cudaGraphDestroy(g);
    RBF_CUDA_TRY(ei);
    *g_out = g;
    return RBF_OK;
}

// u = A lambda for every problem and right-hand side, on the packed buffers
static int batch_matvec(rbf_batch *b, int prec, cudaStream_t s)
{
    if (!b->exec || b->graph_prec != prec) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        // warm-up outside capture: plans and workspace are allocated here
        RBF_TRY(batch_enqueue(b, prec, s));
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        RBF_TRY(capture([&](cudaStream_t cs) { return batch_enqueue(b, prec, cs); }, &b->graph,
                        &b->exec));
        b->graph_prec = prec;
        RBF_TRY(kernel_nodes(b->graph, &b->stats.product_nodes));
    }
    RBF_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    return RBF_OK;
}

extern "C" int rbf_batch_matvec(rbf_batch *b, rbf_precision prec, const double *lambda_packed,
                                double *u_packed, void *stream)
{
    RBF_REQUIRE(b && lambda_packed && u_packed, "rbf_batch_matvec: NULL argument");
    RBF_REQUIRE(prec == RBF_FP32 || prec == RBF_FP64, "rbf_batch_matvec: precision");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_CUDA_TRY(cudaMemcpyAsync(b->lam, lambda_packed, b->total * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
    RBF_TRY(batch_matvec(b, prec, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(u_packed, b->u, b->total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return RBF_OK;
}

// device buffers of one batched solve, freed on every path
struct GmBufs {
    std::vector<void *> ptrs;
    int *pinned = nullptr;
    cudaGraph_t gs = nullptr, gr = nullptr;
    cudaGraphExec_t es = nullptr, er = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    template <typename T>
    int get(T **p, size_t n)
    {
        RBF_TRY(rbf_alloc(p, std::max<size_t>(n, 1)));
        ptrs.push_back(*p);
        return RBF_OK;
    }
    ~GmBufs()
    {
        if (es) cudaGraphExecDestroy(es);
        if (er) cudaGraphExecDestroy(er);
        if (gs) cudaGraphDestroy(gs);
        if (gr) cudaGraphDestroy(gr);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (pinned) cudaFreeHost(pinned);
        for (void *p : ptrs) rbf_free(p);
    }
};

extern "C" int rbf_batch_solve(rbf_batch *b, const double *u_packed, double *lam_packed,
                               int restart_m, int max_iters, double rtol, rbf_precision prec,
                               double *rel_resid_host, int *iters_host, double *step_ms_host,
                               void *stream)
{
    RBF_REQUIRE(b && u_packed && lam_packed, "rbf_batch_solve: NULL argument");
    RBF_REQUIRE(restart_m >= 1 && restart_m <= 200 && max_iters >= 1 && rtol > 0.0,
                "rbf_batch_solve: bad options");
    RBF_REQUIRE(prec == RBF_FP32 || prec == RBF_FP64, "rbf_batch_solve: precision");
    cudaStream_t s = (cudaStream_t)stream;
    // systems: (problem, right-hand side)
    std::vector<int64_t> soff, slen;
    for (int p = 0; p < b->np; ++p)
        for (int r = 0; r < b->probs[p].nrhs; ++r) {
            soff.push_back(b->off[p] + (int64_t)r * b->probs[p].N);
            slen.push_back(b->probs[p].N);
        }
    const int nsys = (int)soff.size();
    RBF_REQUIRE(nsys <= 65535, "rbf_batch_solve: %d systems, at most 65535", nsys);
    const int64_t total = b->total;
    std::vector<int> sys_of(total);
    for (int q = 0; q < nsys; ++q)
        for (int64_t i = 0; i < slen[q]; ++i) sys_of[soff[q] + i] = q;
    GmBufs B;
    Gm g{};
    g.nsys = nsys;
    g.m = restart_m;
    g.ks = restart_m + 1;
    g.total = total;
    g.rtol = rtol;
    int64_t *doff = nullptr, *dlen = nullptr;
    int *dsys = nullptr;
    RBF_TRY(B.get(&doff, nsys));
    RBF_TRY(B.get(&dlen, nsys));
    RBF_TRY(B.get(&dsys, total));
    g.soff = doff;
    g.slen = dlen;
    g.sys_of = dsys;
    RBF_TRY(B.get(&g.V, (size_t)g.ks * total));
    RBF_TRY(B.get(&g.part, (size_t)nsys * g.ks * GM_BB));
    RBF_TRY(B.get(&g.hcur, (size_t)nsys * g.ks));
    RBF_TRY(B.get(&g.hacc, (size_t)nsys * g.ks));
    RBF_TRY(B.get(&g.H, (size_t)nsys * g.ks * g.m));
    RBF_TRY(B.get(&g.cs, (size_t)nsys * g.m));
    RBF_TRY(B.get(&g.sn, (size_t)nsys * g.m));
    RBF_TRY(B.get(&g.g, (size_t)nsys * g.ks));
    RBF_TRY(B.get(&g.y, (size_t)nsys * g.ks));
    RBF_TRY(B.get(&g.beta, nsys));
    RBF_TRY(B.get(&g.bnorm, nsys));
    RBF_TRY(B.get(&g.scale, nsys));
    RBF_TRY(B.get(&g.act, nsys));
    RBF_TRY(B.get(&g.ny, nsys));
    RBF_TRY(B.get(&g.j, 1));
    RBF_TRY(B.get(&g.any, 1));
    RBF_CUDA_TRY(cudaMallocHost(&B.pinned, sizeof(int)));
    RBF_CUDA_TRY(cudaEventCreate(&B.e0));
    RBF_CUDA_TRY(cudaEventCreate(&B.e1));
    RBF_CUDA_TRY(cudaMemcpyAsync(doff, soff.data(), nsys * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(dlen, slen.data(), nsys * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(dsys, sys_of.data(), total * sizeof(int), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemsetAsync(g.ny, 0, nsys * sizeof(int), s));
    RBF_CUDA_TRY(cudaMemsetAsync(g.j, 0, sizeof(int), s));
    RBF_CUDA_TRY(cudaMemsetAsync(g.H, 0, (size_t)nsys * g.ks * g.m * sizeof(double), s));
    const int gb = ceil_div(total, 256), gs = ceil_div(nsys, 128);
    const int gk = ceil_div((int64_t)nsys * g.ks, 256);
    // plans and workspace of every product exist before any capture
    RBF_TRY(batch_matvec(b, prec, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    // one GMRES step of every system: w = A v_j, two CGS passes, ||w||, the
    // Givens update, v_{j+1} = w / ||w||, j += 1
    RBF_TRY(capture(
        [&](cudaStream_t cs) -> int {
            k_gcopy_vj<<<gb, 256, 0, cs>>>(g, b->lam);
            RBF_LAUNCH_CHECK();
            RBF_TRY(batch_enqueue(b, prec, cs));
            for (int pass = 0; pass < 2; ++pass) {
                k_gdots<<<dim3(GM_BB, g.m, nsys), BRED_T, 0, cs>>>(g, b->u, 0);
                RBF_LAUNCH_CHECK();
                k_gdots_final<<<gk, 256, 0, cs>>>(g, pass);
                RBF_LAUNCH_CHECK();
                k_gsub<<<gb, 256, 0, cs>>>(g, b->u);
                RBF_LAUNCH_CHECK();
            }
            k_gdots<<<dim3(GM_BB, 1, nsys), BRED_T, 0, cs>>>(g, b->u, 1);
            RBF_LAUNCH_CHECK();
            k_givens<<<gs, 128, 0, cs>>>(g);
            RBF_LAUNCH_CHECK();
            k_gnext<<<gb, 256, 0, cs>>>(g, b->u);
            RBF_LAUNCH_CHECK();
            k_ginc<<<1, 32, 0, cs>>>(g);
            RBF_LAUNCH_CHECK();
            return RBF_OK;
        },
        &B.gs, &B.es));
    RBF_TRY(kernel_nodes(B.gs, &b->stats.step_nodes));
    // restart: lambda += V y, V_0 = u - A lambda, beta, g = beta e_1, v_0 = r / beta
    RBF_TRY(capture(
        [&](cudaStream_t cs) -> int {
            k_gtri<<<gs, 128, 0, cs>>>(g);
            RBF_LAUNCH_CHECK();
            k_gadd<<<gb, 256, 0, cs>>>(g, lam_packed);
            RBF_LAUNCH_CHECK();
            RBF_CUDA_TRY(cudaMemcpyAsync(b->lam, lam_packed, total * sizeof(double),
                                         cudaMemcpyDeviceToDevice, cs));
            RBF_TRY(batch_enqueue(b, prec, cs));
            k_gresid<<<gb, 256, 0, cs>>>(g, u_packed, b->u);
            RBF_LAUNCH_CHECK();
            k_gactivate<<<gs, 128, 0, cs>>>(g);
            RBF_LAUNCH_CHECK();
            k_gdots<<<dim3(GM_BB, 1, nsys), BRED_T, 0, cs>>>(g, g.V, 1);
            RBF_LAUNCH_CHECK();
            k_gstart<<<gs, 128, 0, cs>>>(g);
            RBF_LAUNCH_CHECK();
            k_gscale0<<<gb, 256, 0, cs>>>(g);
            RBF_LAUNCH_CHECK();
            return RBF_OK;
        },
        &B.gr, &B.er));
    // ||u|| per system
    k_gactivate<<<gs, 128, 0, s>>>(g);
    RBF_LAUNCH_CHECK();
    k_gdots<<<dim3(GM_BB, 1, nsys), BRED_T, 0, s>>>(g, u_packed, 1);
    RBF_LAUNCH_CHECK();
    k_gbnorm<<<gs, 128, 0, s>>>(g);
    RBF_LAUNCH_CHECK();
    auto read_any = [&]() -> int {
        RBF_CUDA_TRY(cudaMemcpyAsync(B.pinned, g.any, sizeof(int), cudaMemcpyDeviceToHost, s));
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        return RBF_OK;
    };
    RBF_CUDA_TRY(cudaGraphLaunch(B.er, s));  // ny = 0: the residual of the initial guess
    RBF_TRY(read_any());
    int it = 0, nsteps = 0;
    double step_ms = 0.0;
    while (it < max_iters && *B.pinned) {
        for (int jj = 0; jj < restart_m && it < max_iters; ++jj) {
            RBF_CUDA_TRY(cudaEventRecord(B.e0, s));
            RBF_CUDA_TRY(cudaGraphLaunch(B.es, s));
            RBF_CUDA_TRY(cudaEventRecord(B.e1, s));
            RBF_TRY(read_any());
            float ms = 0.f;
            RBF_CUDA_TRY(cudaEventElapsedTime(&ms, B.e0, B.e1));
            step_ms += ms;
            ++nsteps;
            ++it;
            if (!*B.pinned) break;
        }
        RBF_CUDA_TRY(cudaGraphLaunch(B.er, s));
        RBF_TRY(read_any());
    }
    std::vector<double> beta(nsys), bn(nsys);
    RBF_CUDA_TRY(cudaMemcpyAsync(beta.data(), g.beta, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(bn.data(), g.bnorm, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    if (rel_resid_host)
        for (int q = 0; q < nsys; ++q) rel_resid_host[q] = beta[q] / bn[q];
    if (iters_host) *iters_host = it;
    if (step_ms_host) *step_ms_host = nsteps ? step_ms / nsteps : 0.0;
    return RBF_OK;
}
