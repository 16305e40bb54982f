// batch.cu -- many independent interpolation problems of uneven size at once,
// and the autotuner that picks each problem's tree depth and expansion order.
//
// Every problem keeps its own tree and plan (autotuned); the FP32 products of
// all problems and all their right-hand sides are captured once into one CUDA
// graph, fanned out over several streams so that small problems run side by
// side, and the graph is replayed for every GMRES step.  The batched GMRES runs
// all systems (problem, right-hand side) in lockstep with packed FP64 Krylov
// bases, batched CGS2 reductions on the device and the small Hessenberg
// problems on the host (one device-to-host copy per step for all systems).
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

// max over sampled far offsets r (w <= |r|_inf <= side) of |K(r) - Phi(r)| with
// K(r) = Re sum_{half spectrum} omegaC e^{i xi.r}; one thread per sample.
__global__ void k_kernel_error(int d, int M, int64_t nmode, const double *xi, const double *omegaC,
                               int kernel, double eps, double w, double side, int nsample,
                               uint64_t seed, double *err)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsample) return;
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
    for (int64_t m = 0; m < nmode; ++m) {
        int64_t rr = m;
        double ph = 0.0;
        for (int t = d - 1; t >= 1; --t) {
            ph += xi[rr % n1] * r[t];
            rr /= n1;
        }
        ph += xi[rr + M / 2] * r[0];
        K += omegaC[m] * cos(ph);
    }
    const double phi = rbf_phi64(kernel, eps * eps * r2);
    err[q] = fabs(K - phi);
}

constexpr int BRED_T = 256;

// part[(s * ks + k) * BB + b]: block b's share of V_k[s] . w[s]  (systems s, k < nk[s])
__global__ void k_bdots(const double *V, int64_t total, const double *w, const int64_t *off,
                        const int64_t *len, int ks, const int *nk, const int *active, double *part,
                        int BB)
{
    const int s = blockIdx.z, k = blockIdx.y, b = blockIdx.x;
    __shared__ double sh[BRED_T];
    double acc = 0.0;
    if (active[s] && k < nk[s]) {
        const double *v = V + (int64_t)k * total + off[s];
        const double *x = w + off[s];
        for (int64_t i = (int64_t)b * BRED_T + threadIdx.x; i < len[s]; i += (int64_t)BB * BRED_T)
            acc = fma(v[i], x[i], acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = BRED_T / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[((int64_t)s * ks + k) * BB + b] = sh[0];
}

__global__ void k_bdots_final(const double *part, int nsys, int ks, int BB, double *h)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)nsys * ks) return;
    double s = 0.0;
    for (int b = 0; b < BB; ++b) s += part[q * BB + b];
    h[q] = s;
}

// w -= sum_{k<nk[s]} V_k h[s][k]   (elementwise, sys_of maps elements to systems)
__global__ void k_bgemv_sub(const double *V, int64_t total, const int *sys_of, const int *nk,
                            const int *active, int ks, const double *h, double *w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int s = sys_of[i];
    if (!active[s]) return;
    double a = w[i];
    for (int k = 0; k < nk[s]; ++k) a = fma(-V[(int64_t)k * total + i], h[(int64_t)s * ks + k], a);
    w[i] = a;
}

// x += sum_{k<ny[s]} V_k y[s][k]
__global__ void k_bgemv_add(const double *V, int64_t total, const int *sys_of, const int *ny, int ks,
                            const double *y, double *x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int s = sys_of[i];
    double a = x[i];
    for (int k = 0; k < ny[s]; ++k) a = fma(V[(int64_t)k * total + i], y[(int64_t)s * ks + k], a);
    x[i] = a;
}

// out = scale[s] * in   (per system)
__global__ void k_bscale(const double *in, const int *sys_of, const double *scale, int64_t total,
                         double *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) out[i] = scale[sys_of[i]] * in[i];
}

__global__ void k_sub2(const double *a, const double *b, int64_t n, double *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
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
        k_kernel_error<<<ceil_div(ns, 128), 128>>>(d, pl->M, pl->nmode, (const double *)pl->xi,
                                                   (const double *)pl->omegaC, kernel, eps, w, side,
                                                   ns, 0x5EEDull, err);
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

extern "C" int rbf_autotune(rbf_kernel kernel, double eps, int d, int64_t N, double side, double tol,
                            rbf_fmm_params *out, int *depth_out, double *err_out)
{
    RBF_REQUIRE(out && depth_out, "rbf_autotune: NULL argument");
    RBF_REQUIRE(eps > 0.0 && side > 0.0 && tol > 0.0 && N >= 1 && d >= 1 && d <= RBF_MAX_DIM,
                "rbf_autotune: bad arguments");
    // depth: about 32 points per leaf in 3-D and up, 64 in 1-D/2-D, at least 2 levels
    const double per_leaf = d >= 3 ? 32.0 : 64.0;
    int D = (int)std::lround(std::log(std::max(1.0, (double)N / per_leaf)) / std::log((double)(1 << d)));
    D = std::max(2, std::min(D, RBF_MAX_DEPTH));
    while (d * D > 63) --D;
    // period and taper: the Gaussian needs Phi(L - side) below tol; the Wendland
    // function needs its support 1/eps inside L - side; the (inverse) multiquadric a
    // taper between side and L - side
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
    // expansion order: the smallest even M in [8, 64] whose measured far-kernel error
    // meets tol (the error falls with M), else 64.  The search starts from the M at
    // which the kernel's Fourier transform has decayed to tol at the band edge
    // pi M / L (Gaussian: exp(-xi^2 / (4 eps^2)); inverse multiquadric: ~exp(-xi / eps))
    // and steps by 2.
    auto error_at = [&](int M, double *e) -> int {
        p.M = M;
        return rbf_kernel_error(kernel, eps, d, &p, side, D, e);
    };
    // no far field at all when the kernel is within tol beyond one leaf width
    // (K = 0 is then a far kernel within tol: narrow Gaussians, compact supports)
    {
        double e0 = INFINITY;
        RBF_TRY(error_at(0, &e0));
        if (e0 <= tol) {
            p.M = 0;
            *out = p;
            *depth_out = D;
            if (err_out) *err_out = e0;
            return RBF_OK;
        }
    }
    const double lt = std::log(1.0 / tol);
    // (the Wendland function's transform decays only algebraically: start at 16)
    const double pred = kernel == RBF_GAUSSIAN ? 2.0 * eps * p.period_L * std::sqrt(lt) / M_PI
                        : kernel == RBF_WENDLAND ? 16.0
                                                 : eps * p.period_L * lt / M_PI;
    int M0 = 2 * (int)std::lround(pred / 2.0);
    M0 = std::max(8, std::min(64, M0));
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
    p.M = Mbest;
    *out = p;
    *depth_out = D;
    if (err_out) *err_out = err;
    return RBF_OK;
}

// ---------------------------------------------------------------- batches ---
struct rbf_batch {
    int np = 0;
    std::vector<rbf_tree *> trees;
    std::vector<rbf_problem> probs;
    std::vector<rbf_fmm_params> params;
    std::vector<int> depth;
    std::vector<int64_t> off;  // packed offset of problem p (all its right-hand sides)
    int64_t total = 0;
    double *lam = nullptr, *u = nullptr;  // packed product buffers
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_prec = -1;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
};

static void batch_release(rbf_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->events) cudaEventDestroy(e);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto t : b->trees) rbf_tree_free(t);
    rbf_free(b->lam);
    rbf_free(b->u);
    delete b;
}

extern "C" void rbf_batch_free(rbf_batch *b)
{
    if (b) batch_release(b);
}

extern "C" int rbf_batch_create(const rbf_problem *probs, int np, double tol_kernel, void *stream,
                                rbf_batch **out)
{
    RBF_REQUIRE(out && probs && np >= 1, "rbf_batch_create: bad arguments");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rbf_batch *b = new rbf_batch();
    b->np = np;
    b->probs.assign(probs, probs + np);
    int st = RBF_OK;
    for (int p = 0; p < np && st == RBF_OK; ++p) {
        const rbf_problem &q = probs[p];
        if (!(q.X && q.N >= 1 && q.d >= 1 && q.d <= RBF_MAX_DIM && q.nrhs >= 1 && q.eps > 0.0)) {
            rbf_set_error("rbf_batch_create: problem %d is malformed", p);
            st = RBF_EINVAL;
            break;
        }
        rbf_fmm_params prm{};
        int D = 2;
        double err = 0.0;
        st = rbf_autotune(q.kernel, q.eps, q.d, q.N, 1.0, tol_kernel, &prm, &D, &err);
        if (st != RBF_OK) break;
        std::vector<double> lo(q.d, 0.0);
        rbf_tree *t = nullptr;
        st = rbf_tree_build(q.X, q.N, q.d, lo.data(), 1.0, D, stream, &t);
        if (st != RBF_OK) break;
        b->trees.push_back(t);
        b->params.push_back(prm);
        b->depth.push_back(D);
        b->off.push_back(b->total);
        b->total += q.N * q.nrhs;
    }
    if (st == RBF_OK) st = rbf_alloc(&b->lam, std::max<int64_t>(b->total, 1));
    if (st == RBF_OK) st = rbf_alloc(&b->u, std::max<int64_t>(b->total, 1));
    if (st == RBF_OK && cudaMemsetAsync(b->lam, 0, b->total * sizeof(double), s) != cudaSuccess)
        st = RBF_ECUDA;
    if (st == RBF_OK) {
        const int ns = std::min(np, 16);
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
    *out = b;
    return RBF_OK;
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


// all products, one stream per problem slot, in the order they are enqueued
static int batch_enqueue(rbf_batch *b, int prec, cudaStream_t s)
{
    const int ns = (int)b->streams.size();
    RBF_CUDA_TRY(cudaEventRecord(b->events[ns], s));
    for (int q = 0; q < ns; ++q) RBF_CUDA_TRY(cudaStreamWaitEvent(b->streams[q], b->events[ns], 0));
    for (int p = 0; p < b->np; ++p) {
        const rbf_problem &q = b->probs[p];
        cudaStream_t sq = b->streams[p % ns];
        RBF_TRY(rbf_fmm_matvec(b->trees[p], q.kernel, q.eps, &b->params[p], (rbf_precision)prec,
                               b->lam + b->off[p], q.N, b->u + b->off[p], q.N, q.nrhs, sq));
    }
    for (int q = 0; q < ns; ++q) {
        RBF_CUDA_TRY(cudaEventRecord(b->events[q], b->streams[q]));
        RBF_CUDA_TRY(cudaStreamWaitEvent(s, b->events[q], 0));
    }
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
        cudaStream_t cs;
        RBF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const cudaError_t eb = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (eb != cudaSuccess) cudaStreamDestroy(cs);
        RBF_CUDA_TRY(eb);
        const int st = batch_enqueue(b, prec, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (st != RBF_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        RBF_CUDA_TRY(e);
        b->graph = g;
        RBF_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
        b->graph_prec = prec;
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

extern "C" int rbf_batch_solve(rbf_batch *b, const double *u_packed, double *lam_packed,
                               int restart_m, int max_iters, double rtol, rbf_precision prec,
                               double *rel_resid_host, int *iters_host, double *step_ms_host,
                               void *stream)
{
    RBF_REQUIRE(b && u_packed && lam_packed, "rbf_batch_solve: NULL argument");
    RBF_REQUIRE(restart_m >= 1 && restart_m <= 200 && max_iters >= 1 && rtol > 0.0,
                "rbf_batch_solve: bad options");
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    // systems: (problem, right-hand side)
    std::vector<int64_t> soff, slen;
    for (int p = 0; p < b->np; ++p)
        for (int r = 0; r < b->probs[p].nrhs; ++r) {
            soff.push_back(b->off[p] + (int64_t)r * b->probs[p].N);
            slen.push_back(b->probs[p].N);
        }
    const int nsys = (int)soff.size();
    const int64_t total = b->total;
    const int m = restart_m, ks = m + 1, BB = 8;
    std::vector<int> sys_of(total);
    for (int q = 0; q < nsys; ++q)
        for (int64_t i = 0; i < slen[q]; ++i) sys_of[soff[q] + i] = q;
    double *V = nullptr, *w = nullptr, *r = nullptr, *part = nullptr, *hd = nullptr, *sc = nullptr;
    int64_t *doff = nullptr, *dlen = nullptr;
    int *dsys = nullptr, *dnk = nullptr, *dact = nullptr;
    RBF_TRY(rbf_alloc(&V, (size_t)(m + 1) * total));
    RBF_TRY(rbf_alloc(&w, total));
    RBF_TRY(rbf_alloc(&r, total));
    RBF_TRY(rbf_alloc(&part, (size_t)nsys * ks * BB));
    RBF_TRY(rbf_alloc(&hd, (size_t)nsys * ks));
    RBF_TRY(rbf_alloc(&sc, nsys));
    RBF_TRY(rbf_alloc(&doff, nsys));
    RBF_TRY(rbf_alloc(&dlen, nsys));
    RBF_TRY(rbf_alloc(&dsys, total));
    RBF_TRY(rbf_alloc(&dnk, nsys));
    RBF_TRY(rbf_alloc(&dact, nsys));
    RBF_CUDA_TRY(cudaMemcpyAsync(doff, soff.data(), nsys * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(dlen, slen.data(), nsys * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(dsys, sys_of.data(), total * sizeof(int), cudaMemcpyHostToDevice, s));
    const int gb = ceil_div(total, 256);
    std::vector<double> hh((size_t)nsys * ks);
    std::vector<int> nk(nsys), act(nsys, 1);
    auto dots = [&](const double *Vb, const double *x, int kmax) -> int {
        RBF_CUDA_TRY(cudaMemcpyAsync(dnk, nk.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, s));
        RBF_CUDA_TRY(cudaMemcpyAsync(dact, act.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, s));
        dim3 g(BB, kmax, nsys);
        k_bdots<<<g, BRED_T, 0, s>>>(Vb, total, x, doff, dlen, ks, dnk, dact, part, BB);
        RBF_LAUNCH_CHECK();
        k_bdots_final<<<ceil_div((int64_t)nsys * ks, 256), 256, 0, s>>>(part, nsys, ks, BB, hd);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaMemcpyAsync(hh.data(), hd, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        return RBF_OK;
    };
    // x = lambda (initial guess), r = u - A x
    std::vector<double> bnorm(nsys), beta(nsys), res(nsys, INFINITY);
    RBF_CUDA_TRY(cudaMemcpyAsync(b->lam, lam_packed, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RBF_TRY(batch_matvec(b, prec, s));
    k_sub2<<<gb, 256, 0, s>>>(u_packed, b->u, total, r);
    RBF_LAUNCH_CHECK();
    // ||u|| and ||r||: the systems' own segments, via V_0 = u then V_0 = r
    RBF_CUDA_TRY(cudaMemcpyAsync(V, u_packed, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::fill(nk.begin(), nk.end(), 1);
    RBF_TRY(dots(V, u_packed, 1));
    for (int q = 0; q < nsys; ++q) bnorm[q] = std::sqrt(hh[(size_t)q * ks]) > 0 ? std::sqrt(hh[(size_t)q * ks]) : 1.0;
    RBF_CUDA_TRY(cudaMemcpyAsync(V, r, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RBF_TRY(dots(V, r, 1));
    for (int q = 0; q < nsys; ++q) beta[q] = std::sqrt(std::max(hh[(size_t)q * ks], 0.0));
    int it = 0;
    double step_ms = 0.0;
    int nsteps = 0;
    std::vector<double> H((size_t)nsys * ks * m), cs((size_t)nsys * m), sn((size_t)nsys * m),
        g((size_t)nsys * ks), y((size_t)nsys * ks);
    std::vector<double> scale(nsys);
    std::vector<int> ny(nsys);
    while (it < max_iters) {
        bool any = false;
        for (int q = 0; q < nsys; ++q) {
            act[q] = beta[q] > rtol * bnorm[q] && std::isfinite(beta[q]);
            any = any || act[q];
            scale[q] = act[q] ? 1.0 / beta[q] : 0.0;
            std::fill(&g[(size_t)q * ks], &g[(size_t)q * ks] + ks, 0.0);
            g[(size_t)q * ks] = beta[q];
            ny[q] = 0;
        }
        if (!any) break;
        RBF_CUDA_TRY(cudaMemcpyAsync(sc, scale.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, s));
        k_bscale<<<gb, 256, 0, s>>>(r, dsys, sc, total, V);
        RBF_LAUNCH_CHECK();
        int j = 0;
        for (; j < m && it < max_iters; ++j, ++it) {
            const auto ts = std::chrono::steady_clock::now();
            // w = A v_j for every system (one graph launch)
            RBF_CUDA_TRY(cudaMemcpyAsync(b->lam, V + (int64_t)j * total, total * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
            RBF_TRY(batch_matvec(b, prec, s));
            RBF_CUDA_TRY(cudaMemcpyAsync(w, b->u, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
            std::vector<double> h((size_t)nsys * ks, 0.0);
            for (int q = 0; q < nsys; ++q) nk[q] = act[q] ? j + 1 : 0;
            for (int pass = 0; pass < 2; ++pass) {
                RBF_TRY(dots(V, w, j + 1));
                for (int q = 0; q < nsys; ++q)
                    for (int k = 0; k <= j; ++k) h[(size_t)q * ks + k] += hh[(size_t)q * ks + k];
                k_bgemv_sub<<<gb, 256, 0, s>>>(V, total, dsys, dnk, dact, ks, hd, w);
                RBF_LAUNCH_CHECK();
            }
            // ||w|| per system
            RBF_CUDA_TRY(cudaMemcpyAsync(V + (int64_t)(j + 1) * total, w, total * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
            for (int q = 0; q < nsys; ++q) nk[q] = act[q] ? 1 : 0;
            RBF_TRY(dots(V + (int64_t)(j + 1) * total, w, 1));
            for (int q = 0; q < nsys; ++q) {
                if (!act[q]) {
                    scale[q] = 0.0;
                    continue;
                }
                double *hq = &h[(size_t)q * ks];
                const double hn = std::sqrt(std::max(hh[(size_t)q * ks], 0.0));
                hq[j + 1] = hn;
                double *c = &cs[(size_t)q * m], *sq = &sn[(size_t)q * m], *gq = &g[(size_t)q * ks];
                for (int k = 0; k < j; ++k) {
                    const double a = c[k] * hq[k] + sq[k] * hq[k + 1];
                    const double bb = -sq[k] * hq[k] + c[k] * hq[k + 1];
                    hq[k] = a;
                    hq[k + 1] = bb;
                }
                const double den = std::hypot(hq[j], hq[j + 1]);
                c[j] = den > 0 ? hq[j] / den : 1.0;
                sq[j] = den > 0 ? hq[j + 1] / den : 0.0;
                hq[j] = den;
                gq[j + 1] = -sq[j] * gq[j];
                gq[j] = c[j] * gq[j];
                for (int k = 0; k <= j; ++k) H[((size_t)q * ks + k) * m + j] = hq[k];
                res[q] = std::fabs(gq[j + 1]);
                ny[q] = j + 1;
                scale[q] = hn > 0 ? 1.0 / hn : 0.0;
                if (res[q] <= rtol * bnorm[q] || hn == 0.0) act[q] = 0;
            }
            RBF_CUDA_TRY(cudaMemcpyAsync(sc, scale.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, s));
            k_bscale<<<gb, 256, 0, s>>>(w, dsys, sc, total, V + (int64_t)(j + 1) * total);
            RBF_LAUNCH_CHECK();
            RBF_CUDA_TRY(cudaStreamSynchronize(s));
            step_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
            ++nsteps;
            bool any_act = false;
            for (int q = 0; q < nsys; ++q) any_act = any_act || act[q];
            if (!any_act) {
                ++j;
                ++it;
                break;
            }
        }
        // x += V y per system
        for (int q = 0; q < nsys; ++q) {
            const int jj = ny[q];
            for (int k = jj - 1; k >= 0; --k) {
                double v = g[(size_t)q * ks + k];
                for (int c = k + 1; c < jj; ++c) v -= H[((size_t)q * ks + k) * m + c] * y[(size_t)q * ks + c];
                y[(size_t)q * ks + k] = v / H[((size_t)q * ks + k) * m + k];
            }
        }
        RBF_CUDA_TRY(cudaMemcpyAsync(dnk, ny.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, s));
        RBF_CUDA_TRY(cudaMemcpyAsync(hd, y.data(), y.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        k_bgemv_add<<<gb, 256, 0, s>>>(V, total, dsys, dnk, ks, hd, lam_packed);
        RBF_LAUNCH_CHECK();
        // restart from the true residual of the product
        RBF_CUDA_TRY(cudaMemcpyAsync(b->lam, lam_packed, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
        RBF_TRY(batch_matvec(b, prec, s));
        k_sub2<<<gb, 256, 0, s>>>(u_packed, b->u, total, r);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaMemcpyAsync(V, r, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
        std::fill(act.begin(), act.end(), 1);
        std::fill(nk.begin(), nk.end(), 1);
        RBF_TRY(dots(V, r, 1));
        for (int q = 0; q < nsys; ++q) beta[q] = std::sqrt(std::max(hh[(size_t)q * ks], 0.0));
    }
    for (int q = 0; q < nsys; ++q) {
        if (rel_resid_host) rel_resid_host[q] = beta[q] / bnorm[q];
    }
    if (iters_host) *iters_host = it;
    if (step_ms_host) *step_ms_host = nsteps ? step_ms / nsteps : 0.0;
    rbf_free(V);
    rbf_free(w);
    rbf_free(r);
    rbf_free(part);
    rbf_free(hd);
    rbf_free(sc);
    rbf_free(doff);
    rbf_free(dlen);
    rbf_free(dsys);
    rbf_free(dnk);
    rbf_free(dact);
    (void)t0;
    return RBF_OK;
}
