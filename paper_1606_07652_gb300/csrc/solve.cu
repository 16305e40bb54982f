// solve.cu -- interpolation solve A lambda = u (Sec. 1: a Krylov method with
// the FMM product in place of the dense matrix-vector product).
//
// Restarted GMRES(m), right-preconditioned, with two-pass classical
// Gram-Schmidt (CGS2) and Givens rotations; the Krylov basis and every
// reduction are FP64 on the device, the small Hessenberg least-squares
// problem is solved on the host.  Around it, FP64 iterative refinement:
//     r = u - A64 lambda;  solve A delta = r with GMRES on the inner-precision
//     product;  lambda += delta;  until ||r|| / ||u|| <= rtol.
// Reductions run in a fixed order (two-stage, fixed grid), so a solve is
// bit-reproducible on one device.
#include <chrono>
#include <cmath>
#include <vector>

#include "rbf_internal.cuh"

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 1024;  // fixed: reduction order does not depend on the device

// part[k * RED_BLOCKS + b] = sum over block b's slice of V_k . w
__global__ void __launch_bounds__(RED_THREADS) k_dots(const double *V, int64_t ldv, const double *w,
                                                      int64_t n, double *part)
{
    __shared__ double sh[RED_THREADS];
    const int k = blockIdx.y;
    const double *v = V + (int64_t)k * ldv;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x; i < n;
         i += (int64_t)RED_BLOCKS * RED_THREADS)
        s = fma(v[i], w[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)k * RED_BLOCKS + blockIdx.x] = sh[0];
}

// out[k] = sum_b part[k * RED_BLOCKS + b]  (one block per k, fixed order)
__global__ void __launch_bounds__(RED_THREADS) k_dots_final(const double *part, double *out)
{
    __shared__ double sh[RED_THREADS];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < RED_BLOCKS; b += RED_THREADS) s += part[(int64_t)k * RED_BLOCKS + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

// w -= sum_{k<nv} V_k h_k   (h on the device)
__global__ void k_gemv_sub(const double *V, int64_t ldv, int nv, const double *h, double *w,
                           int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = w[i];
    for (int k = 0; k < nv; ++k) s = fma(-V[(int64_t)k * ldv + i], h[k], s);
    w[i] = s;
}

// x += sum_{k<nv} V_k y_k
__global__ void k_gemv_add(const double *V, int64_t ldv, int nv, const double *y, double *x,
                           int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = x[i];
    for (int k = 0; k < nv; ++k) s = fma(V[(int64_t)k * ldv + i], y[k], s);
    x[i] = s;
}

__global__ void k_scale_copy(const double *in, double a, double *out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * in[i];
}

// out = a - b
__global__ void k_sub(const double *a, const double *b, double *out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}

__global__ void k_axpy(double a, const double *x, double *y, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], y[i]);
}

__global__ void k_permute(const double *in, const int32_t *perm, int64_t n, double *out, int inverse)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (inverse) out[perm[i]] = in[i];
    else out[i] = in[perm[i]];
}

struct Solver {
    rbf_tree *t;
    rbf_kernel kernel;
    double eps;
    const rbf_fmm_params *params;
    cudaStream_t s;
    int64_t n;
    int m;
    double *V = nullptr;     // (m+1) x n basis
    double *w = nullptr, *z = nullptr, *r = nullptr, *part = nullptr, *hd = nullptr;
    std::vector<double> hh;  // host copy of reductions
    int mv_inner = 0, mv64 = 0;
    bool use_p = false;      // right preconditioner P attached to the tree
    // residual history (rbf_solve_opts::history_host): iterations, seconds,
    // relative residual, kind
    double *hist = nullptr;
    int hist_cap = 0, hist_len = 0;
    int it_base = 0;         // inner iterations taken before the current GMRES call
    double nu = 1.0;         // ||u|| of the column being solved
    std::chrono::steady_clock::time_point t0;
    void record(int iters, double rel, int kind)
    {
        if (!hist || hist_len >= hist_cap) return;
        double *e = hist + 4 * (size_t)hist_len++;
        e[0] = iters;
        e[1] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        e[2] = rel;
        e[3] = kind;
    }

    int alloc(int m_)
    {
        m = m_;
        RBF_TRY(rbf_alloc(&V, (size_t)(m + 1) * n));
        RBF_TRY(rbf_alloc(&w, n));
        RBF_TRY(rbf_alloc(&z, n));
        RBF_TRY(rbf_alloc(&r, n));
        RBF_TRY(rbf_alloc(&part, (size_t)(m + 2) * RED_BLOCKS));
        RBF_TRY(rbf_alloc(&hd, m + 2));
        hh.resize(m + 2);
        return RBF_OK;
    }
    void release()
    {
        rbf_free(V);
        rbf_free(w);
        rbf_free(z);
        rbf_free(r);
        rbf_free(part);
        rbf_free(hd);
    }
    // out[0..nv) = V_k . x on the device (hd) and the host (hh)
    int dots(const double *Vb, int nv, const double *x, bool to_host)
    {
        dim3 g(RED_BLOCKS, nv);
        k_dots<<<g, RED_THREADS, 0, s>>>(Vb, n, x, n, part);
        RBF_LAUNCH_CHECK();
        k_dots_final<<<nv, RED_THREADS, 0, s>>>(part, hd);
        RBF_LAUNCH_CHECK();
        if (to_host) {
            RBF_CUDA_TRY(cudaMemcpyAsync(hh.data(), hd, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
            RBF_CUDA_TRY(cudaStreamSynchronize(s));
        }
        return RBF_OK;
    }
    int norm(const double *x, double *out)
    {
        RBF_TRY(dots(x, 1, x, true));
        *out = std::sqrt(std::max(hh[0], 0.0));
        return RBF_OK;
    }
    int matvec(int prec, const double *x, double *y)
    {
        if (prec == RBF_FP64) ++mv64;
        else ++mv_inner;
        return rbf_matvec_sorted64(t, kernel, eps, params, prec, x, y, s);
    }
    // A (P x): right preconditioning (P = identity unless use_p)
    int apply_op(int prec, const double *x, double *y)
    {
        if (!use_p) return matvec(prec, x, y);
        RBF_TRY(rbf_precond_apply_sorted(t, x, z, s));
        return matvec(prec, z, y);
    }

    // GMRES(m) on A x = b, x in/out, stops when ||b - A x|| <= tol_abs (estimate).
    int gmres(int prec, const double *b, double *x, bool x_zero, double tol_abs, int maxit,
              int *iters, double *est)
    {
        const int bs = 256;
        const int gb = ceil_div(n, bs);
        int it = 0;
        double beta = 0.0;
        // r = b - A x
        if (x_zero) {
            RBF_CUDA_TRY(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            RBF_TRY(apply_op(prec, x, w));
            k_sub<<<gb, bs, 0, s>>>(b, w, r, n);
            RBF_LAUNCH_CHECK();
        }
        RBF_TRY(norm(r, &beta));
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
        while (true) {
            if (!(beta > tol_abs) || it >= maxit || !std::isfinite(beta)) break;
            k_scale_copy<<<gb, bs, 0, s>>>(r, 1.0 / beta, V, n);
            RBF_LAUNCH_CHECK();
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int j = 0;
            double res = beta;
            for (; j < m && it < maxit; ++j, ++it) {
                double *vj = V + (int64_t)j * n, *vn = V + (int64_t)(j + 1) * n;
                RBF_TRY(apply_op(prec, vj, w));
                // CGS2
                std::vector<double> h(j + 2, 0.0);
                for (int pass = 0; pass < 2; ++pass) {
                    RBF_TRY(dots(V, j + 1, w, true));
                    for (int k = 0; k <= j; ++k) h[k] += hh[k];
                    k_gemv_sub<<<gb, bs, 0, s>>>(V, n, j + 1, hd, w, n);
                    RBF_LAUNCH_CHECK();
                }
                double hn = 0.0;
                RBF_TRY(norm(w, &hn));
                h[j + 1] = hn;
                // apply previous rotations, then a new one
                for (int k = 0; k < j; ++k) {
                    double a = cs[k] * h[k] + sn[k] * h[k + 1];
                    double bq = -sn[k] * h[k] + cs[k] * h[k + 1];
                    h[k] = a;
                    h[k + 1] = bq;
                }
                double den = std::hypot(h[j], h[j + 1]);
                cs[j] = den > 0 ? h[j] / den : 1.0;
                sn[j] = den > 0 ? h[j + 1] / den : 0.0;
                h[j] = den;
                h[j + 1] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = h[k];
                res = std::fabs(g[j + 1]);
                if (hn > 0.0) {
                    k_scale_copy<<<gb, bs, 0, s>>>(w, 1.0 / hn, vn, n);
                    RBF_LAUNCH_CHECK();
                }
                if (res <= tol_abs || hn == 0.0 || !std::isfinite(res)) {
                    ++j;
                    ++it;
                    break;
                }
            }
            // back substitution H y = g on the j x j upper triangle
            for (int k = j - 1; k >= 0; --k) {
                double v = g[k];
                for (int q = k + 1; q < j; ++q) v -= H[(size_t)k * m + q] * y[q];
                y[k] = v / H[(size_t)k * m + k];
            }
            RBF_CUDA_TRY(cudaMemcpyAsync(hd, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, s));
            k_gemv_add<<<gb, bs, 0, s>>>(V, n, j, hd, x, n);
            RBF_LAUNCH_CHECK();
            beta = res;
            if (res <= tol_abs || it >= maxit || !std::isfinite(res)) break;
            // restart from the true residual of the inner operator
            RBF_TRY(apply_op(prec, x, w));
            k_sub<<<gb, bs, 0, s>>>(b, w, r, n);
            RBF_LAUNCH_CHECK();
            RBF_TRY(norm(r, &beta));
            record(it_base + it, beta / nu, RBF_HIST_INNER);
        }
        *iters = it;
        *est = beta;
        return RBF_OK;
    }
};

}  // namespace

extern "C" int rbf_interp_solve(rbf_tree *t, rbf_kernel kernel, double eps,
                                const rbf_fmm_params *params, const double *u, double *lambda,
                                int nrhs, const rbf_solve_opts *opts, rbf_solve_report *rep,
                                void *stream)
{
    RBF_REQUIRE(t != nullptr, "rbf_interp_solve: tree is NULL");
    RBF_REQUIRE(u && lambda && opts, "rbf_interp_solve: NULL argument");
    RBF_REQUIRE(nrhs >= 1, "rbf_interp_solve: nrhs=%d", nrhs);
    RBF_REQUIRE(opts->restart_m >= 1 && opts->restart_m <= 200, "restart_m=%d", opts->restart_m);
    RBF_REQUIRE(opts->max_iters >= 1 && opts->max_refine >= 1, "iteration limits must be >= 1");
    RBF_REQUIRE(opts->rtol > 0.0, "rtol must be > 0");
    RBF_REQUIRE(opts->inner_prec == RBF_FP64 || opts->inner_prec == RBF_FP32, "inner_prec");
    RBF_REQUIRE(opts->precond == 0 || opts->precond == 1, "precond=%d", opts->precond);
    RBF_REQUIRE(opts->precond == 0 || t->pc.ready,
                "precond=1: no preconditioner is attached to this tree (rbf_precond_build)");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = t->N;
    Solver sv;
    sv.t = t;
    sv.kernel = kernel;
    sv.eps = eps;
    sv.params = params;
    sv.s = s;
    sv.n = n;
    int st = sv.alloc(opts->restart_m);
    double *us = nullptr, *ls = nullptr, *ax = nullptr, *dl = nullptr, *lprev = nullptr;
    int fallback = 0;
    if (st == RBF_OK) st = rbf_alloc(&lprev, n);
    if (st == RBF_OK) st = rbf_alloc(&us, n);
    if (st == RBF_OK) st = rbf_alloc(&ls, n);
    if (st == RBF_OK) st = rbf_alloc(&ax, n);
    if (st == RBF_OK) st = rbf_alloc(&dl, n);
    double *lbest = nullptr;
    if (st == RBF_OK && opts->precond == 1) st = rbf_alloc(&lbest, n);
    sv.t0 = t0;
    if (opts->history_host && opts->history_cap > 0) {
        sv.hist = opts->history_host;
        sv.hist_cap = opts->history_cap;
    }
    int total_it = 0, refinements = 0, status = RBF_OK;
    double worst = 0.0;
    const int bs = 256, gb = ceil_div(n, bs);
    const double floor_inner = opts->inner_prec == RBF_FP32 ? 2e-6 : 0.0;
    for (int c = 0; c < nrhs && st == RBF_OK; ++c) {
        const double *uc = u + (int64_t)c * n;
        double *lc = lambda + (int64_t)c * n;
        k_permute<<<gb, bs, 0, s>>>(uc, t->perm, n, us, 0);
        k_permute<<<gb, bs, 0, s>>>(lc, t->perm, n, ls, 0);
        double nu = 0.0;
        st = sv.norm(us, &nu);
        if (st != RBF_OK) break;
        if (nu == 0.0) nu = 1.0;
        sv.nu = nu;
        double rel = INFINITY, prev = INFINITY;
        int it_c = 0, k = 0;
        bool conv = false;
        sv.use_p = opts->precond == 1;
        bool last_used_p = false;
        bool stale = true;  // lambda changed since the last FP64 residual
        double last_rn = 0.0;  // ||r|| of that residual (r itself is in sv.r)
        // FP64 residual r = u - A64 lambda into sv.r; its relative norm into *out
        auto fp64_resid = [&](double *out_rel, double *out_norm) -> int {
            RBF_TRY(sv.matvec(RBF_FP64, ls, ax));
            k_sub<<<gb, bs, 0, s>>>(us, ax, sv.r, n);
            RBF_LAUNCH_CHECK();
            RBF_TRY(sv.norm(sv.r, out_norm));
            *out_rel = *out_norm / nu;
            sv.record(total_it + it_c, *out_rel, RBF_HIST_FP64);
            stale = false;
            last_rn = *out_norm;
            return RBF_OK;
        };
        // one correction step: GMRES on A (P) y = r (r in sv.r, FP64 norm rn),
        // lambda += (P) y; at most `budget` inner iterations
        auto correct = [&](double rn, double rel_now, int budget) -> int {
            const double eta = std::max(0.5 * opts->rtol / rel_now, floor_inner);
            RBF_CUDA_TRY(cudaMemsetAsync(dl, 0, n * sizeof(double), s));
            double *rr = ax;  // keep r: gmres reuses sv.r
            RBF_CUDA_TRY(cudaMemcpyAsync(rr, sv.r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            int its = 0;
            double est = 0.0;
            sv.it_base = total_it + it_c;
            RBF_TRY(sv.gmres(opts->inner_prec, rr, dl, true, eta * rn, budget, &its, &est));
            it_c += its;
            ++refinements;
            stale = true;
            last_used_p = sv.use_p;
            if (sv.use_p) {
                RBF_TRY(rbf_precond_apply_sorted(t, dl, sv.w, s));
                k_axpy<<<gb, bs, 0, s>>>(1.0, sv.w, ls, n);
            } else {
                k_axpy<<<gb, bs, 0, s>>>(1.0, dl, ls, n);
            }
            RBF_LAUNCH_CHECK();
            return its;
        };
        if (sv.use_p) {
            // Trial of the preconditioner: one restart cycle with P.  When the inner
            // solve does not converge within that cycle, one plain cycle from the same
            // start is compared with it on the FP64 residual and the better iterate is
            // kept; a useless P so costs at most one cycle.
            double rn = 0.0;
            if ((st = fp64_resid(&rel, &rn)) != RBF_OK) break;
            if (rel <= opts->rtol) {
                conv = true;
            } else {
                RBF_CUDA_TRY(cudaMemcpyAsync(lprev, ls, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                const double rel0 = rel, rn0 = rn;
                const int budget = std::min(opts->restart_m, opts->max_iters);
                const int its = correct(rn0, rel0, budget);
                if (its < 0) { st = its; break; }
                double rel_p = 0.0, rn_p = 0.0;
                if ((st = fp64_resid(&rel_p, &rn_p)) != RBF_OK) break;
                rel = rel_p;
                const bool inner_converged = its < budget;
                if (rel_p > opts->rtol && !inner_converged && it_c < opts->max_iters) {
                    RBF_CUDA_TRY(cudaMemcpyAsync(lbest, ls, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                    RBF_CUDA_TRY(cudaMemcpyAsync(ls, lprev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                    sv.use_p = false;
                    double rel_r = 0.0, rn_r = 0.0;
                    if ((st = fp64_resid(&rel_r, &rn_r)) != RBF_OK) break;
                    const int its2 = correct(rn_r, rel_r, std::min(budget, opts->max_iters - it_c));
                    if (its2 < 0) { st = its2; break; }
                    double rel_i = 0.0, rn_i = 0.0;
                    if ((st = fp64_resid(&rel_i, &rn_i)) != RBF_OK) break;
                    if (rel_i <= rel_p) {
                        fallback = 1;  // the plain cycle did better: drop P
                        rel = rel_i;
                    } else {
                        RBF_CUDA_TRY(cudaMemcpyAsync(ls, lbest, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                        sv.use_p = true;
                        last_used_p = true;
                        rel = rel_p;
                        stale = true;  // sv.r holds the plain iterate's residual
                    }
                }
                prev = rel;
                if (rel <= opts->rtol) conv = true;
            }
        }
        while (!conv && k < opts->max_refine) {
            // true residual with the FP64 product (kept from the trial when the
            // iterate has not changed since)
            double rn = last_rn;
            if (stale && (st = fp64_resid(&rel, &rn)) != RBF_OK) break;
            if (rel <= opts->rtol) {
                conv = true;
                break;
            }
            const bool stalled = !std::isfinite(rel) || (k > 0 && rel > 0.5 * prev);
            if (stalled && last_used_p) {
                // the preconditioned step did not pay off on the FP64 residual: undo it
                // and continue with the plain (identity-preconditioned) iteration
                RBF_CUDA_TRY(cudaMemcpyAsync(ls, lprev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                sv.use_p = false;
                last_used_p = false;
                fallback = 1;
                stale = true;
                prev = INFINITY;  // the restored iterate starts a fresh progress test
                continue;
            }
            if (stalled) break;
            prev = rel;
            if (it_c >= opts->max_iters) break;
            ++k;
            RBF_CUDA_TRY(cudaMemcpyAsync(lprev, ls, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            // inner solve A P y = r, delta = P y; each refinement step gets an equal
            // share of the budget, so that the FP64 residual judges every step
            const int share = std::max(opts->restart_m, opts->max_iters / opts->max_refine);
            const int its = correct(rn, rel, std::min(opts->max_iters - it_c, share));
            if (its < 0) {
                st = its;
                break;
            }
        }
        if (st == RBF_OK && !conv && stale) {
            // the budget ended on a correction step: judge the final iterate
            double rn = 0.0;
            st = fp64_resid(&rel, &rn);
            if (st == RBF_OK && rel <= opts->rtol) conv = true;
        }
        if (st != RBF_OK) break;
        total_it += it_c;
        worst = std::max(worst, rel);
        if (!conv) status = RBF_ENOCONV;
        k_permute<<<gb, bs, 0, s>>>(ls, t->perm, n, lc, 1);
    }
    if (st == RBF_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rbf_set_error("rbf_interp_solve: %s", cudaGetErrorString(e));
            st = RBF_ECUDA;
        }
    }
    sv.release();
    rbf_free(us);
    rbf_free(ls);
    rbf_free(ax);
    rbf_free(dl);
    rbf_free(lprev);
    rbf_free(lbest);
    if (rep) {
        rep->history_len = sv.hist_len;
        rep->iters = total_it;
        rep->refinements = refinements;
        rep->used_fallback = fallback;
        rep->rel_resid = worst;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        rep->matvecs_inner = sv.mv_inner;
        rep->matvecs_fp64 = sv.mv64;
    }
    if (st != RBF_OK) return st;
    if (status != RBF_OK) rbf_set_error("rbf_interp_solve: relative residual %.3e > rtol %.3e", worst,
                                        opts->rtol);
    return status;
}
