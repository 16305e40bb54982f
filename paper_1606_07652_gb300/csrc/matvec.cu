// matvec.cu -- u = A lambda (Eq. (54)): near field + far field, in the
// caller's order (entry points) or in Morton order (solver).
#include <algorithm>

#include "rbf_internal.cuh"

namespace {

template <typename R>
__global__ void k_gather(const double *in, const int32_t *perm, int64_t N, R *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = (R)in[perm ? perm[i] : i];
}

// u[perm[i]] = near[i] + far[i]  (far may be null)
template <typename R>
__global__ void k_scatter(const R *near, const R *far, const int32_t *perm, int64_t N, double *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = (double)near[i];
    if (far) v += (double)far[i];
    out[perm ? perm[i] : i] = v;
}

template <typename R>
int matvec_one(rbf_tree *t, rbf_plan *p, int kernel, double eps, const double *lam,
               const int32_t *perm, double *u, cudaStream_t s)
{
    R *lam_s = (R *)p->lam_s, *un = (R *)p->u_near, *uf = (R *)p->u_far;
    const int64_t N = t->N;
    {
        rbf_pass_timer tm(t, RBF_PASS_PERM, s);
        k_gather<R><<<ceil_div(N, 256), 256, 0, s>>>(lam, perm, N, lam_s);
        RBF_LAUNCH_CHECK();
    }
    RBF_TRY(rbf_run_p2p<R>(t, kernel, eps, lam_s, un, s));
    const bool far = t->D >= 2 && p->M > 0;  // M = 0: near field alone
    if (far) RBF_TRY(rbf_run_far<R>(t, p, lam_s, uf, s));
    {
        rbf_pass_timer tm(t, RBF_PASS_PERM, s);
        k_scatter<R><<<ceil_div(N, 256), 256, 0, s>>>(un, far ? uf : nullptr, perm, N, u);
        RBF_LAUNCH_CHECK();
    }
    return RBF_OK;
}

// lam_s[c][i] = lambda[c * ld + perm[i]], c < G
__global__ void k_gather_cols(const double *in, int64_t ld, const int32_t *perm, int64_t N, int G,
                              float *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t src = perm[i];
    for (int c = 0; c < G; ++c) out[(int64_t)c * N + i] = (float)in[(int64_t)c * ld + src];
}

// u[c * ld + perm[i]] = near[c][i] + far[c][i]
__global__ void k_scatter_cols(const float *near, const float *far, const int32_t *perm, int64_t N,
                               int G, double *out, int64_t ld)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t dst = perm[i];
    for (int c = 0; c < G; ++c) {
        double v = (double)near[(int64_t)c * N + i];
        if (far) v += (double)far[(int64_t)c * N + i];
        out[(int64_t)c * ld + dst] = v;
    }
}

// Workspace of G right-hand sides at once: leaf and local expansions per
// column plus FP32 vectors.  G = min(R, 16, what fits in min(64 GB, half of the
// free device memory)), then balanced over the groups of R columns; the
// workspace is kept and grown only when a later call needs more columns.
int multi_workspace(rbf_tree *t, rbf_plan *p, int R, int *G_out)
{
    const size_t per = 2 * (size_t)t->nleaf() * p->mstride * sizeof(float2) +
                       3 * (size_t)t->N * sizeof(float);
    const int want = std::min(R, 16);
    if (p->mr_G < want) {
        rbf_free(p->mr_V);
        rbf_free(p->mr_L);
        rbf_free(p->mr_lam);
        rbf_free(p->mr_un);
        rbf_free(p->mr_uf);
        p->mr_V = p->mr_L = nullptr;
        p->mr_lam = p->mr_un = p->mr_uf = nullptr;
        p->mr_G = 0;
        size_t fr = 0, tot = 0;
        RBF_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        const size_t budget = std::min<size_t>((size_t)64 << 30, fr / 2);
        RBF_REQUIRE(per <= budget, "rbf_fmm_matvec: %zu bytes per right-hand side exceed the budget",
                    per);
        const int gmax = (int)std::min<size_t>((size_t)want, budget / per);
        RBF_TRY(rbf_alloc(&p->mr_V, (size_t)gmax * t->nleaf() * p->mstride));
        // 64-byte tail: bulk copies of the last mode rows round up to 16 bytes
        RBF_TRY(rbf_alloc(&p->mr_L, (size_t)gmax * t->nleaf() * p->mstride + 8));
        RBF_TRY(rbf_alloc(&p->mr_lam, (size_t)gmax * t->N));
        RBF_TRY(rbf_alloc(&p->mr_un, (size_t)gmax * t->N));
        RBF_TRY(rbf_alloc(&p->mr_uf, (size_t)gmax * t->N));
        p->mr_G = gmax;
    }
    const int groups = (R + p->mr_G - 1) / p->mr_G;
    *G_out = (R + groups - 1) / groups;
    return RBF_OK;
}

// FP32 product of R columns, G at a time: near field per column, far field of
// the group with tensor-core P2M/L2P
int matvec_multi(rbf_tree *t, rbf_plan *p, int kernel, double eps, const double *lambda,
                 int64_t ldl, double *u, int64_t ldu, int R, cudaStream_t s)
{
    int G = 0;
    RBF_TRY(multi_workspace(t, p, R, &G));
    const int64_t N = t->N;
    const bool far = t->D >= 2 && p->M > 0;  // M = 0: near field alone
    for (int c0 = 0; c0 < R; c0 += G) {
        const int g = std::min(G, R - c0);
        {
            rbf_pass_timer tm(t, RBF_PASS_PERM, s);
            k_gather_cols<<<ceil_div(N, 256), 256, 0, s>>>(lambda + c0 * ldl, ldl, t->perm, N, g,
                                                          p->mr_lam);
            RBF_LAUNCH_CHECK();
        }
        RBF_TRY(rbf_run_p2p_multi(t, kernel, eps, p->mr_lam, g, p->mr_un, s));
        if (far) RBF_TRY(rbf_run_far_multi(t, p, p->mr_lam, g, p->mr_V, p->mr_L, p->mr_uf, s));
        {
            rbf_pass_timer tm(t, RBF_PASS_PERM, s);
            k_scatter_cols<<<ceil_div(N, 256), 256, 0, s>>>(p->mr_un, far ? p->mr_uf : nullptr,
                                                           t->perm, N, g, u + c0 * ldu, ldu);
            RBF_LAUNCH_CHECK();
        }
    }
    return RBF_OK;
}

}  // namespace

int rbf_matvec_sorted64(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *pp,
                        int prec, const double *lam_sorted, double *u_sorted, cudaStream_t s)
{
    rbf_plan *p = nullptr;
    RBF_TRY(rbf_plan_get(t, kernel, eps, pp, prec, s, &p));
    if (prec == RBF_FP64) return matvec_one<double>(t, p, kernel, eps, lam_sorted, nullptr, u_sorted, s);
    return matvec_one<float>(t, p, kernel, eps, lam_sorted, nullptr, u_sorted, s);
}

extern "C" int rbf_fmm_matvec(rbf_tree *t, rbf_kernel kernel, double eps,
                              const rbf_fmm_params *params, rbf_precision prec,
                              const double *lambda, int64_t ld_lambda, double *u, int64_t ld_u,
                              int nrhs, void *stream)
{
    RBF_REQUIRE(t != nullptr, "rbf_fmm_matvec: tree is NULL");
    RBF_REQUIRE(lambda && u, "rbf_fmm_matvec: NULL vector");
    RBF_REQUIRE(nrhs >= 1, "rbf_fmm_matvec: nrhs=%d", nrhs);
    RBF_REQUIRE(ld_lambda >= t->N && ld_u >= t->N, "rbf_fmm_matvec: leading dimension < N");
    cudaStream_t s = (cudaStream_t)stream;
    rbf_plan *p = nullptr;
    RBF_TRY(rbf_plan_get(t, kernel, eps, params, prec, s, &p));
    if (prec == RBF_FP32 && nrhs >= RBF_MULTI_RHS_MIN && rbf_far_multi_supported(p))
        return matvec_multi(t, p, kernel, eps, lambda, ld_lambda, u, ld_u, nrhs, s);
    for (int c = 0; c < nrhs; ++c) {
        const double *lc = lambda + (int64_t)c * ld_lambda;
        double *uc = u + (int64_t)c * ld_u;
        if (prec == RBF_FP64) RBF_TRY(matvec_one<double>(t, p, kernel, eps, lc, t->perm, uc, s));
        else RBF_TRY(matvec_one<float>(t, p, kernel, eps, lc, t->perm, uc, s));
    }
    return RBF_OK;
}

extern "C" int rbf_fmm_matvec_host(rbf_tree *t, rbf_kernel kernel, double eps,
                                   const rbf_fmm_params *params, rbf_precision prec,
                                   const double *lambda_host, double *u_host, int nrhs, void *stream)
{
    RBF_REQUIRE(t != nullptr, "rbf_fmm_matvec_host: tree is NULL");
    RBF_REQUIRE(lambda_host && u_host && nrhs >= 1, "rbf_fmm_matvec_host: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)t->N * nrhs * sizeof(double);
    if (t->scratch_bytes < 2 * bytes) {
        rbf_free(t->scratch);
        t->scratch = nullptr;
        t->scratch_bytes = 0;
        RBF_TRY(rbf_malloc(&t->scratch, 2 * bytes));
        t->scratch_bytes = 2 * bytes;
    }
    double *dl = (double *)t->scratch, *du = dl + (size_t)t->N * nrhs;
    RBF_CUDA_TRY(cudaMemcpyAsync(dl, lambda_host, bytes, cudaMemcpyHostToDevice, s));
    RBF_TRY(rbf_fmm_matvec(t, kernel, eps, params, prec, dl, t->N, du, t->N, nrhs, stream));
    RBF_CUDA_TRY(cudaMemcpyAsync(u_host, du, bytes, cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

extern "C" int rbf_check_device_waits(void)
{
    int flags = 0;
    RBF_TRY(rbf_tc_fetch_status(&flags));
    if (flags) {
        rbf_set_error("rbf_check_device_waits: a tensor-core kernel gave up waiting (flags %d)", flags);
        return RBF_ETIMEOUT;
    }
    return RBF_OK;
}
