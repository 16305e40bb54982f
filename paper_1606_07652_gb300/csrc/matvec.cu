// matvec.cu -- u = A lambda (Eq. (54)): near field + far field, in the
// caller's order (entry points) or in Morton order (solver).
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
    const bool far = t->D >= 2;
    if (far) RBF_TRY(rbf_run_far<R>(t, p, lam_s, uf, s));
    {
        rbf_pass_timer tm(t, RBF_PASS_PERM, s);
        k_scatter<R><<<ceil_div(N, 256), 256, 0, s>>>(un, far ? uf : nullptr, perm, N, u);
        RBF_LAUNCH_CHECK();
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
