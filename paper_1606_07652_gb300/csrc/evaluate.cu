// evaluate.cu -- the FMM product at points that are not centres:
//   s(y) = sum_j lambda_j Phi(y - x_j)                       (Eq. (1), y != x_j)
// The centres and the new points share one tree (the source tree's root cube
// and depth), so every pair (y, x_j) is classified and approximated exactly as
// a pair of centres would be: near field over neighbour leaves (Eq. (38)), far
// field through P2M / M2M / M2L / L2L / L2P (Eqs. (43)-(48)).  The new points
// carry zero coefficients; their outputs are the evaluation.
#include "rbf_internal.cuh"

struct rbf_eval {
    rbf_tree *ct = nullptr;   // centres followed by the new points
    int64_t N = 0, nt = 0;
    int d = 0;
    double *lam = nullptr;    // [(N + nt) * ncap] coefficients, zero on the new points
    double *u = nullptr;      // [(N + nt) * ncap] products
    int ncap = 0;             // columns the buffers hold
};

namespace {

// Xc[perm[i]][t] = xs[t][i] (centres back in the caller's order), then the new points;
// flag = 1 when a new point lies outside [lo, lo + side]^d
__global__ void k_combine(const double *xs, const int32_t *perm, int64_t N, const double *Y,
                          int64_t nt, int d, double lo0, double lo1, double lo2, double lo3,
                          double lo4, double lo5, double side, double *Xc, int *flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const int64_t dst = perm[i];
        for (int t = 0; t < d; ++t) Xc[dst * d + t] = xs[(int64_t)t * N + i];
    } else if (i < N + nt) {
        const int64_t q = i - N;
        const double lo[6] = {lo0, lo1, lo2, lo3, lo4, lo5};
        bool out = false;
        for (int t = 0; t < d; ++t) {
            const double y = Y[q * d + t];
            Xc[i * d + t] = y;
            out |= !(y >= lo[t] && y <= lo[t] + side);
        }
        if (out) atomicOr(flag, 1);
    }
}

// column c: lam[c][0..N) = lambda[c * ld + ..], lam[c][N..N+nt) = 0
__global__ void k_pad(const double *lambda, int64_t ld, int64_t N, int64_t nt, int nrhs, double *lam)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = N + nt;
    if (i >= tot * nrhs) return;
    const int64_t c = i / tot, j = i - c * tot;
    lam[i] = j < N ? lambda[c * ld + j] : 0.0;
}

__global__ void k_take(const double *u, int64_t N, int64_t nt, int nrhs, double *s, int64_t ld)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt * nrhs) return;
    const int64_t c = i / nt, q = i - c * nt;
    s[c * ld + q] = u[c * (N + nt) + N + q];
}

}  // namespace

extern "C" int rbf_eval_create(const rbf_tree *t, const double *Y, int64_t nt, void *stream,
                               rbf_eval **out)
{
    RBF_REQUIRE(out != nullptr, "rbf_eval_create: out is NULL");
    *out = nullptr;
    RBF_REQUIRE(t && Y, "rbf_eval_create: NULL argument");
    RBF_REQUIRE(nt >= 1 && t->N + nt < ((int64_t)1 << 31), "rbf_eval_create: nt=%lld",
                (long long)nt);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tot = t->N + nt;
    const int d = t->d;
    double *Xc = nullptr;
    int *flag = nullptr;
    RBF_TRY(rbf_alloc(&Xc, (size_t)tot * d));
    int st = rbf_alloc(&flag, 1);
    int hflag = 0;
    if (st == RBF_OK) {
        double lo[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < d; ++q) lo[q] = t->lo[q];
        const bool zeroed = cudaMemsetAsync(flag, 0, sizeof(int), s) == cudaSuccess;
        if (zeroed)
            k_combine<<<ceil_div(tot, 256), 256, 0, s>>>(t->xs64, t->perm, t->N, Y, nt, d, lo[0], lo[1],
                                                         lo[2], lo[3], lo[4], lo[5], t->side, Xc, flag);
        if (!zeroed || cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rbf_set_error("rbf_eval_create: CUDA failure while combining the points");
            st = RBF_ECUDA;
        } else if (hflag) {
            rbf_set_error("rbf_eval_create: a new point lies outside the tree's root cube");
            st = RBF_EINVAL;
        }
    }
    rbf_eval *e = nullptr;
    if (st == RBF_OK) {
        e = new rbf_eval();
        e->N = t->N;
        e->nt = nt;
        e->d = d;
        st = rbf_tree_build(Xc, tot, d, t->lo, t->side, t->D, stream, &e->ct);
    }
    rbf_free(Xc);
    rbf_free(flag);
    if (st != RBF_OK) {
        rbf_eval_free(e);
        return st;
    }
    *out = e;
    return RBF_OK;
}

extern "C" int rbf_eval_apply(rbf_eval *e, rbf_kernel kernel, double eps, const rbf_fmm_params *params,
                              rbf_precision prec, const double *lambda, int64_t ld_lambda, double *s_out,
                              int64_t ld_s, int nrhs, void *stream)
{
    RBF_REQUIRE(e && e->ct && lambda && s_out, "rbf_eval_apply: NULL argument");
    RBF_REQUIRE(nrhs >= 1 && ld_lambda >= e->N && ld_s >= e->nt, "rbf_eval_apply: bad sizes");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tot = e->N + e->nt;
    if (e->ncap < nrhs) {
        rbf_free(e->lam);
        rbf_free(e->u);
        e->lam = e->u = nullptr;
        e->ncap = 0;
        RBF_TRY(rbf_alloc(&e->lam, (size_t)tot * nrhs));
        RBF_TRY(rbf_alloc(&e->u, (size_t)tot * nrhs));
        e->ncap = nrhs;
    }
    k_pad<<<ceil_div(tot * nrhs, 256), 256, 0, s>>>(lambda, ld_lambda, e->N, e->nt, nrhs, e->lam);
    RBF_LAUNCH_CHECK();
    RBF_TRY(rbf_fmm_matvec(e->ct, kernel, eps, params, prec, e->lam, tot, e->u, tot, nrhs, stream));
    k_take<<<ceil_div(e->nt * nrhs, 256), 256, 0, s>>>(e->u, e->N, e->nt, nrhs, s_out, ld_s);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

extern "C" void rbf_eval_free(rbf_eval *e)
{
    if (!e) return;
    rbf_tree_free(e->ct);
    rbf_free(e->lam);
    rbf_free(e->u);
    delete e;
}
