// plan.cu -- quadrature grid and coefficient tables of the band-limited
// expansion (Sec. 3.2 "Low-rank representation", Eqs. (quadrature),
// (M2Loperator), (28), (29)), built on the device in FP64 and stored in the
// arithmetic of the product.
//
// Grid: xi_k = k * 2pi/L, k = -M/2..M/2 per dimension, weight 2pi/L with half
// weight at k = +-M/2 (band limit sigma = pi M / L).  Coefficients from
// lattice samples (h = L/M):
//     C(xi) = (2pi)^-d h^d sum_{q in {-M/2..M/2-1}^d} f(q) e^{-i xi.qh},
//     f(q)  = sum_{n in {-1,0,1}^d} Phi(|qh + nL|) prod_t w(q_t h + n_t L),
// w the erfc taper (flat on |t| <= side).  f is even in every coordinate on
// the discrete torus, so the transform is a product of cosine sums, done one
// dimension at a time.  K(r) = sum omega C e^{i xi.r} is real and even, so an
// expansion keeps only k0 >= 0: the k0 > 0 half carries weight 2 (times the
// half weight at k0 = M/2), and the far value is the real part of the sum.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "rbf_internal.cuh"

namespace {

__device__ double phi64(int kernel, double eps, double r2) { return rbf_phi64(kernel, eps * eps * r2); }

__device__ double taper(double t, double L, double R_in, double alpha)
{
    if (alpha == 0.0) return 1.0;
    return 0.5 * erfc(alpha * (2.0 * (fabs(t) - R_in) / (L - 2.0 * R_in) - 1.0));
}

// f on the lattice, index sum_t (q_t + M/2) M^t (dimension 0 fastest)
__global__ void k_lattice(int kernel, double eps, int d, int M, double L, double alpha,
                          double R_in, double *f, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = L / M;
    double q[RBF_MAX_DIM];
    int64_t r = i;
    for (int t = 0; t < d; ++t) {
        q[t] = (double)((int)(r % M) - M / 2) * h;
        r /= M;
    }
    int nimg = 1;
    for (int t = 0; t < d; ++t) nimg *= 3;
    double s = 0.0;
    for (int c = 0; c < nimg; ++c) {
        int cc = c;
        double r2 = 0.0, w = 1.0;
        for (int t = 0; t < d; ++t) {
            double x = q[t] + (double)((cc % 3) - 1) * L;
            cc /= 3;
            r2 += x * x;
            w *= taper(x, L, R_in, alpha);
        }
        s += phi64(kernel, eps, r2) * w;
    }
    f[i] = s;
}

// One dimension of the cosine transform: in has shape s[0..d-1] (dimension 0
// fastest) with s[t] = M; out replaces dimension t by kh = 0..M/2:
//   out[.., k, ..] = sum_q in[.., q, ..] cos(2 pi k (q - M/2) / M).
__global__ void k_cos_pass(const double *in, double *out, int d, const int *shape_in, int t, int M,
                           int64_t nout)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nout) return;
    int64_t stride = 1;
    for (int u = 0; u < t; ++u) stride *= shape_in[u];
    const int kh = M / 2 + 1;
    int64_t lo = i % stride, rest = i / stride;
    int k = (int)(rest % kh);
    int64_t hi = rest / kh;
    const double *src = in + lo + hi * stride * M;
    double s = 0.0;
    for (int q = 0; q < M; ++q) s += src[(int64_t)q * stride] * cospi(2.0 * k * (q - M / 2) / (double)M);
    out[i] = s;
}

// Half-spectrum table: omegaC[m] = Wh(k0) prod_t omega(k_t) (2pi)^-d h^d Chalf[|k|]
template <typename R>
__global__ void k_fill_omegaC(const double *Chalf, int d, int M, double L, int closed, double eps,
                              R *omegaC, int64_t nmode)
{
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    const int n1 = M + 1, kh = M / 2 + 1;
    const double dxi = 2.0 * M_PI / L, h = L / M;
    int k[RBF_MAX_DIM];
    int64_t r = m;
    for (int t = d - 1; t >= 1; --t) {
        k[t] = (int)(r % n1) - M / 2;
        r /= n1;
    }
    k[0] = (int)r;  // 0..M/2
    double w = (k[0] == 0) ? 1.0 : 2.0;
    int64_t hidx = 0, hstride = 1;
    double xi2 = 0.0;
    for (int t = 0; t < d; ++t) {
        int a = k[t] < 0 ? -k[t] : k[t];
        w *= (a == M / 2) ? 0.5 * dxi : dxi;
        hidx += a * hstride;
        hstride *= kh;
        xi2 += (k[t] * dxi) * (k[t] * dxi);
    }
    double c;
    if (closed) {
        c = pow(M_PI / (eps * eps), 0.5 * d) * exp(-xi2 / (4.0 * eps * eps)) / pow(2.0 * M_PI, d);
    } else {
        c = Chalf[hidx] * pow(h, d) / pow(2.0 * M_PI, d);
    }
    omegaC[m] = (R)(w * c);
}

template <typename R>
__global__ void k_fill_xi(R *xi, int M, double L)
{
    int j = threadIdx.x;
    if (j <= M) xi[j] = (R)((j - M / 2) * (2.0 * M_PI / L));
}

// root_ph[t][kk][j] = e^{i xi_j ((kk + 1/2) w_D - side/2)}, kk = leaf coordinate
template <typename R>
__global__ void k_fill_root_ph(cplx<R> *ph, int d, int D, int M, double L, double side)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = M + 1;
    const int64_t nk = (int64_t)1 << D;
    if (i >= (int64_t)d * nk * n1) return;
    int j = (int)(i % n1);
    int64_t kk = (i / n1) % nk;
    double off = ((double)kk + 0.5) * (side / (double)nk) - 0.5 * side;
    double xi = (j - M / 2) * (2.0 * M_PI / L);
    double s, c;
    sincos(xi * off, &s, &c);
    ph[i].x = (R)c;
    ph[i].y = (R)s;
}

// shift_ph[l][j] = e^{-i xi_j w_l / 2}, w_l = side / 2^l, l = 0..D: the child-to-parent
// centre shift of M2M at child level l is row l; the leaf-neighbour phase e^{-i xi w_D} is
// the square of row D.
template <typename R>
__global__ void k_fill_shift_ph(cplx<R> *ph, int D, int M, double L, double side)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = M + 1;
    if (i >= (int64_t)(D + 1) * n1) return;
    const int j = (int)(i % n1);
    const int l = (int)(i / n1);
    const double w = side / (double)((int64_t)1 << l);
    const double xi = (j - M / 2) * (2.0 * M_PI / L);
    double s, c;
    sincos(-xi * 0.5 * w, &s, &c);
    ph[i].x = (R)c;
    ph[i].y = (R)s;
}

}  // namespace

void rbf_default_params(rbf_kernel kernel, double side, rbf_fmm_params *p)
{
    p->M = 32;
    p->period_L = 4.0 * side;
    p->window_alpha = kernel == RBF_GAUSSIAN ? 0.0 : 4.5;
    p->csample = 1;
    p->grid = RBF_GRID_SHARED;
    p->lagrange_K = 0;
}

void rbf_plan_free(rbf_plan *p)
{
    if (!p) return;
    rbf_free(p->omegaC);
    rbf_free(p->xi);
    rbf_free(p->root_ph);
    rbf_free(p->shift_ph);
    for (int l = 0; l <= RBF_MAX_DEPTH; ++l) rbf_free(p->V[l]);
    rbf_free(p->Lleaf);
    rbf_free(p->Vzero);
    rbf_free(p->lam_s);
    rbf_free(p->u_near);
    rbf_free(p->u_far);
    rbf_free(p->mr_V);
    rbf_free(p->mr_L);
    rbf_free(p->mr_lam);
    rbf_free(p->mr_un);
    rbf_free(p->mr_uf);
    rbf_free(p->mr_E);
    rbf_free(p->mr_Lt);
    rbf_nested_free(p);
    delete p;
}

// omegaC (half-spectrum weight * omega * C, nmode entries) of one grid: period L,
// taper flat on |t| <= R_in; written to dst in the arithmetic R
template <typename R>
static int make_omegaC(int d, int kernel, double eps, int M, double L, double alpha, double R_in,
                       int csample, int64_t nmode, R *dst, cudaStream_t s)
{
    double *Chalf = nullptr;
    if (!csample) {
        RBF_TRY(rbf_alloc(&Chalf, 1));
    } else {
        int64_t n = 1;
        for (int q = 0; q < d; ++q) n *= M;
        double *a = nullptr, *b = nullptr;
        RBF_TRY(rbf_alloc(&a, n));
        RBF_TRY(rbf_alloc(&b, n));
        k_lattice<<<ceil_div(n, 128), 128, 0, s>>>(kernel, eps, d, M, L, alpha, R_in, a, n);
        RBF_LAUNCH_CHECK();
        int shape[RBF_MAX_DIM];
        for (int q = 0; q < d; ++q) shape[q] = M;
        int *shape_d = nullptr;
        RBF_TRY(rbf_alloc(&shape_d, RBF_MAX_DIM));
        for (int q = 0; q < d; ++q) {
            RBF_CUDA_TRY(cudaMemcpyAsync(shape_d, shape, sizeof(shape), cudaMemcpyHostToDevice, s));
            int64_t nout = 1;
            for (int u = 0; u < d; ++u) nout *= (u == q) ? (M / 2 + 1) : shape[u];
            k_cos_pass<<<ceil_div(nout, 128), 128, 0, s>>>(a, b, d, shape_d, q, M, nout);
            RBF_LAUNCH_CHECK();
            RBF_CUDA_TRY(cudaStreamSynchronize(s));
            shape[q] = M / 2 + 1;
            std::swap(a, b);
        }
        Chalf = a;
        rbf_free(b);
        rbf_free(shape_d);
    }
    k_fill_omegaC<R><<<ceil_div(nmode, 256), 256, 0, s>>>(Chalf, d, M, L, !csample, eps, dst, nmode);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(Chalf);
    return RBF_OK;
}

template <typename R>
static int build_tables(rbf_tree *t, rbf_plan *p, cudaStream_t s)
{
    const int d = t->d, M = p->M;
    RBF_TRY(rbf_alloc(reinterpret_cast<R **>(&p->omegaC), p->nmode));
    RBF_TRY(make_omegaC<R>(d, p->kernel, p->eps, M, p->L, p->alpha, t->side, p->csample, p->nmode,
                           (R *)p->omegaC, s));
    RBF_TRY(rbf_alloc(reinterpret_cast<R **>(&p->xi), M + 1));
    k_fill_xi<R><<<1, 128, 0, s>>>((R *)p->xi, M, p->L);
    RBF_LAUNCH_CHECK();
    const int64_t nph = (int64_t)d * ((int64_t)1 << t->D) * (M + 1);
    RBF_TRY(rbf_alloc(reinterpret_cast<cplx<R> **>(&p->root_ph), nph));
    k_fill_root_ph<R><<<ceil_div(nph, 256), 256, 0, s>>>((cplx<R> *)p->root_ph, d, t->D, M, p->L,
                                                         t->side);
    RBF_LAUNCH_CHECK();
    // half shifts e^{-i xi w_l / 2} for every level l = 0..D (row l uses width side / 2^l)
    const int64_t nsh = (int64_t)(t->D + 1) * (M + 1);
    RBF_TRY(rbf_alloc(reinterpret_cast<cplx<R> **>(&p->shift_ph), nsh));
    k_fill_shift_ph<R><<<ceil_div(nsh, 256), 256, 0, s>>>((cplx<R> *)p->shift_ph, t->D, M, p->L, t->side);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

int rbf_make_omegaC(int prec, int d, int kernel, double eps, int M, double L, double alpha,
                    double R_in, int csample, int64_t nmode, void *dst, cudaStream_t s)
{
    if (prec == RBF_FP64)
        return make_omegaC<double>(d, kernel, eps, M, L, alpha, R_in, csample, nmode, (double *)dst, s);
    return make_omegaC<float>(d, kernel, eps, M, L, alpha, R_in, csample, nmode, (float *)dst, s);
}

template <typename R>
static int alloc_work(rbf_tree *t, rbf_plan *p)
{
    for (int l = 0; l <= t->D; ++l)
        RBF_TRY(rbf_alloc(reinterpret_cast<cplx<R> **>(&p->V[l]), (size_t)t->lev[l].nbox * p->mstride));
    RBF_TRY(rbf_alloc(reinterpret_cast<cplx<R> **>(&p->Lleaf), (size_t)t->nleaf() * p->mstride));
    RBF_TRY(rbf_alloc(reinterpret_cast<cplx<R> **>(&p->Vzero), (size_t)p->mstride));
    RBF_CUDA_TRY(cudaMemset(p->Vzero, 0, (size_t)p->mstride * sizeof(cplx<R>)));
    RBF_TRY(rbf_alloc(reinterpret_cast<R **>(&p->lam_s), t->N));
    RBF_TRY(rbf_alloc(reinterpret_cast<R **>(&p->u_near), t->N));
    RBF_TRY(rbf_alloc(reinterpret_cast<R **>(&p->u_far), t->N));
    return RBF_OK;
}

int rbf_plan_get(rbf_tree *t, rbf_kernel kernel, double eps, const rbf_fmm_params *pp, int prec,
                 cudaStream_t s, rbf_plan **out)
{
    rbf_fmm_params def;
    if (!pp) {
        rbf_default_params(kernel, t->side, &def);
        pp = &def;
    }
    RBF_REQUIRE(kernel >= RBF_GAUSSIAN && kernel <= RBF_WENDLAND, "unknown kernel %d", (int)kernel);
    RBF_REQUIRE(kernel != RBF_MQ || pp->window_alpha > 0.0,
                "the multiquadric grows with r: window_alpha must be > 0");
    RBF_REQUIRE(eps > 0.0 && std::isfinite(eps), "eps must be positive and finite");
    // M = 0: no far field (the product is the near field alone)
    RBF_REQUIRE(pp->M == 0 || (pp->M >= 2 && pp->M <= 64 && pp->M % 2 == 0),
                "M=%d must be 0 or even in [2, 64]", pp->M);
    RBF_REQUIRE(pp->M > 0 || pp->grid == RBF_GRID_SHARED, "M = 0 (no far field) needs the shared grid");
    RBF_REQUIRE(pp->window_alpha >= 0.0, "window_alpha must be >= 0");
    // far offsets reach |r_t| < side: the nearest image sits at >= L - side, and
    // the taper needs a transition zone L - 2 side > 0
    RBF_REQUIRE(pp->M == 0 || pp->period_L > (pp->window_alpha > 0.0 ? 2.0 : 1.0) * t->side,
                "period_L=%g must exceed %s the root side %g", pp->period_L,
                pp->window_alpha > 0.0 ? "twice" : "", t->side);
    RBF_REQUIRE(pp->csample == 0 || pp->csample == 1, "csample must be 0 or 1");
    RBF_REQUIRE(pp->csample == 1 || kernel == RBF_GAUSSIAN,
                "closed-form coefficients exist for the Gaussian only");
    RBF_REQUIRE(prec == RBF_FP64 || prec == RBF_FP32, "unknown precision %d", prec);
    RBF_REQUIRE(pp->grid == RBF_GRID_SHARED || pp->grid == RBF_GRID_NESTED, "unknown grid %d", pp->grid);
    const int lagK = pp->grid == RBF_GRID_NESTED ? (pp->lagrange_K ? pp->lagrange_K : 8) : 0;
    if (pp->grid == RBF_GRID_NESTED) {
        if (t->d > 3) {
            rbf_set_error("nested grids are built for d <= 3 (d = %d)", t->d);
            return RBF_ENOTSUP;
        }
        RBF_REQUIRE(lagK >= 2 && lagK <= 16 && lagK % 2 == 0, "lagrange_K=%d must be even in [2, 16]",
                    lagK);
        RBF_REQUIRE(pp->M >= 2 * lagK, "nested grids need M >= 2 lagrange_K (M=%d, K=%d)", pp->M, lagK);
        RBF_REQUIRE(pp->csample == 1 && pp->window_alpha > 0.0,
                    "nested grids need sampled coefficients and a taper (window_alpha > 0)");
    }
    rbf_plan *p = t->plan[prec];
    const int d = t->d, M = pp->M;
    int64_t nmode = M / 2 + 1;
    for (int q = 1; q < d; ++q) nmode *= (M + 1);
    if (M == 0) nmode = 0;
    if (p && p->kernel == kernel && p->eps == eps && p->M == M && p->L == pp->period_L &&
        p->alpha == pp->window_alpha && p->csample == pp->csample && p->grid == pp->grid &&
        p->lagK == lagK) {
        *out = p;
        return RBF_OK;
    }
    if (p && p->nmode != nmode) {
        rbf_plan_free(p);
        t->plan[prec] = p = nullptr;
    }
    bool fresh = (p == nullptr);
    if (fresh) p = new rbf_plan();
    else {
        rbf_free(p->omegaC);
        rbf_free(p->xi);
        rbf_free(p->root_ph);
        rbf_free(p->shift_ph);
        p->omegaC = p->xi = p->root_ph = p->shift_ph = nullptr;
        rbf_nested_free(p);
    }
    p->prec = prec;
    p->kernel = kernel;
    p->eps = eps;
    p->M = M;
    p->L = pp->period_L;
    p->alpha = pp->window_alpha;
    p->csample = pp->csample;
    p->grid = pp->grid;
    p->lagK = lagK;
    p->n0 = M / 2 + 1;
    p->n1 = M + 1;
    p->nmode = nmode;
    p->mstride = (nmode + 3) & ~(int64_t)3;
    if (d == 1) {
        p->nrow = 1;
        p->ncol = p->n0;
    } else {
        p->ncol = p->n1;
        p->nrow = (int)(nmode / p->n1);
    }
    if (M == 0) p->n0 = p->n1 = p->nrow = p->ncol = 0;
    int st = M == 0 ? RBF_OK
                    : (prec == RBF_FP64 ? build_tables<double>(t, p, s) : build_tables<float>(t, p, s));
    if (st == RBF_OK && fresh) st = prec == RBF_FP64 ? alloc_work<double>(t, p) : alloc_work<float>(t, p);
    if (st == RBF_OK && fresh && prec == RBF_FP32) {
        st = rbf_tune_p2m_shape(t, p, s);
        // RBF_P2M_SHAPE=1 (dense) or 2 (wide) replaces the measured choice of a plan
        // that measures one (tests compare the two shapes' bits)
        const char *env = std::getenv("RBF_P2M_SHAPE");
        const int forced = env ? std::atoi(env) : 0;
        if (st == RBF_OK && p->p2m_shape != 0 && (forced == 1 || forced == 2)) p->p2m_shape = forced;
    }
    if (st == RBF_OK && p->grid == RBF_GRID_NESTED) st = rbf_nested_build(t, p, s);
    if (st != RBF_OK) {
        rbf_plan_free(p);
        t->plan[prec] = nullptr;
        return st;
    }
    t->plan[prec] = p;
    *out = p;
    return RBF_OK;
}
