/*
 * rbf_oracle.c -- plain FP64 CPU oracle for the band-limited FMM of
 * Zhao & Stoll, "A Fast Multipole Method based on Band-limited
 * Approximations for Radial Basis Functions" (arXiv 1606.07652).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load this
 * file: only tests/, the smoke check and bench.py's CPU-baseline leg do.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is FP64 and follows the paper's operators one by one:
 *   near field            Sec. 4, Eq. (38) first term, Eq. (54) sparse part
 *   aggregation (P2M)     Eq. (P2M):  V_b(xi) = sum_j lambda_j e^{-i xi.(x_j-c_b)}
 *   upsweep (M2M)         Eq. (43) with the interpolation P = identity
 *                         (one shared frequency grid on every level)
 *   coupling (M2L)        T_(a2b2) and Eq. (45): omega C(xi) e^{i xi.(c_a-c_b)}
 *   downsweep (L2L)       Eq. (48) with P = identity
 *   disaggregation (L2P)  Eq. (46): sum_xi e^{i xi.(x_i-c_a)} L_a(xi)
 * and the plain O(N^2) sum of Eq. (1).
 *
 * Frequency modes: the full symmetric tensor grid xi_k = k*dxi,
 * k = -M/2..M/2 in every dimension, flattened with dimension 0 fastest:
 * m = sum_t (k_t + M/2) (M+1)^t.  The quadrature weight omega and the
 * coefficient C(xi) arrive pre-multiplied (omegaC[m]) from the Python
 * side of the oracle.  A complex expansion is stored as C99
 * `double complex` (interleaved re, im).
 *
 * Parallelism: OpenMP `parallel for` over independent output boxes or
 * targets only; the arithmetic of every output is a plain serial loop.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_GAUSSIAN = 0, ORC_IMQ = 1, ORC_MQ = 2, ORC_WENDLAND = 3 };

/* Tables "Global functions" and "Compactly supported functions" (Sec. 2.2) in
 * the shape-parameter form: Phi(r) = exp(-(eps r)^2), 1/sqrt(1+(eps r)^2),
 * sqrt(1+(eps r)^2), and the compact Phi_{2,1}(eps r) = (1 - eps r)_+^3 (3 eps r + 1)
 * (the Wendland function of Sec. 5). */
double orc_phi(int kernel, double eps, double r)
{
    double er = eps * r;
    if (kernel == ORC_GAUSSIAN) return exp(-er * er);
    if (kernel == ORC_MQ) return sqrt(1.0 + er * er);
    if (kernel == ORC_WENDLAND) {
        double t = er < 1.0 ? 1.0 - er : 0.0;
        return t * t * t * (3.0 * er + 1.0);
    }
    return 1.0 / sqrt(1.0 + er * er);
}

static double dist(int d, const double *a, const double *b)
{
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
        double q = a[t] - b[t];
        s += q * q;
    }
    return sqrt(s);
}

/* Integer box coordinates from a Morton key at level l
 * (bit b of coordinate t sits at key bit b*d + t). */
static void key_coords(uint64_t key, int d, int l, int64_t *c)
{
    for (int t = 0; t < d; ++t) c[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t)
            c[t] |= (int64_t)((key >> (b * d + t)) & 1u) << b;
}

/* Centre of the level-l box with Morton key `key`:
 * c_t = lo_t + (k_t + 1/2) * side / 2^l. */
static void box_centre(uint64_t key, int d, int l, const double *lo, double side, double *c)
{
    int64_t k[8];
    key_coords(key, d, l, k);
    double w = side / (double)((int64_t)1 << l);
    for (int t = 0; t < d; ++t) c[t] = lo[t] + ((double)k[t] + 0.5) * w;
}

/* e^{sign i xi_m . r} for every mode m of the (M+1)^d grid, built from
 * e^{i xi.r} = prod_t e^{i xi_t r_t}.  xi1[k] holds the 1-D nodes. */
static void mode_phases(int d, int M, const double *xi1, const double *r, double sign,
                        double complex *out)
{
    int n1 = M + 1;
    int64_t stride = 1;
    out[0] = 1.0;
    for (int t = 0; t < d; ++t) {
        for (int k = n1 - 1; k >= 0; --k) {
            double complex ph = cexp(I * sign * xi1[k] * r[t]);
            for (int64_t m = 0; m < stride; ++m) out[k * stride + m] = out[m] * ph;
        }
        stride *= n1;
    }
}

static int64_t n_modes(int d, int M)
{
    int64_t n = 1;
    for (int t = 0; t < d; ++t) n *= (M + 1);
    return n;
}

/* ---- Eq. (1): direct sum u_i = sum_j lambda_j Phi(x_i - x_j) ---------- */
void orc_direct(int64_t N, int d, const double *X, const double *lam, int kernel, double eps,
                int64_t nt, const int64_t *targets, double *u)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nt; ++q) {
        const double *xi = X + targets[q] * d;
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) s += lam[j] * orc_phi(kernel, eps, dist(d, xi, X + j * d));
        u[q] = s;
    }
}

/* ---- Eq. (38) near field: sum over neighbour leaves b in N_a ------------
 * xs: sorted points [N][d]; leaf_off: point range of each non-empty leaf;
 * near_off/near_idx: CSR near lists (compact leaf ids).  u is overwritten. */
void orc_p2p(int d, int64_t nleaf, const int64_t *leaf_off, const int64_t *near_off,
             const int64_t *near_idx, const double *xs, const double *lam, int kernel, double eps,
             double *u)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nleaf; ++a) {
        for (int64_t i = leaf_off[a]; i < leaf_off[a + 1]; ++i) {
            double s = 0.0;
            for (int64_t e = near_off[a]; e < near_off[a + 1]; ++e) {
                int64_t b = near_idx[e];
                for (int64_t j = leaf_off[b]; j < leaf_off[b + 1]; ++j)
                    s += lam[j] * orc_phi(kernel, eps, dist(d, xs + i * d, xs + j * d));
            }
            u[i] = s;
        }
    }
}

/* ---- Eq. (P2M): V_b(xi) = sum_{j in G_b} lambda_j e^{-i xi.(x_j - c_b)} ---- */
void orc_p2m(int d, int M, const double *xi1, int64_t nbox, const uint64_t *box_key, int level,
             const double *lo, double side, const int64_t *pt_off, const double *xs,
             const double *lam, double complex *V)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < nbox; ++b) {
            double c[8], r[8];
            box_centre(box_key[b], d, level, lo, side, c);
            double complex *Vb = V + b * nm;
            for (int64_t m = 0; m < nm; ++m) Vb[m] = 0.0;
            for (int64_t j = pt_off[b]; j < pt_off[b + 1]; ++j) {
                for (int t = 0; t < d; ++t) r[t] = xs[j * d + t] - c[t];
                mode_phases(d, M, xi1, r, -1.0, E);
                for (int64_t m = 0; m < nm; ++m) Vb[m] += lam[j] * E[m];
            }
        }
        free(E);
    }
}

/* ---- Eq. (43), P = I: V_p(xi) = sum_{children c} e^{-i xi.(c_c - c_p)} V_c(xi)
 * Children of parent p are the child boxes child_off[p] .. child_off[p+1]-1. */
void orc_m2m(int d, int M, const double *xi1, int child_level, const double *lo, double side,
             int64_t nparent, const uint64_t *parent_key, const int64_t *child_off,
             const uint64_t *child_key, const double complex *Vc, double complex *Vp)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < nparent; ++p) {
            double cp[8], cc[8], r[8];
            box_centre(parent_key[p], d, child_level - 1, lo, side, cp);
            double complex *Vpp = Vp + p * nm;
            for (int64_t m = 0; m < nm; ++m) Vpp[m] = 0.0;
            for (int64_t c = child_off[p]; c < child_off[p + 1]; ++c) {
                box_centre(child_key[c], d, child_level, lo, side, cc);
                for (int t = 0; t < d; ++t) r[t] = cc[t] - cp[t];
                mode_phases(d, M, xi1, r, -1.0, E);
                for (int64_t m = 0; m < nm; ++m) Vpp[m] += E[m] * Vc[c * nm + m];
            }
        }
        free(E);
    }
}

/* ---- coupling, T_(ab) and Eq. (45): for every box a of this level
 *   L_a(xi) += sum_{b in IL(a)} omega C(xi) e^{i xi.(c_a - c_b)} V_b(xi). */
void orc_m2l(int d, int M, const double *xi1, const double *omegaC, int level, const double *lo,
             double side, int64_t nbox, const uint64_t *box_key, const int64_t *il_off,
             const int64_t *il_idx, const double complex *V, double complex *L)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t a = 0; a < nbox; ++a) {
            double ca[8], cb[8], r[8];
            box_centre(box_key[a], d, level, lo, side, ca);
            for (int64_t e = il_off[a]; e < il_off[a + 1]; ++e) {
                int64_t b = il_idx[e];
                box_centre(box_key[b], d, level, lo, side, cb);
                for (int t = 0; t < d; ++t) r[t] = ca[t] - cb[t];
                mode_phases(d, M, xi1, r, +1.0, E);
                for (int64_t m = 0; m < nm; ++m) L[a * nm + m] += omegaC[m] * E[m] * V[b * nm + m];
            }
        }
        free(E);
    }
}

/* ---- Eq. (48), P = I: L_c(xi) += e^{i xi.(c_c - c_p)} L_p(xi) ----------- */
void orc_l2l(int d, int M, const double *xi1, int child_level, const double *lo, double side,
             int64_t nchild, const uint64_t *child_key, const int64_t *child_parent,
             const uint64_t *parent_key, const double complex *Lp, double complex *Lc)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < nchild; ++c) {
            double cc[8], cp[8], r[8];
            int64_t p = child_parent[c];
            box_centre(child_key[c], d, child_level, lo, side, cc);
            box_centre(parent_key[p], d, child_level - 1, lo, side, cp);
            for (int t = 0; t < d; ++t) r[t] = cc[t] - cp[t];
            mode_phases(d, M, xi1, r, +1.0, E);
            for (int64_t m = 0; m < nm; ++m) Lc[c * nm + m] += E[m] * Lp[p * nm + m];
        }
        free(E);
    }
}

/* ---- Eq. (46): u_i += Re sum_xi e^{i xi.(x_i - c_a)} L_a(xi) ------------ */
void orc_l2p(int d, int M, const double *xi1, int64_t nbox, const uint64_t *box_key, int level,
             const double *lo, double side, const int64_t *pt_off, const double *xs,
             const double complex *L, double *u)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t a = 0; a < nbox; ++a) {
            double c[8], r[8];
            box_centre(box_key[a], d, level, lo, side, c);
            for (int64_t i = pt_off[a]; i < pt_off[a + 1]; ++i) {
                for (int t = 0; t < d; ++t) r[t] = xs[i * d + t] - c[t];
                mode_phases(d, M, xi1, r, +1.0, E);
                double complex s = 0.0;
                for (int64_t m = 0; m < nm; ++m) s += E[m] * L[a * nm + m];
                u[i] += creal(s);
            }
        }
        free(E);
    }
}

/* ---- Eq. (35): the far kernel K(r) = Re sum_xi omega C(xi) e^{i xi.r} ---- */
void orc_kernel_K(int d, int M, const double *xi1, const double *omegaC, int64_t nr,
                  const double *r, double *out)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < nr; ++q) {
            mode_phases(d, M, xi1, r + q * d, +1.0, E);
            double complex s = 0.0;
            for (int64_t m = 0; m < nm; ++m) s += omegaC[m] * E[m];
            out[q] = creal(s);
        }
        free(E);
    }
}

/* ---- Brute-force FMM on tiny inputs: every pair (i, j) is summed with Phi
 * when j's leaf is a near neighbour of i's leaf, and with K otherwise.
 * leaf_of[i]: compact leaf id of sorted point i; is_near(a, b) is read from
 * a dense nleaf x nleaf 0/1 matrix.  O(N^2 (M+1)^d). */
void orc_fmm_brute(int d, int M, const double *xi1, const double *omegaC, int64_t N,
                   const double *xs, const double *lam, const int64_t *leaf_of, int64_t nleaf,
                   const uint8_t *near_mat, int kernel, double eps, double *u)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                if (near_mat[leaf_of[i] * nleaf + leaf_of[j]]) {
                    s += lam[j] * orc_phi(kernel, eps, dist(d, xs + i * d, xs + j * d));
                } else {
                    double r[8];
                    for (int t = 0; t < d; ++t) r[t] = xs[i * d + t] - xs[j * d + t];
                    mode_phases(d, M, xi1, r, +1.0, E);
                    double complex k = 0.0;
                    for (int64_t m = 0; m < nm; ++m) k += omegaC[m] * E[m];
                    s += lam[j] * creal(k);
                }
            }
            u[i] = s;
        }
        free(E);
    }
}

/* ---- FMM output at selected targets, from its definition ---------------
 * u_i = sum_{j near} lambda_j Phi(x_i-x_j) + sum_{j far} lambda_j K(x_i-x_j),
 * with the far sum written as  Re sum_xi omega C e^{i xi.x_i}
 *   ( G(xi) - sum_{j near} lambda_j e^{-i xi.x_j} ),  G(xi) = sum_j lambda_j e^{-i xi.x_j}.
 * orc_global_G computes G; orc_fmm_at_targets evaluates the targets. */
void orc_global_G(int d, int M, const double *xi1, int64_t N, const double *xs, const double *lam,
                  double complex *G)
{
    int64_t nm = n_modes(d, M);
    for (int64_t m = 0; m < nm; ++m) G[m] = 0.0;
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
        double complex *Gp = calloc(nm, sizeof(double complex));
#pragma omp for schedule(static)
        for (int64_t j = 0; j < N; ++j) {
            mode_phases(d, M, xi1, xs + j * d, -1.0, E);
            for (int64_t m = 0; m < nm; ++m) Gp[m] += lam[j] * E[m];
        }
#pragma omp critical
        for (int64_t m = 0; m < nm; ++m) G[m] += Gp[m];
        free(E);
        free(Gp);
    }
}

void orc_fmm_at_targets(int d, int M, const double *xi1, const double *omegaC,
                        const double complex *G, const int64_t *leaf_off, const int64_t *near_off,
                        const int64_t *near_idx, const double *xs, const double *lam, int kernel,
                        double eps, int64_t nt, const int64_t *t_point, const int64_t *t_leaf,
                        double *u)
{
    int64_t nm = n_modes(d, M);
#pragma omp parallel
    {
        double complex *E = malloc(sizeof(double complex) * nm);
        double complex *R = malloc(sizeof(double complex) * nm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nt; ++q) {
            int64_t i = t_point[q], a = t_leaf[q];
            double s = 0.0;
            for (int64_t m = 0; m < nm; ++m) R[m] = G[m];
            for (int64_t e = near_off[a]; e < near_off[a + 1]; ++e) {
                int64_t b = near_idx[e];
                for (int64_t j = leaf_off[b]; j < leaf_off[b + 1]; ++j) {
                    s += lam[j] * orc_phi(kernel, eps, dist(d, xs + i * d, xs + j * d));
                    mode_phases(d, M, xi1, xs + j * d, -1.0, E);
                    for (int64_t m = 0; m < nm; ++m) R[m] -= lam[j] * E[m];
                }
            }
            mode_phases(d, M, xi1, xs + i * d, +1.0, E);
            double complex f = 0.0;
            for (int64_t m = 0; m < nm; ++m) f += omegaC[m] * E[m] * R[m];
            u[q] = s + creal(f);
        }
        free(E);
        free(R);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following parallel regions (timing of the oracle on 1 core) */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
