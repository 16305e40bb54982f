// precond.cu -- learned sparse approximate-inverse preconditioner for the
// interpolation solve.  Column i of P holds weights on the 32 nearest centres
// S_i of centre i, approximating the local cardinal function of i
// (sum_{j in S_i} c_j Phi(x_k - x_j) = delta_{ik} for k in S_i).  The weights
// come either from exact FP64 local solves or from the MLP (mlp.cu) applied
// to eps-scaled neighbour offsets; the network is trained here on exact local
// solves that the method itself generates.  GMRES uses A P (right
// preconditioning); the solve judges P by the FP64 residual and falls back to
// P = I (solve.cu).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "rbf_internal.cuh"

int rbf_radix_sort_pairs(uint64_t *keys, int32_t *vals, int64_t n, int nbits, cudaStream_t s);
int rbf_mlp_dims(const rbf_mlp *n, int *din, int *dout);
int rbf_mlp_forward_dev(rbf_mlp *n, const float *X, int64_t B, const float **Y, cudaStream_t s);
int rbf_mlp_train_step_impl(rbf_mlp *n, const float *X, const float *T, int64_t B, float lr,
                            float *loss, cudaStream_t s);

namespace {

constexpr int KNN = RBF_KNN;

__device__ __forceinline__ void decode_key(uint64_t key, int d, int l, int64_t *k)
{
    for (int t = 0; t < d; ++t) k[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) k[t] |= (int64_t)((key >> (b * d + t)) & 1u) << b;
}
__device__ __forceinline__ uint64_t encode_key(const int64_t *k, int d, int l)
{
    uint64_t key = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) key |= (uint64_t)((k[t] >> b) & 1) << (b * d + t);
    return key;
}
__device__ __forceinline__ int32_t find_leaf(const uint64_t *keys, int32_t n, uint64_t key)
{
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

// Exact k nearest neighbours of every sorted point: rings of leaves around the
// point's leaf are scanned until the k-th distance is certified by the distance
// from the point to the boundary of the scanned block.  Order: (squared
// distance, original index), distance summed in dimension order without FMA.
__global__ void k_knn(const double *xs, int64_t N, int d, int D, const double *lo, double side,
                      const uint64_t *keys, const uint64_t *leaf_key, const int32_t *leaf_off,
                      int32_t nleaf, const int32_t *perm, int32_t *nbr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double bd[KNN];
    int32_t bi[KNN], bo[KNN];
    int cnt = 0;
    double xi[RBF_MAX_DIM];
    for (int t = 0; t < d; ++t) xi[t] = xs[(int64_t)t * N + i];
    int64_t ka[RBF_MAX_DIM], kb[RBF_MAX_DIM];
    decode_key(keys[i], d, D, ka);
    const int64_t kmax = ((int64_t)1 << D) - 1;
    const double w = side / (double)((int64_t)1 << D);
    for (int r = 0; r <= kmax; ++r) {
        // leaves of the shell max_t |kb_t - ka_t| == r, enumerated over the (2r+1)^d block
        int64_t span = 2 * r + 1, total = 1;
        for (int t = 0; t < d; ++t) total *= span;
        for (int64_t c = 0; c < total; ++c) {
            int64_t cc = c;
            bool inside = true, shell = false;
            for (int t = 0; t < d; ++t) {
                int64_t o = cc % span - r;
                cc /= span;
                kb[t] = ka[t] + o;
                inside = inside && kb[t] >= 0 && kb[t] <= kmax;
                shell = shell || (o == r || o == -r);
            }
            if (!inside || (r > 0 && !shell)) continue;
            const int32_t b = find_leaf(leaf_key, nleaf, encode_key(kb, d, D));
            if (b < 0) continue;
            for (int32_t j = leaf_off[b]; j < leaf_off[b + 1]; ++j) {
                double d2 = 0.0;
                for (int t = 0; t < d; ++t) {
                    const double q = __dsub_rn(xs[(int64_t)t * N + j], xi[t]);
                    d2 = __dadd_rn(d2, __dmul_rn(q, q));
                }
                const int32_t oj = perm[j];
                if (cnt == KNN && (d2 > bd[KNN - 1] || (d2 == bd[KNN - 1] && oj > bo[KNN - 1])))
                    continue;
                int p = cnt < KNN ? cnt++ : KNN - 1;
                while (p > 0 && (bd[p - 1] > d2 || (bd[p - 1] == d2 && bo[p - 1] > oj))) {
                    bd[p] = bd[p - 1];
                    bi[p] = bi[p - 1];
                    bo[p] = bo[p - 1];
                    --p;
                }
                bd[p] = d2;
                bi[p] = j;
                bo[p] = oj;
            }
        }
        if (cnt == KNN) {
            // distance from the point to the boundary of the scanned block (sides on the
            // domain boundary do not limit: no point lies beyond them)
            double rho = INFINITY;
            for (int t = 0; t < d; ++t) {
                if (ka[t] - r > 0) rho = fmin(rho, xi[t] - (lo[t] + (double)(ka[t] - r) * w));
                if (ka[t] + r < kmax) rho = fmin(rho, (lo[t] + (double)(ka[t] + r + 1) * w) - xi[t]);
            }
            if (rho == INFINITY || bd[KNN - 1] < rho * rho) break;
        }
    }
    for (int q = 0; q < KNN; ++q) nbr[i * KNN + q] = q < cnt ? bi[q] : -1;
}

__device__ __forceinline__ double phi64(int kernel, double e2, double r2)
{
    return rbf_phi64(kernel, e2 * r2);
}

// One warp per listed centre: A_S + delta I (FP64, 32 x 32) in shared memory,
// Cholesky, then c = (A_S + delta I)^-1 e_1.  A failed pivot writes NaN.
__global__ void __launch_bounds__(128) k_cardinal(const double *xs, int64_t N, int d, int kernel,
                                                  double eps, double delta_rel, const int32_t *nbr,
                                                  const int32_t *centres, int64_t nc, double *cout)
{
    __shared__ double Ash[4][KNN][KNN + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * 4 + warp;
    if (q >= nc) return;
    const int32_t i = centres[q];
    double (*A)[KNN + 1] = Ash[warp];
    const int32_t jl = nbr[(int64_t)i * KNN + lane];
    double xl[RBF_MAX_DIM];
    for (int t = 0; t < d; ++t) xl[t] = xs[(int64_t)t * N + jl];
    const double e2 = eps * eps;
    double fro = 0.0;
    for (int c = 0; c < KNN; ++c) {
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) {
            const double xc = __shfl_sync(0xffffffffu, xl[t], c);
            const double df = xl[t] - xc;
            r2 += df * df;
        }
        const double a = phi64(kernel, e2, r2);
        A[lane][c] = a;
        fro += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    const double delta = delta_rel * sqrt(fro);
    A[lane][lane] += delta;
    __syncwarp();
    // Cholesky A = L L^T in place (lower triangle), lane = row
    bool ok = true;
    for (int k = 0; k < KNN; ++k) {
        const double pivot = A[k][k];
        ok = ok && pivot > 0.0;
        const double lkk = sqrt(fmax(pivot, 1e-300));
        __syncwarp();
        if (lane > k) A[lane][k] /= lkk;
        __syncwarp();
        if (lane == k) A[k][k] = lkk;
        __syncwarp();
        if (lane > k)
            for (int c = k + 1; c <= lane; ++c) A[lane][c] -= A[lane][k] * A[c][k];
        __syncwarp();
    }
    // forward solve L y = e_1, then L^T c = y (lane 0 runs the triangular solves)
    if (lane == 0) {
        double y[KNN];
        for (int r = 0; r < KNN; ++r) {
            double s = r == 0 ? 1.0 : 0.0;
            for (int c = 0; c < r; ++c) s -= A[r][c] * y[c];
            y[r] = s / A[r][r];
        }
        for (int r = KNN - 1; r >= 0; --r) {
            double s = y[r];
            for (int c = r + 1; c < KNN; ++c) s -= A[c][r] * y[c];
            y[r] = s / A[r][r];
        }
        for (int r = 0; r < KNN; ++r) cout[q * KNN + r] = ok ? y[r] : NAN;
    }
}

// features: eps * (x_j - x_i), neighbours in distance order, FP32
__global__ void k_features(const double *xs, int64_t N, int d, double eps, const int32_t *nbr,
                           const int32_t *rows, int64_t nr, float *F)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr * KNN) return;
    const int64_t r = q / KNN;
    const int k = (int)(q % KNN);
    const int32_t i = rows ? rows[r] : (int32_t)r;
    const int32_t j = nbr[(int64_t)i * KNN + k];
    for (int t = 0; t < d; ++t)
        F[(r * KNN + k) * d + t] = (float)(eps * (xs[(int64_t)t * N + j] - xs[(int64_t)t * N + i]));
}

// training targets: c / max_k |c_k| (FP32); rows with a failed solve are zeroed
__global__ void k_targets(const double *c, int64_t nc, float *T, int32_t *valid)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    double mx = 0.0;
    bool ok = true;
    for (int k = 0; k < KNN; ++k) {
        const double v = c[q * KNN + k];
        ok = ok && isfinite(v);
        mx = fmax(mx, fabs(v));
    }
    ok = ok && mx > 0.0;
    for (int k = 0; k < KNN; ++k) T[q * KNN + k] = ok ? (float)(c[q * KNN + k] / mx) : 0.0f;
    valid[q] = ok ? 1 : 0;
}

// weights of column i: w = s * chat with s = 1 / sum_j chat_j Phi(x_i - x_j) (cardinal at
// the centre itself); chat from FP64 solves (cd) or the network (cf)
__global__ void k_scale_columns(const double *xs, int64_t N, int d, int kernel, double eps,
                                const int32_t *nbr, const double *cd, const float *cf, double *W)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double e2 = eps * eps;
    double s = 0.0;
    for (int k = 0; k < KNN; ++k) {
        const int32_t j = nbr[i * KNN + k];
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) {
            const double df = xs[(int64_t)t * N + i] - xs[(int64_t)t * N + j];
            r2 += df * df;
        }
        const double c = cd ? cd[i * KNN + k] : (double)cf[i * KNN + k];
        s += c * phi64(kernel, e2, r2);
    }
    const bool ok = isfinite(s) && s != 0.0;
    for (int k = 0; k < KNN; ++k) {
        const double c = cd ? cd[i * KNN + k] : (double)cf[i * KNN + k];
        // a degenerate column keeps the identity
        W[i * KNN + k] = ok ? c / s : (k == 0 ? 1.0 : 0.0);
    }
}

__global__ void k_entry_keys(const int32_t *nbr, int64_t ne, uint64_t *key, int32_t *val)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    key[e] = (uint64_t)nbr[e];
    val[e] = (int32_t)e;
}

__global__ void k_row_starts(const uint64_t *key, int64_t ne, int32_t *row_off, int64_t N)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ne) return;
    const int64_t r = (int64_t)key[p];
    if (p == 0 || key[p - 1] != key[p]) row_off[r] = (int32_t)p;
    if (p == ne - 1) row_off[N] = (int32_t)ne;
}

// z[j] = sum over the entries of row j of w[e] y[col e]  (sorted order)
__global__ void k_apply_P(const int32_t *row_off, const int32_t *ent, const double *W, const double *y,
                          int64_t N, double *z)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int32_t p = row_off[j]; p < row_off[j + 1]; ++p) {
        const int32_t e = ent[p];
        s = fma(W[e], y[e / KNN], s);
    }
    z[j] = s;
}

__global__ void k_gather_rows(const int32_t *nbr, const int32_t *perm, int64_t N, int64_t *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N * KNN) return;
    const int64_t i = q / KNN;
    const int k = (int)(q % KNN);
    out[(int64_t)perm[i] * KNN + k] = perm[nbr[q]];
}

__global__ void k_inv_perm(const int32_t *perm, int64_t N, int32_t *inv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) inv[perm[i]] = (int32_t)i;
}

__global__ void k_permute64(const double *in, const int32_t *perm, int64_t N, double *out, int inverse)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (inverse) out[perm[i]] = in[i];
    else out[i] = in[perm[i]];
}

}  // namespace

// ----------------------------------------------------------- host side ----
int rbf_knn_build(rbf_tree *t, cudaStream_t s)
{
    if (t->pc.nbr) return RBF_OK;
    RBF_REQUIRE(t->N >= KNN, "k-nearest neighbours need N >= %d centres", KNN);
    double *lo_d = nullptr;
    RBF_TRY(rbf_alloc(&lo_d, RBF_MAX_DIM));
    RBF_CUDA_TRY(cudaMemcpyAsync(lo_d, t->lo, sizeof(t->lo), cudaMemcpyHostToDevice, s));
    RBF_TRY(rbf_alloc(&t->pc.nbr, (size_t)t->N * KNN));
    k_knn<<<ceil_div(t->N, 128), 128, 0, s>>>(t->xs64, t->N, t->d, t->D, lo_d, t->side, t->keys,
                                              t->leaf_key(), t->leaf_off, t->nleaf(), t->perm,
                                              t->pc.nbr);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(lo_d);
    return RBF_OK;
}

extern "C" int rbf_knn(rbf_tree *t, int64_t *idx_host, void *stream)
{
    RBF_REQUIRE(t && idx_host, "rbf_knn: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(rbf_knn_build(t, s));
    int64_t *tmp = nullptr;
    RBF_TRY(rbf_alloc(&tmp, (size_t)t->N * KNN));
    k_gather_rows<<<ceil_div(t->N * KNN, 256), 256, 0, s>>>(t->pc.nbr, t->perm, t->N, tmp);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaMemcpyAsync(idx_host, tmp, t->N * KNN * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(tmp);
    return RBF_OK;
}

// sorted ids of caller centres (original indices)
static int to_sorted_ids(rbf_tree *t, const int64_t *centres_host, int64_t nc, int32_t **out,
                         cudaStream_t s)
{
    int32_t *inv = nullptr;
    RBF_TRY(rbf_alloc(&inv, t->N));
    k_inv_perm<<<ceil_div(t->N, 256), 256, 0, s>>>(t->perm, t->N, inv);
    RBF_LAUNCH_CHECK();
    std::vector<int32_t> hinv(t->N);
    RBF_CUDA_TRY(cudaMemcpyAsync(hinv.data(), inv, t->N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(inv);
    std::vector<int32_t> ids(nc);
    for (int64_t q = 0; q < nc; ++q) {
        RBF_REQUIRE(centres_host[q] >= 0 && centres_host[q] < t->N, "centre index out of range");
        ids[q] = hinv[centres_host[q]];
    }
    RBF_TRY(rbf_alloc(out, std::max<int64_t>(nc, 1)));
    RBF_CUDA_TRY(cudaMemcpyAsync(*out, ids.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

extern "C" int rbf_cardinal_weights(rbf_tree *t, rbf_kernel kernel, double eps, double delta_rel,
                                    const int64_t *centres_host, int64_t nc, double *c_host,
                                    void *stream)
{
    RBF_REQUIRE(t && centres_host && c_host && nc >= 1, "rbf_cardinal_weights: bad arguments");
    RBF_REQUIRE(eps > 0.0 && delta_rel >= 0.0, "rbf_cardinal_weights: eps > 0, delta_rel >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(rbf_knn_build(t, s));
    int32_t *ids = nullptr;
    double *c = nullptr;
    RBF_TRY(to_sorted_ids(t, centres_host, nc, &ids, s));
    RBF_TRY(rbf_alloc(&c, (size_t)nc * KNN));
    k_cardinal<<<ceil_div(nc, 4), 128, 0, s>>>(t->xs64, t->N, t->d, kernel, eps, delta_rel, t->pc.nbr,
                                               ids, nc, c);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaMemcpyAsync(c_host, c, nc * KNN * sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(ids);
    rbf_free(c);
    return RBF_OK;
}

extern "C" int rbf_precond_features(rbf_tree *t, double eps, const int64_t *centres_host, int64_t nc,
                                    float *F, void *stream)
{
    RBF_REQUIRE(t && centres_host && F && nc >= 1, "rbf_precond_features: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(rbf_knn_build(t, s));
    int32_t *ids = nullptr;
    RBF_TRY(to_sorted_ids(t, centres_host, nc, &ids, s));
    k_features<<<ceil_div(nc * KNN, 256), 256, 0, s>>>(t->xs64, t->N, t->d, eps, t->pc.nbr, ids, nc, F);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(ids);
    return RBF_OK;
}

extern "C" int rbf_precond_train(rbf_tree *t, rbf_kernel kernel, double eps, rbf_mlp *net,
                                 const rbf_train_opts *o, rbf_train_report *rep, void *stream)
{
    RBF_REQUIRE(t && net && o, "rbf_precond_train: NULL argument");
    int din = 0, dout = 0;
    rbf_mlp_dims(net, &din, &dout);
    RBF_REQUIRE(din == KNN * t->d && dout == KNN, "network shape must be %d -> %d", KNN * t->d, KNN);
    RBF_REQUIRE(o->n_train >= 1 && o->epochs >= 1 && o->batch >= 1 && o->lr > 0.0f,
                "rbf_precond_train: bad options");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(rbf_knn_build(t, s));
    const int64_t nt = std::min<int64_t>(o->n_train, t->N);
    // training centres: evenly spaced in Morton order (spatially uniform coverage)
    std::vector<int32_t> hid(nt);
    for (int64_t q = 0; q < nt; ++q) hid[q] = (int32_t)((q * t->N) / nt);
    int32_t *ids = nullptr, *valid = nullptr;
    double *c = nullptr;
    float *F = nullptr, *T = nullptr;
    RBF_TRY(rbf_alloc(&ids, nt));
    RBF_TRY(rbf_alloc(&valid, nt));
    RBF_TRY(rbf_alloc(&c, (size_t)nt * KNN));
    RBF_TRY(rbf_alloc(&F, (size_t)nt * KNN * t->d));
    RBF_TRY(rbf_alloc(&T, (size_t)nt * KNN));
    RBF_CUDA_TRY(cudaMemcpyAsync(ids, hid.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_cardinal<<<ceil_div(nt, 4), 128, 0, s>>>(t->xs64, t->N, t->d, kernel, eps, o->delta_rel, t->pc.nbr,
                                               ids, nt, c);
    RBF_LAUNCH_CHECK();
    k_targets<<<ceil_div(nt, 256), 256, 0, s>>>(c, nt, T, valid);
    RBF_LAUNCH_CHECK();
    k_features<<<ceil_div(nt * KNN, 256), 256, 0, s>>>(t->xs64, t->N, t->d, eps, t->pc.nbr, ids, nt, F);
    RBF_LAUNCH_CHECK();
    float first = NAN, last = NAN;
    int steps = 0;
    const int64_t B = std::min<int64_t>(o->batch, nt);
    for (int ep = 0; ep < o->epochs; ++ep) {
        for (int64_t b0 = 0; b0 + B <= nt; b0 += B) {
            float loss = 0.0f;
            const bool want = (ep == 0 && b0 == 0) || (ep == o->epochs - 1 && b0 + 2 * B > nt);
            RBF_TRY(rbf_mlp_train_step_impl(net, F + b0 * KNN * t->d, T + b0 * KNN, B, o->lr,
                                            want ? &loss : nullptr, s));
            if (ep == 0 && b0 == 0) first = loss;
            if (want) last = loss;
            ++steps;
        }
    }
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(ids);
    rbf_free(valid);
    rbf_free(c);
    rbf_free(F);
    rbf_free(T);
    if (rep) {
        rep->loss_first = first;
        rep->loss_last = last;
        rep->steps = steps;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return RBF_OK;
}

extern "C" int rbf_precond_build(rbf_tree *t, rbf_kernel kernel, double eps, rbf_mlp *net,
                                 double delta_rel, void *stream)
{
    RBF_REQUIRE(t != nullptr, "rbf_precond_build: tree is NULL");
    RBF_REQUIRE(eps > 0.0 && delta_rel >= 0.0, "rbf_precond_build: eps > 0, delta_rel >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(rbf_knn_build(t, s));
    const int64_t N = t->N, ne = N * KNN;
    RBF_REQUIRE(ne < ((int64_t)1 << 31), "rbf_precond_build: N too large");
    if (!t->pc.W) {
        RBF_TRY(rbf_alloc(&t->pc.W, ne));
        RBF_TRY(rbf_alloc(&t->pc.row_off, N + 1));
        RBF_TRY(rbf_alloc(&t->pc.ent, ne));
    }
    if (net) {
        int din = 0, dout = 0;
        rbf_mlp_dims(net, &din, &dout);
        RBF_REQUIRE(din == KNN * t->d && dout == KNN, "network shape must be %d -> %d", KNN * t->d, KNN);
        // inference in chunks of rows
        const int64_t chunk = 1 << 16;
        float *F = nullptr, *Cf = nullptr;
        RBF_TRY(rbf_alloc(&F, (size_t)chunk * KNN * t->d));
        RBF_TRY(rbf_alloc(&Cf, (size_t)ne));
        for (int64_t r0 = 0; r0 < N; r0 += chunk) {
            const int64_t nr = std::min(chunk, N - r0);
            std::vector<int32_t> rows(nr);
            for (int64_t q = 0; q < nr; ++q) rows[q] = (int32_t)(r0 + q);
            int32_t *rd = nullptr;
            RBF_TRY(rbf_alloc(&rd, nr));
            RBF_CUDA_TRY(cudaMemcpyAsync(rd, rows.data(), nr * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            k_features<<<ceil_div(nr * KNN, 256), 256, 0, s>>>(t->xs64, N, t->d, eps, t->pc.nbr, rd, nr, F);
            RBF_LAUNCH_CHECK();
            const float *Y = nullptr;
            RBF_TRY(rbf_mlp_forward_dev(net, F, nr, &Y, s));
            RBF_CUDA_TRY(cudaMemcpyAsync(Cf + r0 * KNN, Y, nr * KNN * sizeof(float), cudaMemcpyDeviceToDevice, s));
            RBF_CUDA_TRY(cudaStreamSynchronize(s));
            rbf_free(rd);
        }
        k_scale_columns<<<ceil_div(N, 256), 256, 0, s>>>(t->xs64, N, t->d, kernel, eps, t->pc.nbr, nullptr,
                                                         Cf, t->pc.W);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        rbf_free(F);
        rbf_free(Cf);
    } else {
        // exact local cardinal solves for every centre
        double *c = nullptr;
        int32_t *ids = nullptr;
        RBF_TRY(rbf_alloc(&c, (size_t)ne));
        RBF_TRY(rbf_alloc(&ids, N));
        std::vector<int32_t> h(N);
        for (int64_t q = 0; q < N; ++q) h[q] = (int32_t)q;
        RBF_CUDA_TRY(cudaMemcpyAsync(ids, h.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k_cardinal<<<ceil_div(N, 4), 128, 0, s>>>(t->xs64, N, t->d, kernel, eps, delta_rel, t->pc.nbr, ids,
                                                  N, c);
        RBF_LAUNCH_CHECK();
        k_scale_columns<<<ceil_div(N, 256), 256, 0, s>>>(t->xs64, N, t->d, kernel, eps, t->pc.nbr, c,
                                                         nullptr, t->pc.W);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        rbf_free(c);
        rbf_free(ids);
    }
    // rows of P: a stable sort of the entries by row keeps columns ascending
    uint64_t *key = nullptr;
    RBF_TRY(rbf_alloc(&key, ne));
    k_entry_keys<<<ceil_div(ne, 256), 256, 0, s>>>(t->pc.nbr, ne, key, t->pc.ent);
    RBF_LAUNCH_CHECK();
    int nbits = 1;
    while (((int64_t)1 << nbits) < N) ++nbits;
    RBF_TRY(rbf_radix_sort_pairs(key, t->pc.ent, ne, nbits, s));
    k_row_starts<<<ceil_div(ne, 256), 256, 0, s>>>(key, ne, t->pc.row_off, N);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(key);
    t->pc.ready = true;
    t->pc.kernel = kernel;
    t->pc.eps = eps;
    return RBF_OK;
}

int rbf_precond_apply_sorted(const rbf_tree *t, const double *y, double *z, cudaStream_t s)
{
    k_apply_P<<<ceil_div(t->N, 256), 256, 0, s>>>(t->pc.row_off, t->pc.ent, t->pc.W, y, t->N, z);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

extern "C" int rbf_precond_apply(rbf_tree *t, const double *y, double *z, void *stream)
{
    RBF_REQUIRE(t && y && z, "rbf_precond_apply: NULL argument");
    RBF_REQUIRE(t->pc.ready, "rbf_precond_apply: no preconditioner built");
    cudaStream_t s = (cudaStream_t)stream;
    double *a = nullptr, *b = nullptr;
    RBF_TRY(rbf_alloc(&a, t->N));
    RBF_TRY(rbf_alloc(&b, t->N));
    k_permute64<<<ceil_div(t->N, 256), 256, 0, s>>>(y, t->perm, t->N, a, 0);
    RBF_TRY(rbf_precond_apply_sorted(t, a, b, s));
    k_permute64<<<ceil_div(t->N, 256), 256, 0, s>>>(b, t->perm, t->N, z, 1);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(a);
    rbf_free(b);
    return RBF_OK;
}

void rbf_precond_release(rbf_tree *t)
{
    rbf_free(t->pc.nbr);
    rbf_free(t->pc.W);
    rbf_free(t->pc.row_off);
    rbf_free(t->pc.ent);
    t->pc = rbf_precond_data();
}
