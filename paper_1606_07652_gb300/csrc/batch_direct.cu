// batch_direct.cu -- the plain sum of Eq. (1), u_i = sum_j lambda_j Phi(x_i - x_j),
// for every problem of a batch whose direct sum costs less than its FMM (small
// N, or kernels that need a high expansion order), in ONE persistent launch.
//
// Work list: items (problem, column group of 4 right-hand sides, tile of
// DB_T * TT targets), ordered by source count, largest first, so that the
// longest items start first and the tail is made of short ones.  Each CTA takes
// the next item from a device counter (atomicAdd; no CTA waits on another),
// keeps its TT targets per thread in registers, and streams the problem's
// sources through shared memory in chunks of DB_T points (coordinates and the
// four coefficients as 16-byte records, the next chunk prefetched into
// registers while the current one is summed).  Every shared-memory read is a
// broadcast and feeds TT pair evaluations.  Sums are two-level: a segment of
// DB_SEG sources into a fresh partial, partials into the total by compensated
// (Kahan) addition, so the rounding error does not grow with N (kernels like
// the multiquadric sum large terms of both signs).  Padded sources carry lambda = 0
// and finite coordinates, so every chunk runs the full unrolled loop.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "rbf_internal.cuh"

namespace {

constexpr int DB_T = 128;  // threads per CTA = sources per staged chunk
constexpr int DB_SEG = 16; // sources per partial sum (then added with compensation)

template <typename R>
struct V4t;
template <>
struct V4t<float> {
    using type = float4;
    static constexpr int TT = 4;  // targets per thread
};
template <>
struct V4t<double> {
    using type = double4_32a;
    static constexpr int TT = 2;
};

struct DirectArgs {
    const int4 *items;
    int nitems;
    int *ctr;
    const int64_t *N, *off, *xoff;
    const int *nrhs, *ker, *dim;
    const double *eps;
    const void *x;  // coordinate records, 4 per point, zero-padded
    const double *lam;
    double *u;
};

template <typename V>
__device__ __forceinline__ V v4_zero()
{
    V v;
    v.x = v.y = v.z = v.w = 0;
    return v;
}

template <typename R, int KER, int DIM>
__device__ __forceinline__ void direct_item(const DirectArgs &a, const int4 w,
                                            typename V4t<R>::type *sx,
                                            typename V4t<R>::type *sl)
{
    using V = typename V4t<R>::type;
    constexpr int TT = V4t<R>::TT;
    const int p = w.x, cg = w.y, t0 = w.z, tn = w.w;
    const int64_t N = a.N[p], off = a.off[p];
    const V *X = reinterpret_cast<const V *>(a.x) + a.xoff[p];
    const int nc = min(4, a.nrhs[p] - 4 * cg);
    const double *L = a.lam + off + (int64_t)4 * cg * N;
    // the coordinate records are pre-scaled by sqrt(e2) (k_pack_coords): Phi from phi_s
    constexpr R c0 = (R)phi_c0<KER>();
    R xt[TT][DIM];
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const int i = t0 + min((int)threadIdx.x + k * DB_T, tn - 1);
        const V v = X[i];
        xt[k][0] = v.x;
        if (DIM > 1) xt[k][1] = v.y;
        if (DIM > 2) xt[k][2] = v.z;
        if (DIM > 3) xt[k][DIM > 3 ? 3 : 0] = v.w;
    }
    R acc[TT][4], comp[TT][4];
#pragma unroll
    for (int k = 0; k < TT; ++k)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[k][r] = comp[k][r] = 0;
    V px, pl;
    auto fetch = [&](int64_t j0) {
        const int64_t j = j0 + threadIdx.x;
        if (j < N) {
            px = X[j];
            pl.x = (R)L[j];
            pl.y = nc > 1 ? (R)L[N + j] : (R)0;
            pl.z = nc > 2 ? (R)L[2 * N + j] : (R)0;
            pl.w = nc > 3 ? (R)L[3 * N + j] : (R)0;
        } else {
            px = v4_zero<V>();
            pl = v4_zero<V>();
        }
    };
    fetch(0);
    for (int64_t j0 = 0; j0 < N; j0 += DB_T) {
        __syncthreads();  // every thread is done with the previous chunk
        sx[threadIdx.x] = px;
        sl[threadIdx.x] = pl;
        __syncthreads();
        if (j0 + DB_T < N) fetch(j0 + DB_T);
        for (int s0 = 0; s0 < DB_T; s0 += DB_SEG) {
            R c[TT][4];
#pragma unroll
            for (int k = 0; k < TT; ++k)
#pragma unroll
                for (int r = 0; r < 4; ++r) c[k][r] = 0;
#pragma unroll 4
            for (int s = s0; s < s0 + DB_SEG; ++s) {
                const V xs = sx[s], ls = sl[s];
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    const R dx = xt[k][0] - xs.x;
                    R r2 = fma(dx, dx, c0);
                    if (DIM > 1) {
                        const R dy = xt[k][DIM > 1 ? 1 : 0] - xs.y;
                        r2 = fma(dy, dy, r2);
                    }
                    if (DIM > 2) {
                        const R dz = xt[k][DIM > 2 ? 2 : 0] - xs.z;
                        r2 = fma(dz, dz, r2);
                    }
                    if (DIM > 3) {
                        const R dw = xt[k][DIM > 3 ? 3 : 0] - xs.w;
                        r2 = fma(dw, dw, r2);
                    }
                    const R ph = phi_s<KER>(r2);
                    c[k][0] = fma(ph, ls.x, c[k][0]);
                    c[k][1] = fma(ph, ls.y, c[k][1]);
                    c[k][2] = fma(ph, ls.z, c[k][2]);
                    c[k][3] = fma(ph, ls.w, c[k][3]);
                }
            }
            // compensated (Kahan) addition of the segment's partial sums
#pragma unroll
            for (int k = 0; k < TT; ++k)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const R y = c[k][r] - comp[k][r];
                    const R t = acc[k][r] + y;
                    comp[k][r] = (t - acc[k][r]) - y;
                    acc[k][r] = t;
                }
        }
    }
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const int i = (int)threadIdx.x + k * DB_T;
        if (i < tn) {
            double *U = a.u + off + (int64_t)4 * cg * N + t0 + i;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < nc) U[(int64_t)r * N] = (double)acc[k][r];
        }
    }
}

template <typename R, int KER>
__device__ __forceinline__ void direct_item_dim(const DirectArgs &a, const int4 w, int dim,
                                                typename V4t<R>::type *sx,
                                                typename V4t<R>::type *sl)
{
    if (dim <= 2) direct_item<R, KER, 2>(a, w, sx, sl);
    else if (dim == 3) direct_item<R, KER, 3>(a, w, sx, sl);
    else direct_item<R, KER, 4>(a, w, sx, sl);
}

// persistent: one CTA per resident slot, items from a device counter
template <typename R>
__global__ void __launch_bounds__(DB_T) k_direct_batch(const DirectArgs a)
{
    using V = typename V4t<R>::type;
    __shared__ V sx[DB_T];
    __shared__ V sl[DB_T];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();  // s_item of the previous item has been read by every thread
        if (threadIdx.x == 0) s_item = atomicAdd(a.ctr, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) break;
        const int4 w = a.items[it];
        const int ker = a.ker[w.x], dim = a.dim[w.x];
        switch (ker) {
        case RBF_GAUSSIAN: direct_item_dim<R, RBF_GAUSSIAN>(a, w, dim, sx, sl); break;
        case RBF_IMQ: direct_item_dim<R, RBF_IMQ>(a, w, dim, sx, sl); break;
        case RBF_MQ: direct_item_dim<R, RBF_MQ>(a, w, dim, sx, sl); break;
        default: direct_item_dim<R, RBF_WENDLAND>(a, w, dim, sx, sl); break;
        }
    }
}

// records of 4 coordinates per point (zero-padded) from X [n][d] FP64, relative to
// the centre of the root cube [0,1]^d (so that the rounding is relative to half the
// cube) and scaled by sqrt(e2) of each precision (FP32 Gaussian: eps^2 log2(e), for
// exp2; else eps^2)
__global__ void k_pack_coords(const double *X, int64_t n, int d, double s64, double s32,
                              double4_32a *x64, float4 *x32)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = 0; t < d; ++t) v[t] = X[i * d + t] - 0.5;
    double4_32a r;
    r.x = s64 * v[0];
    r.y = s64 * v[1];
    r.z = s64 * v[2];
    r.w = s64 * v[3];
    x64[i] = r;
    x32[i] = make_float4((float)(s32 * v[0]), (float)(s32 * v[1]), (float)(s32 * v[2]),
                         (float)(s32 * v[3]));
}

template <typename R>
int resident_grid(int nitems)
{
    int dev = 0, nsm = 0, per = 0;
    RBF_CUDA_TRY(cudaGetDevice(&dev));
    RBF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RBF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_direct_batch<R>, DB_T, 0));
    return std::max(1, std::min(nitems, nsm * std::max(per, 1)));
}

}  // namespace

int rbf_direct_set_build(rbf_direct_set *ds, const rbf_problem *probs, const int64_t *off,
                         const std::vector<int> &which, cudaStream_t s)
{
    ds->np = (int)which.size();
    if (ds->np == 0) return RBF_OK;
    std::vector<int64_t> N(ds->np), o(ds->np), xo(ds->np);
    std::vector<int> nrhs(ds->np), ker(ds->np), dim(ds->np);
    std::vector<double> eps(ds->np);
    int64_t xtot = 0;
    for (int k = 0; k < ds->np; ++k) {
        const rbf_problem &q = probs[which[k]];
        RBF_REQUIRE(q.d >= 1 && q.d <= 4, "direct set: problem %d has d = %d > 4", which[k], q.d);
        N[k] = q.N;
        o[k] = off[which[k]];
        xo[k] = xtot;
        xtot += q.N;
        nrhs[k] = q.nrhs;
        ker[k] = (int)q.kernel;
        dim[k] = q.d;
        eps[k] = q.eps;
    }
    RBF_REQUIRE(xtot < (int64_t)INT32_MAX, "direct set: too many points");
    // items: largest source count first; within a problem, column groups then tiles
    std::vector<int> order(ds->np);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return N[a] > N[b]; });
    std::vector<int4> items;
    for (int k : order) {
        const int ncg = (nrhs[k] + 3) / 4;
        for (int cg = 0; cg < ncg; ++cg) {
            for (int64_t t0 = 0; t0 < N[k]; t0 += (int64_t)DB_T * 4)
                items.push_back(make_int4(k, cg, (int)t0, (int)std::min<int64_t>(DB_T * 4, N[k] - t0)));
        }
    }
    // the FP64 kernel takes half the targets per thread: split its tiles in two
    std::vector<int4> items64;
    for (const int4 &w : items) {
        for (int h = 0; h < w.w; h += DB_T * 2)
            items64.push_back(make_int4(w.x, w.y, w.z + h, std::min(DB_T * 2, w.w - h)));
    }
    ds->nitems = (int)items.size();
    ds->nitems64 = (int)items64.size();
    RBF_TRY(rbf_alloc(&ds->items, items.size() + items64.size()));
    RBF_TRY(rbf_alloc(&ds->ctr, 2));
    RBF_TRY(rbf_alloc(&ds->N, ds->np));
    RBF_TRY(rbf_alloc(&ds->off, ds->np));
    RBF_TRY(rbf_alloc(&ds->xoff, ds->np));
    RBF_TRY(rbf_alloc(&ds->nrhs, ds->np));
    RBF_TRY(rbf_alloc(&ds->ker, ds->np));
    RBF_TRY(rbf_alloc(&ds->dim, ds->np));
    RBF_TRY(rbf_alloc(&ds->eps, ds->np));
    RBF_TRY(rbf_alloc(&ds->x64, (size_t)xtot * 4));
    RBF_TRY(rbf_alloc(&ds->x32, (size_t)xtot));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->items, items.data(), items.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->items + items.size(), items64.data(),
                                 items64.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->N, N.data(), ds->np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->off, o.data(), ds->np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->xoff, xo.data(), ds->np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->nrhs, nrhs.data(), ds->np * sizeof(int), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->ker, ker.data(), ds->np * sizeof(int), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->dim, dim.data(), ds->np * sizeof(int), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(ds->eps, eps.data(), ds->np * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < ds->np; ++k) {
        const rbf_problem &q = probs[which[k]];
        const double s32 = q.kernel == RBF_GAUSSIAN ? q.eps * std::sqrt(1.4426950408889634) : q.eps;
        k_pack_coords<<<ceil_div(q.N, 256), 256, 0, s>>>(
            q.X, q.N, q.d, q.eps, s32, reinterpret_cast<double4_32a *>(ds->x64) + xo[k],
            ds->x32 + xo[k]);
        RBF_LAUNCH_CHECK();
    }
    ds->grid32 = resident_grid<float>(ds->nitems);
    ds->grid64 = resident_grid<double>(ds->nitems64);
    RBF_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors above go out of scope
    return RBF_OK;
}

int rbf_direct_set_run(const rbf_direct_set *ds, int prec, const double *lam, double *u,
                       cudaStream_t s)
{
    if (ds->np == 0) return RBF_OK;
    DirectArgs a;
    a.N = ds->N;
    a.off = ds->off;
    a.xoff = ds->xoff;
    a.nrhs = ds->nrhs;
    a.ker = ds->ker;
    a.dim = ds->dim;
    a.eps = ds->eps;
    a.lam = lam;
    a.u = u;
    if (prec == RBF_FP32) {
        a.items = ds->items;
        a.nitems = ds->nitems;
        a.ctr = ds->ctr;
        a.x = ds->x32;
        RBF_CUDA_TRY(cudaMemsetAsync(ds->ctr, 0, sizeof(int), s));
        k_direct_batch<float><<<ds->grid32, DB_T, 0, s>>>(a);
    } else {
        a.items = ds->items + ds->nitems;
        a.nitems = ds->nitems64;
        a.ctr = ds->ctr + 1;
        a.x = ds->x64;
        RBF_CUDA_TRY(cudaMemsetAsync(ds->ctr + 1, 0, sizeof(int), s));
        k_direct_batch<double><<<ds->grid64, DB_T, 0, s>>>(a);
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

void rbf_direct_set_free(rbf_direct_set *ds)
{
    rbf_free(ds->items);
    rbf_free(ds->ctr);
    rbf_free(ds->N);
    rbf_free(ds->off);
    rbf_free(ds->xoff);
    rbf_free(ds->nrhs);
    rbf_free(ds->ker);
    rbf_free(ds->dim);
    rbf_free(ds->eps);
    rbf_free(ds->x64);
    rbf_free(ds->x32);
    *ds = rbf_direct_set();
}
