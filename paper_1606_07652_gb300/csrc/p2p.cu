// p2p.cu -- near field of Eq. (38) (the sparse part A^diag + A^near-diag of
// Eq. (54)) and the plain O(N^2) sum of Eq. (1).
//
// Near field: one CTA per target leaf a.  The points of the neighbour leaves
// N_a are staged from HBM into shared memory in chunks (coordinates and lambda
// as one 16-byte record per point in FP32, two in FP64); each warp takes a
// quarter of the staged sources, lane = target, so every shared-memory read is
// a broadcast.  The four partial sums of a target are added in a fixed order.
#include <algorithm>
#include <type_traits>

#include "rbf_internal.cuh"

namespace {

constexpr int P2P_THREADS = 128;
constexpr int P2P_WARPS = P2P_THREADS / 32;
constexpr int P2P_STAGE_BYTES = 16384;         // shared memory for staged sources
#ifndef RBF_P2P_SU
#define RBF_P2P_SU 4                           // sources per step (independent partial sums)
#endif
#ifndef RBF_P2P_TGMAX
#define RBF_P2P_TGMAX 4                        // target groups of 32 per pass, at most
#endif
#ifndef RBF_P2P_TT
#define RBF_P2P_TT 2                           // targets per thread of the split kernel
#endif
#ifndef RBF_P2P_SMALL
#define RBF_P2P_SMALL 64                       // leaves up to this size: one group per pass
#endif

template <typename R>
struct Src4;
template <>
struct Src4<float> {
    using type = float4;
};
template <>
struct Src4<double> {
    using type = double4_32a;
};

// f(std::integral_constant<int, K>) for the run-time kernel id K
template <typename F>
int with_kernel(int kernel, F f)
{
    switch (kernel) {
    case RBF_GAUSSIAN: return f(std::integral_constant<int, RBF_GAUSSIAN>());
    case RBF_IMQ: return f(std::integral_constant<int, RBF_IMQ>());
    case RBF_MQ: return f(std::integral_constant<int, RBF_MQ>());
    case RBF_WENDLAND: return f(std::integral_constant<int, RBF_WENDLAND>());
    default:
        rbf_set_error("p2p: unknown kernel %d", kernel);
        return RBF_EINVAL;
    }
}

// The source ranges of a target leaf's neighbours (near list entries e0 ..
// e0 + ne - 1): rstart[e] = first point of neighbour e, rpre[e] = points of the
// neighbours before it, rpre[ne] = all of them.  Warp 0 loads 32 entries at a
// time in parallel and prefix-sums their lengths with shuffles, so the
// neighbour loads are in flight together.  Ends with __syncthreads().
__device__ __forceinline__ void near_ranges(int e0, int ne, const int32_t *near_idx,
                                            const int32_t *leaf_off, int32_t *rstart,
                                            int32_t *rlen, int32_t *rpre)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int carry = 0;
        for (int c0 = 0; c0 < ne; c0 += 32) {
            const int e = c0 + lane;
            int st = 0, len = 0;
            if (e < ne) {
                const int b = near_idx[e0 + e];
                st = leaf_off[b];
                len = leaf_off[b + 1] - st;
            }
            int inc = len;  // inclusive scan over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            if (e < ne) {
                rstart[e] = st;
                if (rlen) rlen[e] = len;
                rpre[e] = carry + inc - len;
            }
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) rpre[ne] = carry;
    }
    __syncthreads();
}

template <typename R, int DIM, int TG, int KER>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p(R e2, int64_t N, const R *xs,
                                                     const R *lam, const int32_t *leaf_off,
                                                     const int32_t *near_off,
                                                     const int32_t *near_idx, R *u)
{
    using S4 = typename Src4<R>::type;
    // per source: (x0, x1, x2, lambda) for DIM <= 3; DIM > 3 uses two records
    constexpr int REC = DIM <= 3 ? 1 : 2;
    constexpr int P2P_SCHUNK = P2P_STAGE_BYTES / (int)(sizeof(S4) * REC);
    constexpr int TB = 32 * TG;   // targets per pass
    constexpr int SU = RBF_P2P_SU;   // sources per iteration, one partial sum each
    __shared__ S4 src[P2P_SCHUNK * REC];
    __shared__ int32_t rstart[729], rlen[729], rpre[730];
    __shared__ R red[P2P_WARPS][TB];
    const int a = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e0 = near_off[a], ne = near_off[a + 1] - e0;
    near_ranges(e0, ne, near_idx, leaf_off, rstart, rlen, rpre);
    const int nsrc = rpre[ne];
    const int t0 = leaf_off[a], nt = leaf_off[a + 1] - t0;
    // coordinates relative to the leaf's first point, then scaled: Phi from
    // phi_s(c0 + sum d^2), rounding relative to the neighbourhood's size
    const R sc = sqrt(e2);
    R org[DIM];
#pragma unroll
    for (int t = 0; t < DIM; ++t) org[t] = xs[(int64_t)t * N + t0];
    for (int tb = 0; tb < nt; tb += TB) {
        R xt[TG][DIM];
        R acc[TG][SU];
#pragma unroll
        for (int g = 0; g < TG; ++g) {
            int i = tb + g * 32 + lane;
#pragma unroll
            for (int k = 0; k < SU; ++k) acc[g][k] = (R)0;
#pragma unroll
            for (int t = 0; t < DIM; ++t) xt[g][t] = i < nt ? sc * (xs[(int64_t)t * N + t0 + i] - org[t]) : (R)0;
        }
        for (int s0 = 0; s0 < nsrc; s0 += P2P_SCHUNK) {
            const int cnt = min(P2P_SCHUNK, nsrc - s0);
            __syncthreads();
            for (int v = threadIdx.x; v < cnt; v += P2P_THREADS) {
                // virtual source index -> neighbour range (<= 3^d ranges)
                int vv = s0 + v, lo = 0, hi = ne - 1;
                while (lo < hi) {  // last range with rpre[e] <= vv
                    int mid = (lo + hi + 1) >> 1;
                    if (rpre[mid] <= vv) lo = mid;
                    else hi = mid - 1;
                }
                const int e = lo;
                int64_t j = rstart[e] + (vv - rpre[e]);
                R c[8] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
#pragma unroll
                for (int t = 0; t < DIM; ++t) c[t] = sc * (xs[(int64_t)t * N + j] - org[t]);
                if (REC == 1) {
                    S4 r;
                    r.x = c[0];
                    r.y = c[1];
                    r.z = c[2];
                    r.w = lam[j];
                    src[v] = r;
                } else {
                    S4 r0, r1;
                    r0.x = c[0];
                    r0.y = c[1];
                    r0.z = c[2];
                    r0.w = lam[j];
                    r1.x = c[3];
                    r1.y = c[4];
                    r1.z = c[5];
                    r1.w = (R)0;
                    src[2 * v] = r0;
                    src[2 * v + 1] = r1;
                }
            }
            // pad the chunk to a multiple of SU sources per warp stride with zero weights
            for (int v = cnt + threadIdx.x; v < cnt + P2P_WARPS * SU; v += P2P_THREADS) {
                if (v < P2P_SCHUNK) {
                    S4 z;
                    z.x = z.y = z.z = z.w = (R)0;
                    src[REC * v] = z;
                    if (REC == 2) src[REC * v + 1] = z;
                }
            }
            __syncthreads();
            // warp w takes sources w*SU + k + j*(WARPS*SU), k < SU: SU independent pairs per step
            for (int j0 = warp * SU; j0 < cnt; j0 += P2P_WARPS * SU) {
#pragma unroll
                for (int k = 0; k < SU; ++k) {
                    const int j = min(j0 + k, P2P_SCHUNK - 1);
                    const S4 r0 = src[REC * j];
                    S4 r1;
                    if (REC == 2) r1 = src[REC * j + 1];
                    const R wgt = j0 + k < cnt ? r0.w : (R)0;
#pragma unroll
                    for (int g = 0; g < TG; ++g) {
                        R d0 = xt[g][0] - r0.x;
                        R r2 = fma(d0, d0, (R)phi_c0<KER>());
                        if (DIM > 1) {
                            R d1 = xt[g][DIM > 1 ? 1 : 0] - r0.y;
                            r2 = fma(d1, d1, r2);
                        }
                        if (DIM > 2) {
                            R d2 = xt[g][DIM > 2 ? 2 : 0] - r0.z;
                            r2 = fma(d2, d2, r2);
                        }
                        if (DIM > 3) {
                            R d3 = xt[g][DIM > 3 ? 3 : 0] - r1.x;
                            r2 = fma(d3, d3, r2);
                        }
                        if (DIM > 4) {
                            R d4 = xt[g][DIM > 4 ? 4 : 0] - r1.y;
                            r2 = fma(d4, d4, r2);
                        }
                        if (DIM > 5) {
                            R d5 = xt[g][DIM > 5 ? 5 : 0] - r1.z;
                            r2 = fma(d5, d5, r2);
                        }
                        acc[g][k] = fma(wgt, phi_s<KER>(r2), acc[g][k]);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int g = 0; g < TG; ++g)
        {
            R t = acc[g][0];
#pragma unroll
            for (int k = 1; k < SU; ++k) t += acc[g][k];
            red[warp][g * 32 + lane] = t;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < min(TB, nt - tb); i += P2P_THREADS) {
            R s = red[0][i];
#pragma unroll
            for (int w = 1; w < P2P_WARPS; ++w) s += red[w][i];
            u[t0 + tb + i] = s;
        }
    }
}

// Leaves of at most P2P_THREADS points: the CTA's threads are (target group,
// source split) pairs.  A group holds TT targets (g, g + ng, ... with ng =
// ceil(nt / TT) groups), so every staged source read feeds TT pair evaluations;
// nsplit = floor(P2P_THREADS / ng) splits of the staged sources, so that nearly
// every lane works whatever the leaf size and the sources are staged once.
// Thread tid takes group tid % ng and split tid / ng; the lanes of a warp
// mostly share a split and so read the same staged source (one broadcast).
// Split k takes the sources j = k, k + nsplit, ... of each chunk, SU at a time
// with independent partial sums; the partial sums of a target are added over
// the splits in a fixed order.
template <typename R, int DIM, int KER, int TT>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_split(R e2, int64_t N, const R *xs,
                                                           const R *lam, const int32_t *leaf_off,
                                                           const int32_t *near_off,
                                                           const int32_t *near_idx, R *u)
{
    using S4 = typename Src4<R>::type;
    constexpr int REC = DIM <= 3 ? 1 : 2;
    constexpr int P2P_SCHUNK = P2P_STAGE_BYTES / (int)(sizeof(S4) * REC);
    constexpr int SU = RBF_P2P_SU;
    __shared__ S4 src[P2P_SCHUNK * REC];
    __shared__ int32_t rstart[729], rpre[730];
    __shared__ R red[TT][P2P_THREADS];
    const int a = blockIdx.x;
    const int e0 = near_off[a], ne = near_off[a + 1] - e0;
    near_ranges(e0, ne, near_idx, leaf_off, rstart, nullptr, rpre);
    const int nsrc = rpre[ne];
    const int t0 = leaf_off[a], nt = leaf_off[a + 1] - t0;  // 1 <= nt <= P2P_THREADS
    const int ng = (nt + TT - 1) / TT;
    const int nsplit = P2P_THREADS / ng;
    const int grp = threadIdx.x % ng, sp = threadIdx.x / ng;
    const bool active = sp < nsplit;
    // coordinates relative to the leaf's first point, then scaled: Phi from
    // phi_s(c0 + sum d^2), rounding relative to the neighbourhood's size
    const R sc = sqrt(e2);
    R org[DIM];
#pragma unroll
    for (int t = 0; t < DIM; ++t) org[t] = xs[(int64_t)t * N + t0];
    R xt[TT][DIM];
#pragma unroll
    for (int q = 0; q < TT; ++q) {
        const int tq = min(grp + q * ng, nt - 1);
#pragma unroll
        for (int t = 0; t < DIM; ++t) xt[q][t] = sc * (xs[(int64_t)t * N + t0 + tq] - org[t]);
    }
    R acc[TT][SU];
#pragma unroll
    for (int q = 0; q < TT; ++q)
#pragma unroll
        for (int k = 0; k < SU; ++k) acc[q][k] = (R)0;
    for (int s0 = 0; s0 < nsrc; s0 += P2P_SCHUNK) {
        const int cnt = min(P2P_SCHUNK, nsrc - s0);
        __syncthreads();
        // warp w copies the parts of ranges w, w + 4, ... that fall in the chunk,
        // lane by lane (consecutive lanes read consecutive points)
        for (int e = threadIdx.x >> 5; e < ne; e += P2P_WARPS) {
            const int b0 = max(rpre[e], s0), b1 = min(rpre[e + 1], s0 + cnt);
            for (int vv = b0 + (threadIdx.x & 31); vv < b1; vv += 32) {
                const int v = vv - s0;
                const int64_t j = rstart[e] + (vv - rpre[e]);
                R c[8] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
#pragma unroll
                for (int t = 0; t < DIM; ++t) c[t] = sc * (xs[(int64_t)t * N + j] - org[t]);
                S4 r0;
                r0.x = c[0];
                r0.y = c[1];
                r0.z = c[2];
                r0.w = lam[j];
                src[REC * v] = r0;
                if (REC == 2) {
                    S4 r1;
                    r1.x = c[3];
                    r1.y = c[4];
                    r1.z = c[5];
                    r1.w = (R)0;
                    src[REC * v + 1] = r1;
                }
            }
        }
        __syncthreads();
        if (!active) continue;
        // steps whose SU sources all lie in the chunk need no masks; one masked
        // step takes the rest
        auto step = [&](int j0, bool masked) {
#pragma unroll
            for (int k = 0; k < SU; ++k) {
                const int jj = j0 + k * nsplit;
                const int j = masked ? min(jj, cnt - 1) : jj;
                const S4 r0 = src[REC * j];
                S4 r1;
                if (REC == 2) r1 = src[REC * j + 1];
                const R wgt = !masked || jj < cnt ? r0.w : (R)0;
#pragma unroll
                for (int q = 0; q < TT; ++q) {
                    R d0 = xt[q][0] - r0.x;
                    R r2 = fma(d0, d0, (R)phi_c0<KER>());
                    if (DIM > 1) {
                        R d1 = xt[q][DIM > 1 ? 1 : 0] - r0.y;
                        r2 = fma(d1, d1, r2);
                    }
                    if (DIM > 2) {
                        R d2 = xt[q][DIM > 2 ? 2 : 0] - r0.z;
                        r2 = fma(d2, d2, r2);
                    }
                    if (DIM > 3) {
                        R d3 = xt[q][DIM > 3 ? 3 : 0] - r1.x;
                        r2 = fma(d3, d3, r2);
                    }
                    if (DIM > 4) {
                        R d4 = xt[q][DIM > 4 ? 4 : 0] - r1.y;
                        r2 = fma(d4, d4, r2);
                    }
                    if (DIM > 5) {
                        R d5 = xt[q][DIM > 5 ? 5 : 0] - r1.z;
                        r2 = fma(d5, d5, r2);
                    }
                    const R ph = phi_s<KER>(r2);
                    acc[q][k] = fma(wgt, ph, acc[q][k]);
                }
            }
        };
        int j0 = sp;
        for (; j0 + (SU - 1) * nsplit < cnt; j0 += SU * nsplit) step(j0, false);
        if (j0 < cnt) step(j0, true);
    }
#pragma unroll
    for (int q = 0; q < TT; ++q) {
        R tsum = acc[q][0];
#pragma unroll
        for (int k = 1; k < SU; ++k) tsum += acc[q][k];
        red[q][threadIdx.x] = active ? tsum : (R)0;
    }
    __syncthreads();
    if (threadIdx.x < nt) {
        const int g = threadIdx.x % ng, q = threadIdx.x / ng;
        R sum = red[q][g];
        for (int k = 1; k < nsplit; ++k) sum += red[q][k * ng + g];
        u[t0 + threadIdx.x] = sum;
    }
}

template <typename R, int KER>
int launch_p2p_split(int d, R e2, const rbf_tree *t, const R *xs, const R *lam, R *u,
                     cudaStream_t s)
{
    const int nleaf = t->nleaf();
    switch (d) {
#define RBF_P2P_CASE(DD)                                                                          \
    case DD:                                                                                      \
        k_p2p_split<R, DD, KER, RBF_P2P_TT><<<nleaf, P2P_THREADS, 0, s>>>(                          \
            e2, t->N, xs, lam, t->leaf_off, t->near_off, t->near_idx, u);                          \
        break;
        RBF_P2P_CASE(1)
        RBF_P2P_CASE(2)
        RBF_P2P_CASE(3)
        RBF_P2P_CASE(4)
        RBF_P2P_CASE(5)
        RBF_P2P_CASE(6)
#undef RBF_P2P_CASE
        default:
            rbf_set_error("p2p: unsupported dimension %d", d);
            return RBF_EINVAL;
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

template <typename R, int TG, int KER>
int launch_p2p_tg(int d, R e2, const rbf_tree *t, const R *xs, const R *lam, R *u, cudaStream_t s)
{
    const int nleaf = t->nleaf();
    switch (d) {
#define RBF_P2P_CASE(DD)                                                                          \
    case DD:                                                                                      \
        k_p2p<R, DD, TG, KER><<<nleaf, P2P_THREADS, 0, s>>>(e2, t->N, xs, lam, t->leaf_off,        \
                                                            t->near_off, t->near_idx, u);          \
        break;
        RBF_P2P_CASE(1)
        RBF_P2P_CASE(2)
        RBF_P2P_CASE(3)
        RBF_P2P_CASE(4)
        RBF_P2P_CASE(5)
        RBF_P2P_CASE(6)
#undef RBF_P2P_CASE
        default:
            rbf_set_error("p2p: unsupported dimension %d", d);
            return RBF_EINVAL;
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

// leaves of up to P2P_THREADS points: the split kernel; larger ones: target groups of
// 32 per pass (four per pass for large leaves)
template <typename R>
int launch_p2p(int d, int kernel, R e2, const rbf_tree *t, const R *xs, const R *lam, R *u,
               cudaStream_t s)
{
    const int ml = std::max<int>(1, t->max_leaf);
    // leaves of at most one CTA of points: (target, source split) threads
    if (ml <= P2P_THREADS)
        return with_kernel(kernel, [&](auto K) {
            return launch_p2p_split<R, decltype(K)::value>(d, e2, t, xs, lam, u, s);
        });
    const bool small = ml <= RBF_P2P_SMALL || RBF_P2P_TGMAX == 1;
    return with_kernel(kernel, [&](auto K) {
        return small ? launch_p2p_tg<R, 1, decltype(K)::value>(d, e2, t, xs, lam, u, s)
                     : launch_p2p_tg<R, 4, decltype(K)::value>(d, e2, t, xs, lam, u, s);
    });
}

// ---------------------------------------------- several right-hand sides --
// The near field of RG columns at once: Phi(x_i - x_j) is evaluated once per
// pair and multiplies the RG coefficients of the source.  Sources are staged
// as records (coordinates padded to 4 or 8 floats, then RG coefficients);
// lane = target, TG targets per lane, warps split the staged sources and their
// partial sums are added in a fixed order.
constexpr int P2PM_SCH = 256;   // sources per staged chunk

template <int DIM, int RG>
struct P2pmShape {
    static constexpr int C4 = DIM <= 4 ? 4 : 8;            // padded coordinates
    static constexpr int REC = C4 + RG;                    // floats per source record
    static constexpr int TG = RG >= 16 ? 4 : 4;            // target groups of 32 per pass
    static constexpr int TB = 32 * TG;
    static constexpr int STAGE = P2PM_SCH * REC;
    static constexpr int RED = P2P_WARPS * TB * RG;
    static constexpr int BUF = STAGE > RED ? STAGE : RED;
};

template <int DIM, int RG, int KER>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_multi(float e2, int64_t N,
                                                           const float *xs, const float *lam,
                                                           int G, const int32_t *leaf_off,
                                                           const int32_t *near_off,
                                                           const int32_t *near_idx, float *u)
{
    using SH = P2pmShape<DIM, RG>;
    constexpr int C4 = SH::C4, REC = SH::REC, TG = SH::TG, TB = SH::TB;
    __shared__ __align__(16) float buf[SH::BUF];
    __shared__ int32_t rstart[729], rpre[730];
    const int a = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e0 = near_off[a], ne = near_off[a + 1] - e0;
    near_ranges(e0, ne, near_idx, leaf_off, rstart, nullptr, rpre);
    const int nsrc = rpre[ne];
    const int t0 = leaf_off[a], nt = leaf_off[a + 1] - t0;
    // coordinates relative to the leaf's first point, then scaled: Phi from
    // phi_s(c0 + sum d^2), rounding relative to the neighbourhood's size
    const float sc = sqrtf(e2);
    float org[DIM];
#pragma unroll
    for (int t = 0; t < DIM; ++t) org[t] = xs[(int64_t)t * N + t0];
    for (int tb = 0; tb < nt; tb += TB) {
        float xt[TG][DIM];
        float acc[TG][RG];
#pragma unroll
        for (int g = 0; g < TG; ++g) {
            const int i = tb + g * 32 + lane;
#pragma unroll
            for (int t = 0; t < DIM; ++t) xt[g][t] = i < nt ? sc * (xs[(int64_t)t * N + t0 + i] - org[t]) : 0.0f;
#pragma unroll
            for (int r = 0; r < RG; ++r) acc[g][r] = 0.0f;
        }
        const int ngrp = min(TG, (nt - tb + 31) / 32);
        for (int s0 = 0; s0 < nsrc; s0 += P2PM_SCH) {
            const int cnt = min(P2PM_SCH, nsrc - s0);
            __syncthreads();
            for (int v = threadIdx.x; v < cnt; v += P2P_THREADS) {
                const int vv = s0 + v;
                int lo = 0, hi = ne - 1;
                while (lo < hi) {  // last range with rpre[e] <= vv
                    const int mid = (lo + hi + 1) >> 1;
                    if (rpre[mid] <= vv) lo = mid;
                    else hi = mid - 1;
                }
                const int64_t j = rstart[lo] + (vv - rpre[lo]);
                float *rec = buf + v * REC;
#pragma unroll
                for (int t = 0; t < C4; ++t) rec[t] = t < DIM ? sc * (xs[(int64_t)t * N + j] - org[t]) : 0.0f;
#pragma unroll
                for (int r = 0; r < RG; ++r) rec[C4 + r] = r < G ? lam[(int64_t)r * N + j] : 0.0f;
            }
            __syncthreads();
            for (int j = warp; j < cnt; j += P2P_WARPS) {
                const float4 *rec = reinterpret_cast<const float4 *>(buf + j * REC);
                float xs_[C4], l[RG];
#pragma unroll
                for (int c = 0; c < C4 / 4; ++c) {
                    const float4 v = rec[c];
                    xs_[4 * c] = v.x;
                    xs_[4 * c + 1] = v.y;
                    xs_[4 * c + 2] = v.z;
                    xs_[4 * c + 3] = v.w;
                }
#pragma unroll
                for (int c = 0; c < RG / 4; ++c) {
                    const float4 v = rec[C4 / 4 + c];
                    l[4 * c] = v.x;
                    l[4 * c + 1] = v.y;
                    l[4 * c + 2] = v.z;
                    l[4 * c + 3] = v.w;
                }
#pragma unroll
                for (int g = 0; g < TG; ++g) {
                    if (g < ngrp) {
                        float r2 = phi_c0<KER>();
#pragma unroll
                        for (int t = 0; t < DIM; ++t) {
                            const float df = xt[g][t] - xs_[t];
                            r2 = fmaf(df, df, r2);
                        }
                        const float ph = phi_s<KER>(r2);
#pragma unroll
                        for (int r = 0; r < RG; ++r) acc[g][r] = fmaf(l[r], ph, acc[g][r]);
                    }
                }
            }
        }
        __syncthreads();
        // partial sums of the warps -> fixed-order total
#pragma unroll
        for (int g = 0; g < TG; ++g)
#pragma unroll
            for (int r = 0; r < RG; ++r) buf[(warp * TB + g * 32 + lane) * RG + r] = acc[g][r];
        __syncthreads();
        const int nb = min(TB, nt - tb);
        for (int idx = threadIdx.x; idx < nb * G; idx += P2P_THREADS) {
            const int r = idx / nb, i = idx - r * nb;
            float sum = buf[i * RG + r];
#pragma unroll
            for (int w = 1; w < P2P_WARPS; ++w) sum += buf[(w * TB + i) * RG + r];
            u[(int64_t)r * N + t0 + tb + i] = sum;
        }
    }
}

template <int RG, int KER>
int launch_p2p_multi(int d, float e2, const rbf_tree *t, const float *lam, int G, float *u,
                     cudaStream_t s)
{
    const int nleaf = t->nleaf();
    switch (d) {
#define RBF_P2PM_CASE(DD)                                                                         \
    case DD:                                                                                      \
        k_p2p_multi<DD, RG, KER><<<nleaf, P2P_THREADS, 0, s>>>(e2, t->N, t->xs32, lam, G,         \
                                                               t->leaf_off, t->near_off,          \
                                                               t->near_idx, u);                   \
        break;
        RBF_P2PM_CASE(1)
        RBF_P2PM_CASE(2)
        RBF_P2PM_CASE(3)
        RBF_P2PM_CASE(4)
        RBF_P2PM_CASE(5)
        RBF_P2PM_CASE(6)
#undef RBF_P2PM_CASE
        default:
            rbf_set_error("p2p: unsupported dimension %d", d);
            return RBF_EINVAL;
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

// ------------------------------------------------------- direct sum -------
constexpr int DS_THREADS = 256;
constexpr int DS_TILE = 256;

__global__ void __launch_bounds__(DS_THREADS) k_direct(const double *X, int64_t N, int d, int kernel,
                                                       double eps, const double *lam,
                                                       const int64_t *targets, int64_t nt,
                                                       double *u)
{
    __shared__ double sx[DS_TILE * RBF_MAX_DIM];
    __shared__ double sl[DS_TILE];
    const int64_t q = (int64_t)blockIdx.x * DS_THREADS + threadIdx.x;
    double xt[RBF_MAX_DIM];
    const bool active = q < nt;
    int64_t ti = active ? targets[q] : 0;
    // a target index outside [0, N) reads nothing and gives NaN
    const bool valid = ti >= 0 && ti < N;
    if (!valid) ti = 0;
    for (int t = 0; t < d; ++t) xt[t] = active ? X[ti * d + t] : 0.0;
    const double e2 = eps * eps;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < N; j0 += DS_TILE) {
        const int cnt = (int)min((int64_t)DS_TILE, N - j0);
        __syncthreads();
        for (int v = threadIdx.x; v < cnt * d; v += DS_THREADS) sx[v] = X[j0 * d + v];
        for (int v = threadIdx.x; v < cnt; v += DS_THREADS) sl[v] = lam[j0 + v];
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            double r2 = 0.0;
            for (int t = 0; t < d; ++t) {
                double df = xt[t] - sx[j * d + t];
                r2 += df * df;
            }
            double ph;
            if (kernel == RBF_GAUSSIAN) ph = exp(-e2 * r2);
            else if (kernel == RBF_MQ) ph = sqrt(1.0 + e2 * r2);
            else if (kernel == RBF_WENDLAND) {
                const double q = sqrt(e2 * r2), w = q < 1.0 ? 1.0 - q : 0.0;
                ph = w * w * w * (3.0 * q + 1.0);
            } else ph = 1.0 / sqrt(1.0 + e2 * r2);
            acc += sl[j] * ph;
        }
    }
    if (active) u[q] = valid ? acc : __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace

template <typename R>
int rbf_run_p2p(rbf_tree *t, int kernel, double eps, const R *lam_s, R *u, cudaStream_t s)
{
    rbf_pass_timer tm(t, RBF_PASS_P2P, s);
    const R *xs = (const R *)(sizeof(R) == 8 ? (const void *)t->xs64 : (const void *)t->xs32);
    // the FP32 Gaussian goes through exp2, so fold log2(e) into eps^2
    double e2 = eps * eps;
    if (sizeof(R) == 4 && kernel == RBF_GAUSSIAN) e2 *= 1.4426950408889634;
    return launch_p2p<R>(t->d, kernel, (R)e2, t, xs, lam_s, u, s);
}

template int rbf_run_p2p<float>(rbf_tree *, int, double, const float *, float *, cudaStream_t);

int rbf_run_p2p_multi(rbf_tree *t, int kernel, double eps, const float *lam_s, int G, float *u,
                      cudaStream_t s)
{
    RBF_REQUIRE(G >= 1 && G <= 16, "rbf_run_p2p_multi: G=%d", G);
    rbf_pass_timer tm(t, RBF_PASS_P2P, s);
    double e2 = eps * eps;
    if (kernel == RBF_GAUSSIAN) e2 *= 1.4426950408889634;
    return with_kernel(kernel, [&](auto K) {
        constexpr int KER = decltype(K)::value;
        if (G <= 4) return launch_p2p_multi<4, KER>(t->d, (float)e2, t, lam_s, G, u, s);
        if (G <= 8) return launch_p2p_multi<8, KER>(t->d, (float)e2, t, lam_s, G, u, s);
        return launch_p2p_multi<16, KER>(t->d, (float)e2, t, lam_s, G, u, s);
    });
}
template int rbf_run_p2p<double>(rbf_tree *, int, double, const double *, double *,
                                 cudaStream_t);

extern "C" int rbf_direct_sum(const double *X, int64_t N, int d, rbf_kernel kernel, double eps,
                              const double *lambda, const int64_t *targets, int64_t nt, double *u,
                              void *stream)
{
    RBF_REQUIRE(X && lambda && targets && u, "rbf_direct_sum: NULL pointer");
    RBF_REQUIRE(N >= 1 && d >= 1 && d <= RBF_MAX_DIM && nt >= 0, "rbf_direct_sum: bad sizes");
    RBF_REQUIRE(kernel >= RBF_GAUSSIAN && kernel <= RBF_WENDLAND, "rbf_direct_sum: unknown kernel");
    if (nt == 0) return RBF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_direct<<<ceil_div(nt, DS_THREADS), DS_THREADS, 0, s>>>(X, N, d, kernel, eps, lambda, targets,
                                                             nt, u);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}
