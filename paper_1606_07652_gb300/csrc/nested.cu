// nested.cu -- far field of the MLFMM on nested (scale-invariant) frequency
// grids: Sec. 4.1 "Upsweep", "Coupling", "Downsweep" with the interpolation
// and anterpolation of Sec. 4.1.1.
//
// Level l has the grid xi_{l,k} = k 2pi / L_l, L_l = L 2^(2-l), k = -M/2..M/2
// (the same M on every level, xi_{l-1} = xi_l / 2) and its own coefficients
// omega_l C_l (lattice samples with period L_l, taper flat on
// |t| <= side 2^(2-l)).  With box width w_l = side 2^-l every translation phase
// depends on k theta only, theta = xi_{l,1} w_l = pi side / (2 L), on all levels.
//
//   P2M  on the leaf grid                         -> V_D
//   M2M  Eq. (43):  V_{l-1} = sum_c e^{-i xi_{l-1}.(c_c - c_p)} (P x ... x P) V_c
//        P = K-point Lagrange stencil in xi (child node k/2 for parent node k),
//        applied one dimension at a time
//   M2L  Eq. (45) over IL_l(a), written as the children of the parent's
//        neighbours minus a's own neighbours (the 2^d siblings together):
//          L_l(a) = omega_l C_l [ sum_{p' in N(par a)} e^{i xi_l.(c_a - c_p')} Vt_p'
//                                - sum_{b in N(a)} e^{i xi_l.(c_a - c_b)} V_b ],
//          Vt_p' = sum_{children b} e^{-i xi_l.(c_b - c_p')} V_b  (level-l grid)
//   L2L  Eqs. (47)-(48):  L_c += (P^T x ... x P^T)(e^{i xi_{l-1}.(c_c - c_p)} L_p)
//   L2P  on the leaf grid
//
// Expansions keep the half spectrum k0 >= 0 (layout of rbf_internal.cuh).
// Every omega_l C_l carries the weight 2 of k0 > 0, so local expansions are in
// that weighted form; multipole expansions are plain.  Values at k0 < 0 come
// from V(-xi) = conj V(xi), which the real, mirror-symmetric stencils keep.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rbf_internal.cuh"

namespace {

constexpr int kThreads = 256;
// rows of the phase table (n1 complex entries each, index k + M/2)
constexpr int kPhVt = 0;    // [2]    e^{-i theta k (2b-1)/2}: child b -> parent, child grid
constexpr int kPhM2M = 2;   // [2]    e^{-i theta k (2b-1)/4}: child b -> parent, parent grid
constexpr int kPhL2L = 4;   // [2]    e^{+i theta k (2b-1)/4}: parent -> child b, parent grid
constexpr int kPhNb = 6;    // [3]    e^{-i theta k e}: neighbour at offset e = -1, 0, 1
constexpr int kPhPar = 9;   // [2][3] e^{i theta k ((2b-1)/2 - 2e)}: parent's neighbour at offset e
constexpr int kPhRows = 15;

// kk[t] = k_t + M/2 of half-spectrum mode m (dimension d-1 fastest)
template <int DIM>
__device__ __forceinline__ void mode_digits(int64_t m, int n1, int M, int *kk)
{
#pragma unroll
    for (int t = DIM - 1; t >= 1; --t) {
        kk[t] = (int)(m % n1);
        m /= n1;
    }
    kk[0] = (int)m + M / 2;
}

// neighbours at Chebyshev distance <= 1 on level l: nbr[b][q], q = sum_t (e_t + 1) 3^t,
// -1 where the box is empty or outside the root
__global__ void k_build_nbr(const uint64_t *key, int nbox, int d, int l, int nq, int32_t *nbr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nbox * nq) return;
    const int b = (int)(i / nq);
    int q = (int)(i % nq);
    const uint64_t kb = key[b];
    uint64_t nk = 0;
    bool inside = true;
    for (int t = 0; t < d; ++t) {
        int c = 0;
        for (int bit = 0; bit < l; ++bit) c |= (int)((kb >> (bit * d + t)) & 1u) << bit;
        const int x = c + (q % 3) - 1;
        q /= 3;
        if (x < 0 || x >= (1 << l)) inside = false;
        for (int bit = 0; bit < l && inside; ++bit)
            nk |= (uint64_t)((x >> bit) & 1) << (bit * d + t);
    }
    int32_t out = -1;
    if (inside) {
        int lo = 0, hi = nbox;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (key[mid] < nk) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nbox && key[lo] == nk) out = lo;
    }
    nbr[i] = out;
}

// Vt_p = sum_children e^{-i xi_l.(c_c - c_p)} V_c on the children's grid
template <typename R, int DIM>
__global__ void __launch_bounds__(kThreads) k_vt(int M, int n1, int64_t nmode, int64_t ms,
                                                 const cplx<R> *ph, const int32_t *child_off,
                                                 const uint64_t *child_key, const cplx<R> *Vc,
                                                 cplx<R> *Vt)
{
    using C = cplx<R>;
    const int p = blockIdx.x;
    const int64_t m = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    int kk[DIM];
    mode_digits<DIM>(m, n1, M, kk);
    C acc{(R)0, (R)0};
    for (int c = child_off[p]; c < child_off[p + 1]; ++c) {
        const unsigned bits = (unsigned)(child_key[c] & ((1u << DIM) - 1u));
        C f = ph[(kPhVt + (bits & 1u)) * n1 + kk[0]];
#pragma unroll
        for (int t = 1; t < DIM; ++t) f = cmul(f, ph[(kPhVt + ((bits >> t) & 1u)) * n1 + kk[t]]);
        cmac(acc, f, Vc[(int64_t)c * ms + m]);
    }
    Vt[(int64_t)p * ms + m] = acc;
}

// One dimension t >= 1 of a stencil product on every box:
//   out[b][.. k_t ..] (+)= sum_tap w[k_t][tap] in[b][.. idx[k_t][tap] ..]
// (stride of dimension t in the mode index: n1^(d-1-t))
template <typename R>
__global__ void __launch_bounds__(kThreads) k_axis(int n1, int64_t nmode, int64_t ms, int64_t stride,
                                                   int ntap, const int32_t *idx, const R *w,
                                                   const cplx<R> *in, cplx<R> *out, int accumulate,
                                                   int nch)
{
    using C = cplx<R>;
    const int64_t b = blockIdx.x / nch;  // mode chunks of one box run back to back
    const int64_t m = (int64_t)(blockIdx.x % nch) * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    const int dig = (int)((m / stride) % n1);
    const C *src = in + b * ms + (m - (int64_t)dig * stride);
    C acc{(R)0, (R)0};
    for (int a = 0; a < ntap; ++a) {
        const R wt = w[dig * ntap + a];
        const C v = src[(int64_t)idx[dig * ntap + a] * stride];
        acc.x = fma(wt, v.x, acc.x);
        acc.y = fma(wt, v.y, acc.y);
    }
    C *dst = out + b * ms + m;
    if (accumulate) {
        acc.x += dst->x;
        acc.y += dst->y;
    }
    *dst = acc;
}

// M2M, last step: dimension 0 of the interpolation (k0 < 0 by symmetry), the
// translation to the parent centre on the parent grid, and the sum over children.
// T holds the children with dimensions 1..d-1 already interpolated.
template <typename R, int DIM>
__global__ void __launch_bounds__(kThreads) k_m2m_last(int M, int n1, int64_t nmode, int64_t ms,
                                                       int64_t rows, int K, const int32_t *fidx,
                                                       const R *fw, const cplx<R> *ph,
                                                       const int32_t *child_off,
                                                       const uint64_t *child_key, const cplx<R> *T,
                                                       cplx<R> *Vp, int nch)
{
    using C = cplx<R>;
    const int p = (int)(blockIdx.x / nch);  // the taps of one parent's rows stay in L2
    const int64_t m = (int64_t)(blockIdx.x % nch) * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    int kk[DIM];
    mode_digits<DIM>(m, n1, M, kk);
    const int kp = kk[0];
    const int64_t rest = m - (int64_t)(kp - M / 2) * rows;
    const int64_t mrest = rows - 1 - rest;  // every digit k_t -> -k_t
    C acc{(R)0, (R)0};
    for (int c = child_off[p]; c < child_off[p + 1]; ++c) {
        const C *Tc = T + (int64_t)c * ms;
        C sv{(R)0, (R)0};
        for (int a = 0; a < K; ++a) {
            const int j = fidx[kp * K + a] - M / 2;
            const R wt = fw[kp * K + a];
            const C v = j >= 0 ? Tc[(int64_t)j * rows + rest] : cconj(Tc[(int64_t)(-j) * rows + mrest]);
            sv.x = fma(wt, v.x, sv.x);
            sv.y = fma(wt, v.y, sv.y);
        }
        const unsigned bits = (unsigned)(child_key[c] & ((1u << DIM) - 1u));
        C f = ph[(kPhM2M + (bits & 1u)) * n1 + kk[0]];
#pragma unroll
        for (int t = 1; t < DIM; ++t) f = cmul(f, ph[(kPhM2M + ((bits >> t) & 1u)) * n1 + kk[t]]);
        cmac(acc, f, sv);
    }
    Vp[(int64_t)p * ms + m] = acc;
}

// L2L, first step for every child c at level l: the translation of the
// parent's local expansion to c on the parent grid, then dimension 0 of the
// anterpolation (parent nodes k0 < 0 by symmetry).  Input and output are in
// the weighted half-spectrum form.  Dimensions 1..d-1 stay on the parent grid.
template <typename R, int DIM>
__global__ void __launch_bounds__(kThreads) k_l2l_first(int M, int n1, int64_t nmode, int64_t ms,
                                                        int64_t rows, int KT, const int32_t *tidx,
                                                        const R *tw, const cplx<R> *ph,
                                                        const int32_t *parent, const uint64_t *key,
                                                        const cplx<R> *Lp, cplx<R> *out,
                                                        int accumulate, int nch)
{
    using C = cplx<R>;
    const int64_t c = blockIdx.x / nch;
    const int64_t m = (int64_t)(blockIdx.x % nch) * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    int kk[DIM];
    mode_digits<DIM>(m, n1, M, kk);
    const int jp = kk[0];
    const int64_t rest = m - (int64_t)(jp - M / 2) * rows;
    const int64_t mrest = rows - 1 - rest;
    const unsigned bits = (unsigned)(key[c] & ((1u << DIM) - 1u));
    // translation phase of dimensions 1..d-1 at rest and at the mirrored rest
    C fr{(R)1, (R)0}, fm{(R)1, (R)0};
#pragma unroll
    for (int t = 1; t < DIM; ++t) {
        const int row = (kPhL2L + ((bits >> t) & 1u)) * n1;
        fr = cmul(fr, ph[row + kk[t]]);
        fm = cmul(fm, ph[row + (n1 - 1 - kk[t])]);
    }
    const C *P = Lp + (int64_t)parent[c] * ms;
    const int row0 = (kPhL2L + (bits & 1u)) * n1;
    // taps with k0 >= 0 and k0 < 0 are summed apart, so that the translation of
    // dimensions 1..d-1 (fr, or fm for the mirrored rest) multiplies each sum once:
    // sum_a wt ph v fr + conj(sum_a wt ph v fm) = fr S+ + conj(fm S-)  (wt real)
    C sp{(R)0, (R)0}, sm{(R)0, (R)0};
    for (int a = 0; a < KT; ++a) {
        const int k = tidx[jp * KT + a] - M / 2;
        const int ka = k >= 0 ? k : -k;
        // weighted -> plain value at |k0|: halve the weight of k0 != 0
        const R wt = ka > 0 ? (R)0.5 * tw[jp * KT + a] : tw[jp * KT + a];
        const C v = P[(int64_t)ka * rows + (k >= 0 ? rest : mrest)];
        const C pv = cmul(ph[row0 + ka + M / 2], v);
        if (k >= 0) {
            sp.x = fma(wt, pv.x, sp.x);
            sp.y = fma(wt, pv.y, sp.y);
        } else {
            sm.x = fma(wt, pv.x, sm.x);
            sm.y = fma(wt, pv.y, sm.y);
        }
    }
    C acc = cmul(fr, sp);
    const C tm = cconj(cmul(fm, sm));
    acc.x += tm.x;
    acc.y += tm.y;
    const R wgt = jp > M / 2 ? (R)2 : (R)1;  // plain -> weighted at the child's k0
    acc.x *= wgt;
    acc.y *= wgt;
    C *dst = out + c * ms + m;
    if (accumulate) {
        acc.x += dst->x;
        acc.y += dst->y;
    }
    *dst = acc;
}

constexpr int ipow(int b, int e) { return e <= 0 ? 1 : b * ipow(b, e - 1); }

// One dimension t of a separable offset sum.  in[bs + 2^t (j + W r)], j < W, holds
// partial sums with the dimensions below t already reduced to the child bit bs;
// out[bs + 2^t b + 2^(t+1) r] = sum_{e<3} f[b][e] in[bs + 2^t (s + W r)], s = e for
// the 3 offsets around the parent (W = 3) or s = b + e for the block of 4 around
// the children (W = 4).
template <int T, int W, int DIM, typename C>
__device__ __forceinline__ void sep_step(const C *in, C *out, const C (&f)[2][3])
{
    constexpr int NBS = 1 << T;
    constexpr int NR = ipow(W, DIM - T - 1);
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int bs = 0; bs < NBS; ++bs)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                C acc;
                acc.x = acc.y = 0;
#pragma unroll
                for (int e = 0; e < 3; ++e) cmac(acc, f[b][e], in[bs + NBS * ((W == 3 ? e : b + e) + W * r)]);
                out[bs + NBS * b + 2 * NBS * r] = acc;
            }
}

// Offset sum of one parent's 2^d children: out[b] = sum over the 3^d offsets of
// prod_t f_t[b_t][e_t] * val(offset), val read from src at the boxes ids[] (-1 =
// empty), W = 3 (ids = the parent's neighbours, e is the offset) or W = 4 (ids =
// the 4^d block around the children, child b's neighbour at offset e sits at b + e).
template <int W, int DIM, typename C>
__device__ __forceinline__ void offset_sum(const C *src, int64_t ms, int64_t m, const int32_t *ids,
                                           const C *ph, int n1, const int *kk, int row0, int brow,
                                           C *out)
{
    constexpr int R0 = ipow(W, DIM - 1);
    C a[2 * R0];
    C f[2][3];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 3; ++e) f[b][e] = ph[(row0 + brow * b + e) * n1 + kk[0]];
#pragma unroll
    for (int r = 0; r < R0; ++r) {
        C v[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int id = ids[j + W * r];
            if (id >= 0) v[j] = src[(int64_t)id * ms + m];
            else v[j].x = v[j].y = 0;
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            C acc;
            acc.x = acc.y = 0;
#pragma unroll
            for (int e = 0; e < 3; ++e) cmac(acc, f[b][e], v[W == 3 ? e : b + e]);
            a[b + 2 * r] = acc;
        }
    }
    if constexpr (DIM == 1) {
        out[0] = a[0];
        out[1] = a[1];
    } else {
        C g[2][3];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 3; ++e) g[b][e] = ph[(row0 + brow * b + e) * n1 + kk[1]];
        if constexpr (DIM == 2) {
            sep_step<1, W, DIM>(a, out, g);
        } else {
            C a1[4 * ipow(W, DIM - 2)];
            sep_step<1, W, DIM>(a, a1, g);
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 3; ++e) g[b][e] = ph[(row0 + brow * b + e) * n1 + kk[2]];
            sep_step<2, W, DIM>(a1, out, g);
        }
    }
}

// M2L of level l for the 2^d children of every parent p at level l-1 (file
// header): the 3^d parent-neighbour terms are shared by the siblings, and their
// own 3^d neighbours all lie in the 4^d block around them; both sums are done
// one dimension at a time.  Writes L_l of every child.
template <typename R, int DIM>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) k_m2l_sib(int M, int n1, int64_t nmode, int64_t ms,
                                                      const cplx<R> *ph, const int32_t *nb4,
                                                      const int32_t *pnbr, const cplx<R> *Vt,
                                                      const cplx<R> *V, const R *wc, cplx<R> *L)
{
    using C = cplx<R>;
    constexpr int NB = 1 << DIM, Q3 = ipow(3, DIM), Q4 = ipow(4, DIM);
    const int64_t p = blockIdx.x;
    const int64_t m = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    int kk[DIM];
    mode_digits<DIM>(m, n1, M, kk);
    const int32_t *blk = nb4 + p * Q4;
    C sp[NB], sn[NB];
    offset_sum<3, DIM>(Vt, ms, m, pnbr + p * Q3, ph, n1, kk, kPhPar, 3, sp);
    offset_sum<4, DIM>(V, ms, m, blk, ph, n1, kk, kPhNb, 0, sn);
    const R w = wc[m];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        int q = 0, st = 1;
#pragma unroll
        for (int t = 0; t < DIM; ++t) {
            q += (1 + ((b >> t) & 1)) * st;
            st *= 4;
        }
        const int id = blk[q];
        if (id >= 0) {
            C o;
            o.x = w * (sp[b].x - sn[b].x);
            o.y = w * (sp[b].y - sn[b].y);
            L[(int64_t)id * ms + m] = o;
        }
    }
}

// nb4[p][q]: level-l box at block coordinate 2 c_p - 1 + q_t (q = sum_t q_t 4^t, q_t < 4)
// around the children of parent p (level l-1), -1 where empty or outside
__global__ void k_build_nb4(const uint64_t *pkey, int np, const uint64_t *key, int nbox, int d, int l,
                            int nq, int32_t *nb4)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)np * nq) return;
    const int p = (int)(i / nq);
    int q = (int)(i % nq);
    const uint64_t kp = pkey[p];
    uint64_t nk = 0;
    bool inside = true;
    for (int t = 0; t < d; ++t) {
        int c = 0;
        for (int bit = 0; bit < l - 1; ++bit) c |= (int)((kp >> (bit * d + t)) & 1u) << bit;
        const int x = 2 * c - 1 + (q % 4);
        q /= 4;
        if (x < 0 || x >= (1 << l)) inside = false;
        for (int bit = 0; bit < l && inside; ++bit)
            nk |= (uint64_t)((x >> bit) & 1) << (bit * d + t);
    }
    int32_t out = -1;
    if (inside) {
        int lo = 0, hi = nbox;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (key[mid] < nk) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nbox && key[lo] == nk) out = lo;
    }
    nb4[i] = out;
}

// ------------------------------------------------------------ host tables --
struct LagTables {
    int K = 0, KT = 0;
    std::vector<int32_t> fidx, tidx;
    std::vector<double> fw, tw;
};

// Parent node k (index k + M/2) takes child nodes floor(k/2) - K/2 + 1 ..
// floor(k/2) + K/2 with the Lagrange basis l_a(t) = prod_{b != a} (t - t_b)/(t_a - t_b)
// at t = k/2 (node units).  Rows k < 0 are the mirror images of rows -k, so the
// table is exactly symmetric; the transpose lists, for every child node, the
// parent nodes whose stencils hold it with a nonzero weight.
LagTables lagrange_tables(int M, int K)
{
    LagTables g;
    const int n1 = M + 1;
    g.K = K;
    g.fidx.assign((size_t)n1 * K, 0);
    g.fw.assign((size_t)n1 * K, 0.0);
    for (int k = 0; k <= M / 2; ++k) {
        const int kp = k + M / 2;
        const int j0 = k / 2 - K / 2 + 1;
        const double tt = 0.5 * k;
        for (int a = 0; a < K; ++a) {
            double v = 1.0;
            for (int b = 0; b < K; ++b)
                if (b != a) v *= (tt - (double)(j0 + b)) / (double)(a - b);
            g.fidx[(size_t)kp * K + a] = j0 + a + M / 2;
            g.fw[(size_t)kp * K + a] = v;
        }
    }
    for (int k = -M / 2; k < 0; ++k) {
        const int kp = k + M / 2, km = -k + M / 2;
        for (int a = 0; a < K; ++a) {
            g.fidx[(size_t)kp * K + a] = n1 - 1 - g.fidx[(size_t)km * K + (K - 1 - a)];
            g.fw[(size_t)kp * K + a] = g.fw[(size_t)km * K + (K - 1 - a)];
        }
    }
    std::vector<std::vector<std::pair<int, double>>> cols(n1);
    for (int kp = 0; kp < n1; ++kp)
        for (int a = 0; a < K; ++a) {
            const double w = g.fw[(size_t)kp * K + a];
            if (w != 0.0) cols[g.fidx[(size_t)kp * K + a]].push_back({kp, w});
        }
    for (auto &c : cols) g.KT = std::max<int>(g.KT, (int)c.size());
    g.tidx.assign((size_t)n1 * g.KT, 0);
    g.tw.assign((size_t)n1 * g.KT, 0.0);
    for (int j = 0; j < n1; ++j)
        for (size_t a = 0; a < cols[j].size(); ++a) {
            g.tidx[(size_t)j * g.KT + a] = cols[j][a].first;
            g.tw[(size_t)j * g.KT + a] = cols[j][a].second;
        }
    return g;
}

template <typename T, typename S>
int upload(T **dst, const std::vector<S> &src, cudaStream_t s)
{
    std::vector<T> h(src.begin(), src.end());
    RBF_TRY(rbf_alloc(dst, h.size()));
    RBF_CUDA_TRY(cudaMemcpyAsync(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

template <typename R>
int build_nested(rbf_tree *t, rbf_plan *p, cudaStream_t s)
{
    using C = cplx<R>;
    const int d = t->d, D = t->D, M = p->M, n1 = p->n1;
    const int64_t ms = p->mstride;
    // Lagrange stencils and their transpose
    const LagTables g = lagrange_tables(M, p->lagK);
    p->lagKT = g.KT;
    RBF_TRY(upload(&p->lag_fidx, g.fidx, s));
    RBF_TRY(upload(&p->lag_tidx, g.tidx, s));
    R *fw = nullptr, *tw = nullptr;
    RBF_TRY(upload(&fw, g.fw, s));
    p->lag_fw = fw;
    RBF_TRY(upload(&tw, g.tw, s));
    p->lag_tw = tw;
    // level-independent translation phases, e^{i theta k q}
    const double theta = 0.5 * M_PI * t->side / p->L;
    std::vector<double> phr((size_t)kPhRows * n1), phi((size_t)kPhRows * n1);
    auto put = [&](int row, double q) {
        for (int j = 0; j < n1; ++j) {
            const double ang = theta * (double)(j - M / 2) * q;
            phr[(size_t)row * n1 + j] = std::cos(ang);
            phi[(size_t)row * n1 + j] = std::sin(ang);
        }
    };
    for (int b = 0; b < 2; ++b) {
        const double h = (2 * b - 1) * 0.5;
        put(kPhVt + b, -h);
        put(kPhM2M + b, -0.5 * h);
        put(kPhL2L + b, 0.5 * h);
        for (int e = 0; e < 3; ++e) put(kPhPar + 3 * b + e, h - 2.0 * (e - 1));
    }
    for (int e = 0; e < 3; ++e) put(kPhNb + e, -(double)(e - 1));
    std::vector<C> ph(phr.size());
    for (size_t i = 0; i < ph.size(); ++i) {
        ph[i].x = (R)phr[i];
        ph[i].y = (R)phi[i];
    }
    C *phd = nullptr;
    RBF_TRY(rbf_alloc(&phd, ph.size()));
    p->nest_ph = phd;
    RBF_CUDA_TRY(cudaMemcpyAsync(phd, ph.data(), ph.size() * sizeof(C), cudaMemcpyHostToDevice, s));
    // leaf grid nodes
    std::vector<double> xi(n1);
    const double LD = p->L * std::ldexp(1.0, 2 - D);
    for (int j = 0; j < n1; ++j) xi[j] = (j - M / 2) * (2.0 * M_PI / LD);
    R *xid = nullptr;
    RBF_TRY(upload(&xid, xi, s));
    p->nest_xi = xid;
    // coefficients of every coupling level
    for (int l = 2; l <= D; ++l) {
        R *wc = nullptr;
        RBF_TRY(rbf_alloc(&wc, p->nmode));
        p->nest_wc[l] = wc;
        RBF_TRY(rbf_make_omegaC(p->prec, d, p->kernel, p->eps, M, p->L * std::ldexp(1.0, 2 - l),
                                p->alpha, t->side * std::ldexp(1.0, 2 - l), 1, p->nmode, wc, s));
    }
    // neighbour tables of levels 1..D-1 (the parents' neighbours in M2L)
    int nq = 1;
    for (int q = 0; q < d; ++q) nq *= 3;
    for (int l = 1; l < D; ++l) {
        const int nb = t->lev[l].nbox;
        RBF_TRY(rbf_alloc(&p->nest_nbr[l], (size_t)std::max(nb, 1) * nq));
        if (nb > 0) {
            k_build_nbr<<<ceil_div((int64_t)nb * nq, 256), 256, 0, s>>>(t->lev[l].key, nb, d, l, nq,
                                                                         p->nest_nbr[l]);
            RBF_LAUNCH_CHECK();
        }
    }
    // blocks of 4^d boxes around the children of every parent, levels 2..D
    int nq4 = 1;
    for (int q = 0; q < d; ++q) nq4 *= 4;
    for (int l = 2; l <= D; ++l) {
        const int np = t->lev[l - 1].nbox;
        RBF_TRY(rbf_alloc(&p->nest_nb4[l], (size_t)std::max(np, 1) * nq4));
        if (np > 0) {
            k_build_nb4<<<ceil_div((int64_t)np * nq4, 256), 256, 0, s>>>(
                t->lev[l - 1].key, np, t->lev[l].key, t->lev[l].nbox, d, l, nq4, p->nest_nb4[l]);
            RBF_LAUNCH_CHECK();
        }
    }
    // workspace
    for (int l = 1; l < D; ++l) {
        C *v = nullptr;
        RBF_TRY(rbf_alloc(&v, (size_t)t->lev[l].nbox * ms));
        p->nest_Vt[l] = v;
    }
    for (int l = 2; l < D; ++l) {
        C *v = nullptr;
        RBF_TRY(rbf_alloc(&v, (size_t)t->lev[l].nbox * ms));
        p->nest_L[l] = v;
    }
    if (D >= 3 && d >= 2) {
        for (int q = 0; q < 2; ++q) {
            C *v = nullptr;
            RBF_TRY(rbf_alloc(&v, (size_t)t->nleaf() * ms));
            p->nest_tmp[q] = v;
        }
    }
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

template <typename R, int DIM>
int run_nested(rbf_tree *t, const rbf_plan *p, const R *lam_s, R *u_far, cudaStream_t s)
{
    using C = cplx<R>;
    const int d = DIM, D = t->D, M = p->M, n1 = p->n1;
    const int64_t nmode = p->nmode, ms = p->mstride;
    const int64_t rows = nmode / p->n0;  // n1^(d-1)
    const int K = p->lagK, KT = p->lagKT;
    const C *ph = (const C *)p->nest_ph;
    const R *fw = (const R *)p->lag_fw, *tw = (const R *)p->lag_tw;
    C *tmp[2] = {(C *)p->nest_tmp[0], (C *)p->nest_tmp[1]};
    const unsigned ych = (unsigned)ceil_div(nmode, kThreads);
    auto stride_of = [&](int ax) {
        int64_t st = 1;
        for (int u = ax + 1; u < d; ++u) st *= n1;
        return st;
    };
    // P2M and L2P run on the leaf grid: a view of the plan with the leaf nodes
    rbf_plan leaf = *p;
    leaf.xi = p->nest_xi;
    RBF_TRY(rbf_run_p2m<R>(t, &leaf, lam_s, (C *)p->V[D], s));
    {
        int launches = 0;
        for (int l = D; l >= 2; --l) launches += l < 3 ? 1 : 1 + d;
        rbf_pass_timer tm(t, RBF_PASS_M2M, s, launches);
        for (int l = D; l >= 2; --l) {
            const rbf_level &lc = t->lev[l], &lp = t->lev[l - 1];
            k_vt<R, DIM><<<dim3(lp.nbox, ych), kThreads, 0, s>>>(M, n1, nmode, ms, ph, lp.child_off,
                                                                  lc.key, (const C *)p->V[l],
                                                                  (C *)p->nest_Vt[l - 1]);
            RBF_LAUNCH_CHECK();
            if (l < 3) continue;
            const C *src = (const C *)p->V[l];
            int pb = 0;
            for (int ax = d - 1; ax >= 1; --ax) {
                k_axis<R><<<(unsigned)lc.nbox * ych, kThreads, 0, s>>>(
                    n1, nmode, ms, stride_of(ax), K, p->lag_fidx, fw, src, tmp[pb], 0, (int)ych);
                RBF_LAUNCH_CHECK();
                src = tmp[pb];
                pb ^= 1;
            }
            k_m2m_last<R, DIM><<<(unsigned)lp.nbox * ych, kThreads, 0, s>>>(
                M, n1, nmode, ms, rows, K, p->lag_fidx, fw, ph, lp.child_off, lc.key, src,
                (C *)p->V[l - 1], (int)ych);
            RBF_LAUNCH_CHECK();
        }
    }
    {
        rbf_pass_timer tm(t, RBF_PASS_M2L, s, (D - 1) + (D - 2) * d);
        for (int l = 2; l <= D; ++l) {
            C *Ll = l == D ? (C *)p->Lleaf : (C *)p->nest_L[l];
            k_m2l_sib<R, DIM><<<dim3(t->lev[l - 1].nbox, ych), kThreads, 0, s>>>(
                M, n1, nmode, ms, ph, p->nest_nb4[l], p->nest_nbr[l - 1],
                (const C *)p->nest_Vt[l - 1], (const C *)p->V[l], (const R *)p->nest_wc[l], Ll);
            RBF_LAUNCH_CHECK();
        }
        for (int l = 3; l <= D; ++l) {
            const rbf_level &lv = t->lev[l];
            C *Ll = l == D ? (C *)p->Lleaf : (C *)p->nest_L[l];
            const C *Lp = (const C *)p->nest_L[l - 1];
            if (d == 1) {
                k_l2l_first<R, DIM><<<(unsigned)lv.nbox * ych, kThreads, 0, s>>>(
                    M, n1, nmode, ms, rows, KT, p->lag_tidx, tw, ph, lv.parent, lv.key, Lp, Ll, 1,
                    (int)ych);
                RBF_LAUNCH_CHECK();
                continue;
            }
            k_l2l_first<R, DIM><<<(unsigned)lv.nbox * ych, kThreads, 0, s>>>(
                M, n1, nmode, ms, rows, KT, p->lag_tidx, tw, ph, lv.parent, lv.key, Lp, tmp[0], 0,
                (int)ych);
            RBF_LAUNCH_CHECK();
            const C *src = tmp[0];
            int pb = 1;
            for (int ax = 1; ax < d; ++ax) {
                const bool last = ax == d - 1;
                C *dst = last ? Ll : tmp[pb];
                k_axis<R><<<(unsigned)lv.nbox * ych, kThreads, 0, s>>>(
                    n1, nmode, ms, stride_of(ax), KT, p->lag_tidx, tw, src, dst, last, (int)ych);
                RBF_LAUNCH_CHECK();
                src = dst;
                pb ^= 1;
            }
        }
    }
    RBF_TRY(rbf_run_l2p<R>(t, &leaf, (const C *)p->Lleaf, u_far, s));
    return RBF_OK;
}

}  // namespace

int rbf_nested_build(rbf_tree *t, rbf_plan *p, cudaStream_t s)
{
    if (t->D < 2) return RBF_OK;  // no far field
    int st = p->prec == RBF_FP64 ? build_nested<double>(t, p, s) : build_nested<float>(t, p, s);
    if (st != RBF_OK) rbf_nested_free(p);
    return st;
}

void rbf_nested_free(rbf_plan *p)
{
    for (int l = 0; l <= RBF_MAX_DEPTH; ++l) {
        rbf_free(p->nest_wc[l]);
        rbf_free(p->nest_nbr[l]);
        rbf_free(p->nest_nb4[l]);
        p->nest_nb4[l] = nullptr;
        rbf_free(p->nest_Vt[l]);
        rbf_free(p->nest_L[l]);
        p->nest_wc[l] = p->nest_Vt[l] = p->nest_L[l] = nullptr;
        p->nest_nbr[l] = nullptr;
    }
    rbf_free(p->nest_xi);
    rbf_free(p->nest_ph);
    rbf_free(p->lag_fidx);
    rbf_free(p->lag_fw);
    rbf_free(p->lag_tidx);
    rbf_free(p->lag_tw);
    rbf_free(p->nest_tmp[0]);
    rbf_free(p->nest_tmp[1]);
    p->nest_xi = p->nest_ph = p->lag_fw = p->lag_tw = nullptr;
    p->lag_fidx = p->lag_tidx = nullptr;
    p->nest_tmp[0] = p->nest_tmp[1] = nullptr;
    p->lagKT = 0;
}

template <typename R>
int rbf_run_far_nested(rbf_tree *t, const rbf_plan *p, const R *lam_s, R *u_far, cudaStream_t s)
{
    RBF_REQUIRE(p->grid == RBF_GRID_NESTED && p->nest_ph, "rbf_run_far_nested: plan has no nested grids");
    switch (t->d) {
    case 1: return run_nested<R, 1>(t, p, lam_s, u_far, s);
    case 2: return run_nested<R, 2>(t, p, lam_s, u_far, s);
    case 3: return run_nested<R, 3>(t, p, lam_s, u_far, s);
    default:
        rbf_set_error("nested grids are built for d <= 3");
        return RBF_ENOTSUP;
    }
}

template int rbf_run_far_nested<float>(rbf_tree *, const rbf_plan *, const float *, float *, cudaStream_t);
template int rbf_run_far_nested<double>(rbf_tree *, const rbf_plan *, const double *, double *,
                                        cudaStream_t);
