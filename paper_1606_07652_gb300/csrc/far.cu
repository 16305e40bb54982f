// far.cu -- far field of the band-limited FMM on the device.
//
//   P2M  (Eq. (P2M)):  V_b(xi) = sum_{j in G_b} lambda_j e^{-i xi.(x_j - c_b)}
//   M2M  (Eq. (43), interpolation P = I on one shared grid):
//        V_p(xi) = sum_{children c} e^{-i xi.(c_c - c_p)} V_c(xi),  up to the root
//   M2L  (Eq. (45)) and L2L (Eq. (48)) on the shared grid: every translation
//        is diagonal and e^{i xi.(c_a - c_l)} e^{i xi.(c_l - c_{l-1})} ... telescopes,
//        so the coupling of all levels 2..D followed by the downsweep to leaf a is
//          L_a(xi) = omega C(xi) [ e^{i xi.(c_a - c_0)} V_0(xi)
//                                  - sum_{b in N_a} e^{i xi.(c_a - c_b)} V_b(xi) ],
//        because N_a together with IL_2(a) .. IL_D(a) covers every leaf exactly once.
//   L2P  (Eq. (46)):   u_i = Re sum_xi e^{i xi.(x_i - c_a)} L_a(xi)
//
// Expansions hold the half spectrum k0 >= 0 (row-major, see rbf_internal.cuh);
// the weight 2 of the k0 > 0 half is inside omegaC.  P2M and L2P are dense
// per-leaf contractions  V[row][col] = sum_j A_j[row] B_j[col]  with
// A_j[row] = lambda_j prod_{t<d-1} E_t[j][k_t] and B_j[col] = E_{d-1}[j][col],
// E_t[j][k] = e^{-+ i xi_k (x_{j,t} - c_t)}: each thread owns one row and keeps
// its NC columns in registers, the per-point phase tables sit in shared memory.
#include <algorithm>

#include "rbf_internal.cuh"

namespace {

template <typename R>
struct FarArgs {
    int d, M, D, n0, n1, nrow, ncol;
    int64_t nmode, N;
    double lo[RBF_MAX_DIM];
    double side;
    const R *xs;           // SoA [d][N]
    const R *lam;          // [N] sorted order
    const int32_t *leaf_off;
    const uint64_t *leaf_key;
    const R *xi;           // [n1]
    cplx<R> *V;            // [nleaf][nmode] (P2M out)
    const cplx<R> *Lx;     // [nleaf][nmode] (L2P in)
    R *u;                  // [N] (L2P out)
    int pch;               // points per shared-memory chunk
};

__device__ __forceinline__ void decode_key(uint64_t key, int d, int l, int *k)
{
    for (int t = 0; t < d; ++t) k[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) k[t] |= (int)((key >> (b * d + t)) & 1u) << b;
}

// Fill the per-point phase tables of one chunk:
//   dim 0: E0[p][k0] = s0 * e^{sign i xi_{k0} r_0}, k0 = 0..M/2  (s0 = lambda_p or 1)
//   dim t>=1: Et[p][j] = e^{sign i xi_{j-M/2} r_t}, j = 0..M
template <typename R>
__device__ void fill_tables(const FarArgs<R> &a, int64_t p0, int cnt, const double *c,
                            R sign, bool with_lambda, cplx<R> *E)
{
    const int rowlen = a.n0 + (a.d - 1) * a.n1;
    for (int idx = threadIdx.x; idx < cnt * rowlen; idx += blockDim.x) {
        int p = idx / rowlen, j = idx - p * rowlen;
        int t, kidx;
        if (j < a.n0) {
            t = 0;
            kidx = j + a.M / 2;
        } else {
            t = 1 + (j - a.n0) / a.n1;
            kidx = (j - a.n0) % a.n1;
        }
        R r = a.xs[(int64_t)t * a.N + p0 + p] - (R)c[t];
        R s, co;
        sincos_r(sign * a.xi[kidx] * r, &s, &co);
        cplx<R> e;
        e.x = co;
        e.y = s;
        if (t == 0 && with_lambda) {
            R l = a.lam[p0 + p];
            e.x *= l;
            e.y *= l;
        }
        E[idx] = e;
    }
}

__device__ __forceinline__ void leaf_centre(const uint64_t key, int d, int D, const double *lo,
                                            double side, double *c)
{
    int k[RBF_MAX_DIM];
    decode_key(key, d, D, k);
    double w = side / (double)(1 << D);
    for (int t = 0; t < d; ++t) c[t] = lo[t] + ((double)k[t] + 0.5) * w;
}

// row -> (k0 index 0..M/2, k_t index 0..M for 1 <= t < d-1)
__device__ __forceinline__ void decode_row(int row, int d, int n1, int *kk)
{
    for (int t = d - 2; t >= 1; --t) {
        kk[t] = row % n1;
        row /= n1;
    }
    kk[0] = row;
}

// ------------------------------------------------------------------ P2M ---
template <typename R, int NC>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512) k_p2m(FarArgs<R> a)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *E = reinterpret_cast<C *>(smem_raw);
    const int rowlen = a.n0 + (a.d - 1) * a.n1;
    const int leaf = blockIdx.x;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = a.leaf_off[leaf + 1] - (int)p0;
    double c[RBF_MAX_DIM];
    leaf_centre(a.leaf_key[leaf], a.d, a.D, a.lo, a.side, c);
    const int nchunk = (np + a.pch - 1) / a.pch;
    if (nchunk == 1) {
        fill_tables<R>(a, p0, np, c, (R)-1, true, E);
        __syncthreads();
    }
    for (int row0 = 0; row0 < a.nrow; row0 += blockDim.x) {
        const int row = row0 + threadIdx.x;
        const bool active = row < a.nrow;
        int kk[RBF_MAX_DIM];
        decode_row(active ? row : 0, a.d, a.n1, kk);
        C acc[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) acc[q].x = acc[q].y = (R)0;
        for (int ch = 0; ch < nchunk; ++ch) {
            const int cnt = min(a.pch, np - ch * a.pch);
            if (nchunk > 1) {
                __syncthreads();
                fill_tables<R>(a, p0 + (int64_t)ch * a.pch, cnt, c, (R)-1, true, E);
                __syncthreads();
            }
            if (!active) continue;
            for (int p = 0; p < cnt; ++p) {
                const C *Ep = E + p * rowlen;
                C A;
                const C *B;
                if (a.d == 1) {
                    A.x = (R)1;
                    A.y = (R)0;
                    B = Ep;
                } else {
                    A = Ep[kk[0]];
                    for (int t = 1; t < a.d - 1; ++t) A = cmul(A, Ep[a.n0 + (t - 1) * a.n1 + kk[t]]);
                    B = Ep + a.n0 + (a.d - 2) * a.n1;
                }
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    if (q < a.ncol) cmac(acc[q], A, B[q]);
            }
        }
        if (active) {
            C *out = a.V + (int64_t)leaf * a.nmode + (int64_t)row * a.ncol;
#pragma unroll
            for (int q = 0; q < NC; ++q)
                if (q < a.ncol) out[q] = acc[q];
        }
    }
}

// ------------------------------------------------------------------ L2P ---
template <typename R, int NC>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 256 : 512) k_l2p(FarArgs<R> a)
{
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rowlen = a.n0 + (a.d - 1) * a.n1;
    C *E = reinterpret_cast<C *>(smem_raw);
    R *part = reinterpret_cast<R *>(E + (size_t)a.pch * rowlen);  // [nwarp][pch]
    const int nwarp = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int leaf = blockIdx.x;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = a.leaf_off[leaf + 1] - (int)p0;
    double c[RBF_MAX_DIM];
    leaf_centre(a.leaf_key[leaf], a.d, a.D, a.lo, a.side, c);
    const C *Lleaf = a.Lx + (int64_t)leaf * a.nmode;
    for (int ch0 = 0; ch0 < np; ch0 += a.pch) {
        const int cnt = min(a.pch, np - ch0);
        __syncthreads();
        fill_tables<R>(a, p0 + ch0, cnt, c, (R)1, false, E);
        for (int q = threadIdx.x; q < nwarp * a.pch; q += blockDim.x) part[q] = (R)0;
        __syncthreads();
        for (int row0 = 0; row0 < a.nrow; row0 += blockDim.x) {
            const int row = row0 + threadIdx.x;
            const bool active = row < a.nrow;
            int kk[RBF_MAX_DIM];
            decode_row(active ? row : 0, a.d, a.n1, kk);
            C Lr[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                if (active && q < a.ncol) Lr[q] = Lleaf[(int64_t)row * a.ncol + q];
                else Lr[q].x = Lr[q].y = (R)0;
            }
            for (int p = 0; p < cnt; ++p) {
                const C *Ep = E + p * rowlen;
                C P;
                P.x = P.y = (R)0;
                const C *B = (a.d == 1) ? Ep : Ep + a.n0 + (a.d - 2) * a.n1;
#pragma unroll
                for (int q = 0; q < NC; ++q)
                    if (q < a.ncol) cmac(P, Lr[q], B[q]);
                R v;
                if (a.d == 1) {
                    v = P.x;
                } else {
                    C A = Ep[kk[0]];
                    for (int t = 1; t < a.d - 1; ++t) A = cmul(A, Ep[a.n0 + (t - 1) * a.n1 + kk[t]]);
                    v = A.x * P.x - A.y * P.y;
                }
                if (!active) v = (R)0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) part[warp * a.pch + p] += v;
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            R s = (R)0;
            for (int w = 0; w < nwarp; ++w) s += part[w * a.pch + p];
            a.u[p0 + ch0 + p] = s;
        }
    }
}

// ------------------------------------------------------------------ M2M ---
// Parents at level l from their children at level l+1 (child width wc).
template <typename R>
__global__ void k_m2m(int d, int M, int n1, int64_t nmode, const R *xi, double wc,
                      const int32_t *child_off, const uint64_t *child_key, const cplx<R> *Vc,
                      cplx<R> *Vp)
{
    using C = cplx<R>;
    const int64_t m = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    const int p = blockIdx.x;
    // per-dimension half shift e^{-i xi_k wc/2}
    C P[RBF_MAX_DIM];
    int64_t r = m;
    for (int t = d - 1; t >= 0; --t) {
        int kidx;
        if (t > 0) {
            kidx = (int)(r % n1);
            r /= n1;
        } else {
            kidx = (int)r + M / 2;
        }
        R s, co;
        sincos_r(-xi[kidx] * (R)(0.5 * wc), &s, &co);
        P[t].x = co;
        P[t].y = s;
    }
    C acc;
    acc.x = acc.y = (R)0;
    const int c0 = child_off[p], c1 = child_off[p + 1];
    for (int cidx = c0; cidx < c1; ++cidx) {
        const unsigned bits = (unsigned)(child_key[cidx] & ((1u << d) - 1u));
        C ph = (bits & 1u) ? P[0] : cconj(P[0]);
        for (int t = 1; t < d; ++t) ph = cmul(ph, ((bits >> t) & 1u) ? P[t] : cconj(P[t]));
        cmac(acc, ph, Vc[(int64_t)cidx * nmode + m]);
    }
    Vp[(int64_t)p * nmode + m] = acc;
}

// ------------------------------------------------------------------ M2L ---
// Telescoped coupling + downsweep at the leaves (see file header).  The
// neighbours of the leaf are placed on their 3^d offset grid in shared memory
// and the offset phases are summed one dimension at a time.
template <typename R>
__global__ void k_m2l(int d, int M, int D, int n1, int64_t nmode, const R *xi, const R *omegaC,
                      double wD, const cplx<R> *root_ph, const uint64_t *leaf_key,
                      const int32_t *near_off, const int32_t *near_idx, const cplx<R> *V0,
                      const cplx<R> *VD, cplx<R> *Lx)
{
    using C = cplx<R>;
    __shared__ int32_t grid[729];
    const int a = blockIdx.x;
    int ka[RBF_MAX_DIM];
    decode_key(leaf_key[a], d, D, ka);
    int ngrid = 1;
    for (int t = 0; t < d; ++t) ngrid *= 3;
    for (int q = threadIdx.x; q < ngrid; q += blockDim.x) grid[q] = -1;
    __syncthreads();
    for (int e = near_off[a] + threadIdx.x; e < near_off[a + 1]; e += blockDim.x) {
        int b = near_idx[e];
        int kb[RBF_MAX_DIM];
        decode_key(leaf_key[b], d, D, kb);
        int g = 0, stride = 1;
        for (int t = 0; t < d; ++t) {
            g += (kb[t] - ka[t] + 1) * stride;
            stride *= 3;
        }
        grid[g] = b;
    }
    __syncthreads();
    const int64_t m = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    int kidx[RBF_MAX_DIM];
    {
        int64_t r = m;
        for (int t = d - 1; t >= 1; --t) {
            kidx[t] = (int)(r % n1);
            r /= n1;
        }
        kidx[0] = (int)r + M / 2;
    }
    // Q_t = e^{-i xi_k wD}: phase of a neighbour one box up in dimension t
    C Q[RBF_MAX_DIM];
    for (int t = 0; t < d; ++t) {
        R s, co;
        sincos_r(-xi[kidx[t]] * (R)wD, &s, &co);
        Q[t].x = co;
        Q[t].y = s;
    }
    // root term e^{i xi.(c_a - c_0)} V_0
    const int64_t nk = (int64_t)1 << D;
    C ph = root_ph[((int64_t)0 * nk + ka[0]) * n1 + kidx[0]];
    for (int t = 1; t < d; ++t) ph = cmul(ph, root_ph[((int64_t)t * nk + ka[t]) * n1 + kidx[t]]);
    C acc = cmul(ph, V0[m]);
    // near subtraction, grouped by the offsets of dimensions 0..d-2
    const int ngroup = ngrid / 3;
    const int tl = d - 1;
    for (int g = 0; g < ngroup; ++g) {
        // grid index: sum_t (delta_t + 1) 3^t; the last dimension has stride 3^{d-1}
        const int bm = grid[g], bz = grid[g + ngroup], bp = grid[g + 2 * ngroup];
        if (bm < 0 && bz < 0 && bp < 0) continue;
        C inner;
        inner.x = inner.y = (R)0;
        if (bz >= 0) {
            C v = VD[(int64_t)bz * nmode + m];
            inner.x += v.x;
            inner.y += v.y;
        }
        if (bp >= 0) cmac(inner, Q[tl], VD[(int64_t)bp * nmode + m]);
        if (bm >= 0) cmac(inner, cconj(Q[tl]), VD[(int64_t)bm * nmode + m]);
        // factor of the other dimensions
        int gg = g;
        C f;
        f.x = (R)1;
        f.y = (R)0;
        for (int t = 0; t < tl; ++t) {
            int dl = gg % 3 - 1;
            gg /= 3;
            if (dl == 1) f = cmul(f, Q[t]);
            else if (dl == -1) f = cmul(f, cconj(Q[t]));
        }
        C prod = cmul(f, inner);
        acc.x -= prod.x;
        acc.y -= prod.y;
    }
    const R w = omegaC[m];
    C out;
    out.x = w * acc.x;
    out.y = w * acc.y;
    Lx[(int64_t)a * nmode + m] = out;
}

template <typename R>
int pick_block(int nrow)
{
    const int bmax = sizeof(R) == 8 ? 256 : 512;
    int best = 128, best_waste = 1 << 30;
    for (int bd = 128; bd <= bmax; bd += 32) {
        int passes = (nrow + bd - 1) / bd;
        int waste = passes * bd - nrow;
        if (waste < best_waste || (waste == best_waste && bd > best)) {
            best = bd;
            best_waste = waste;
        }
    }
    return best;
}

template <typename R, int NC>
int launch_p2m_l2p(bool l2p, const FarArgs<R> &a, int nleaf, cudaStream_t s)
{
    const int bd = pick_block<R>(a.nrow);
    const int rowlen = a.n0 + (a.d - 1) * a.n1;
    size_t smem = (size_t)a.pch * rowlen * sizeof(cplx<R>);
    if (l2p) smem += (size_t)(bd / 32) * a.pch * sizeof(R);
    if (l2p) {
        RBF_CUDA_TRY(cudaFuncSetAttribute(k_l2p<R, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        k_l2p<R, NC><<<nleaf, bd, smem, s>>>(a);
    } else {
        RBF_CUDA_TRY(cudaFuncSetAttribute(k_p2m<R, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        k_p2m<R, NC><<<nleaf, bd, smem, s>>>(a);
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

template <typename R>
int dispatch_p2m_l2p(bool l2p, const FarArgs<R> &a, int nleaf, cudaStream_t s)
{
    const int nc = a.ncol;
    if (nc <= 9) return launch_p2m_l2p<R, 9>(l2p, a, nleaf, s);
    if (nc <= 17) return launch_p2m_l2p<R, 17>(l2p, a, nleaf, s);
    if (nc <= 25) return launch_p2m_l2p<R, 25>(l2p, a, nleaf, s);
    if (nc <= 33) return launch_p2m_l2p<R, 33>(l2p, a, nleaf, s);
    if (nc <= 41) return launch_p2m_l2p<R, 41>(l2p, a, nleaf, s);
    if (nc <= 49) return launch_p2m_l2p<R, 49>(l2p, a, nleaf, s);
    return launch_p2m_l2p<R, 65>(l2p, a, nleaf, s);
}

}  // namespace

template <typename R>
int rbf_run_far(rbf_tree *t, const rbf_plan *p, const R *lam_s, R *u_far, cudaStream_t s)
{
    using C = cplx<R>;
    const int d = t->d, D = t->D;
    const int nleaf = t->nleaf();
    FarArgs<R> a;
    a.d = d;
    a.M = p->M;
    a.D = D;
    a.n0 = p->n0;
    a.n1 = p->n1;
    a.nrow = p->nrow;
    a.ncol = p->ncol;
    a.nmode = p->nmode;
    a.N = t->N;
    for (int q = 0; q < RBF_MAX_DIM; ++q) a.lo[q] = t->lo[q];
    a.side = t->side;
    a.xs = (const R *)(sizeof(R) == 8 ? (const void *)t->xs64 : (const void *)t->xs32);
    a.lam = lam_s;
    a.leaf_off = t->leaf_off;
    a.leaf_key = t->leaf_key();
    a.xi = (const R *)p->xi;
    a.V = (C *)p->V[D];
    a.Lx = (const C *)p->Lleaf;
    a.u = u_far;
    const int rowlen = a.n0 + (d - 1) * a.n1;
    // chunk size: as many points as fit in ~96 KB of phase tables, at most 64
    a.pch = (int)std::max<int64_t>(1, std::min<int64_t>(64, (96 * 1024) / ((int64_t)rowlen * sizeof(C))));
    // P2M at the leaves
    {
        rbf_pass_timer tm(t, RBF_PASS_P2M, s);
        RBF_TRY(dispatch_p2m_l2p<R>(false, a, nleaf, s));
    }
    // M2M up to the root
    const int mb = 256;
    const int mchunks = ceil_div(p->nmode, mb);
    RBF_REQUIRE(mchunks < 65536, "expansion too large (%lld modes)", (long long)p->nmode);
    {
    rbf_pass_timer tm(t, RBF_PASS_M2M, s, D);
    for (int l = D - 1; l >= 0; --l) {
        const double wc = t->side / (double)(1 << (l + 1));
        dim3 grid(t->lev[l].nbox, mchunks);
        k_m2m<R><<<grid, mb, 0, s>>>(d, p->M, p->n1, p->nmode, (const R *)p->xi, wc,
                                     t->lev[l].child_off, t->lev[l + 1].key,
                                     (const C *)p->V[l + 1], (C *)p->V[l]);
        RBF_LAUNCH_CHECK();
    }
    }
    // coupling + downsweep at the leaves
    {
        rbf_pass_timer tm(t, RBF_PASS_M2L, s);
        const double wD = t->side / (double)(1 << D);
        dim3 grid(nleaf, mchunks);
        k_m2l<R><<<grid, mb, 0, s>>>(d, p->M, D, p->n1, p->nmode, (const R *)p->xi,
                                     (const R *)p->omegaC, wD, (const C *)p->root_ph, t->leaf_key(),
                                     t->near_off, t->near_idx, (const C *)p->V[0],
                                     (const C *)p->V[D], (C *)p->Lleaf);
        RBF_LAUNCH_CHECK();
    }
    // L2P
    {
        rbf_pass_timer tm(t, RBF_PASS_L2P, s);
        RBF_TRY(dispatch_p2m_l2p<R>(true, a, nleaf, s));
    }
    return RBF_OK;
}

template int rbf_run_far<float>(rbf_tree *, const rbf_plan *, const float *, float *, cudaStream_t);
template int rbf_run_far<double>(rbf_tree *, const rbf_plan *, const double *, double *,
                                 cudaStream_t);
