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
// E_t[j][k] = e^{-+ i xi_k (x_{j,t} - c_t)}, the per-point phase tables in shared
// memory.  P2M: a thread accumulates one row times a segment of columns.  FP32 L2P
// (k_l2p_horner2): a warp pair shares 32 rows, each thread holds half a row of the
// local expansion in registers and sums its columns by Horner's rule in
// z = e^{i dxi (x_{j,d-1} - c_{d-1})}, in groups of 8 columns shifted by the
// group's start phase.  3-D M2L (k_m2l_pencil): pencils of 2 x 2 x 8 leaves, the
// three-tap stencil one dimension at a time with a window of three planes.
#include <algorithm>
#include <type_traits>

#include "rbf_internal.cuh"

// tuning knobs of the FP32 P2M/L2P tiles: point-loop unroll, rows per thread,
// column groups.  Each kernel is built in two launch shapes, picked per product:
// "dense" (leaves of up to 96 points on average and column segments of at most
// 36): five resident CTAs of up to 192 threads per SM, 52-point P2M chunks
// and, for leaves of up to 32 points, 26-point L2P chunks, so that five CTAs'
// tables fit in shared memory; "wide": four CTAs of up to 256 threads (192 for
// column segments wider than 36, three CTAs for segments wider than 52) and
// 64- / 32-point chunks, fewer chunks for large leaves.  (Measured: 3-D M = 32 product
// 16.87 -> 16.54 ms and the 256-problem batch faster with the dense shape; 5-D
// leaves of 512 points keep the wide one.)
#ifndef RBF_FAR_UNROLL
#define RBF_FAR_UNROLL 1
#endif
#ifndef RBF_FAR_RPT
#define RBF_FAR_RPT 1
#endif
#ifndef RBF_FAR_NH
#define RBF_FAR_NH 2
#endif
#ifndef RBF_L2P_RPT
#define RBF_L2P_RPT RBF_FAR_RPT
#endif
#ifndef RBF_L2P_NH
#define RBF_L2P_NH RBF_FAR_NH
#endif
#ifndef RBF_DENSE_BMAX
#define RBF_DENSE_BMAX 192
#endif
#ifndef RBF_DENSE_MINB
#define RBF_DENSE_MINB 5
#endif
#ifndef RBF_WIDE_BMAX
#define RBF_WIDE_BMAX 256
#endif
#ifndef RBF_WIDE_MINB
#define RBF_WIDE_MINB 4
#endif
#ifndef RBF_P2M_PCH_DENSE
#define RBF_P2M_PCH_DENSE 52
#endif
#ifndef RBF_P2M_PCH_WIDE
#define RBF_P2M_PCH_WIDE 64
#endif
#ifndef RBF_L2P_PCH_DENSE
#define RBF_L2P_PCH_DENSE 26
#endif
#ifndef RBF_L2P_PCH_WIDE
#define RBF_L2P_PCH_WIDE 32
#endif
#ifndef RBF_L2P_NARROW
#define RBF_L2P_NARROW 36
#endif
// FP32 L2P points per step of the point loop (1 or 2; the tail of an odd count
// takes the one-point step).  Two: 6.39 -> 6.20 ms at the 3-D M = 32 product.
// (The same step in P2M spills under the 64-register bound.)
#ifndef RBF_L2P_POINTS
#define RBF_L2P_POINTS 2
#endif
// FP32 3-D grouped coupling: modes per thread (1 or 2; two need 141 registers and ran
// slower, 3.53 against 3.42 ms at the 3-D M = 32 product)
#ifndef RBF_M2L_MP
#define RBF_M2L_MP 1
#endif
// 3-D coupling by pencils of 2 x 2 x 8 leaves (1) or by parent blocks (0)
#ifndef RBF_M2L_PENCIL
#define RBF_M2L_PENCIL 1
#endif
#ifndef RBF_M2L_PENCIL_MINB
#define RBF_M2L_PENCIL_MINB 6          // resident CTAs of the FP32 pencil kernel (80 registers)
#endif
// grouped coupling: resident CTAs of 128 threads the register budget targets
// (8: 64 registers, no spills; 3.43 -> 3.25 ms against the compiler's 71 registers)
#ifndef RBF_M2L_MINB
#define RBF_M2L_MINB 8                 // resident CTAs of 128 threads: 64 registers, no spills
#endif
#if RBF_M2L_MINB > 0
#define RBF_M2L_BOUNDS __launch_bounds__(128, RBF_M2L_MINB)
#else
#define RBF_M2L_BOUNDS __launch_bounds__(128)
#endif
// L2P partial sums: 1 = one shared-memory slot per thread and point, reduced
// once per chunk; 0 = warp shuffles per point
#ifndef RBF_L2P_SMEMRED
#define RBF_L2P_SMEMRED 1
#endif

namespace {

constexpr int kFarUnroll = RBF_FAR_UNROLL;
constexpr int kL2PPoints = RBF_L2P_POINTS;
static_assert(kL2PPoints == 1 || kL2PPoints == 2, "RBF_L2P_POINTS must be 1 or 2");
// largest block of a launch shape: the wide shape keeps 256 threads for narrow
// column segments and drops to 192 (more registers per thread) for wider ones
constexpr int far_bmax(bool dense, int nce)
{
    return dense ? RBF_DENSE_BMAX : (nce <= RBF_L2P_NARROW ? RBF_WIDE_BMAX : RBF_DENSE_BMAX);
}
// resident CTAs per SM a launch shape is compiled for; the widest column
// segments (M > 50) drop to three so that their 34 columns per thread stay in
// registers (four CTAs of 192 threads spilled 192 bytes per thread)
constexpr int far_minb(bool dense, int nce)
{
    return dense ? RBF_DENSE_MINB : (nce <= 52 ? RBF_WIDE_MINB : 3);
}
// FP64 column groups: one, except for the widest segments (68 columns of FP64
// accumulators do not fit in 255 registers)
constexpr int far_nh64(int nce) { return nce > 52 ? 2 : 1; }

template <typename R>
struct FarArgs {
    int d, M, D, n0, n1, nrow, ncol;
    int64_t nmode, mstride, N;   // modes; per-box stride (multiple of 4)
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
    int seg0, seg;         // table segment lengths (even; seg >= columns read per point)
    int shape;             // P2M launch shape: 0 by rule, 1 dense, 2 wide (measured per plan)
};

__device__ __forceinline__ void decode_key(uint64_t key, int d, int l, int *k)
{
    for (int t = 0; t < d; ++t) k[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) k[t] |= (int)((key >> (b * d + t)) & 1u) << b;
}

// Per-point phase tables of one chunk, one segment per dimension, each segment
// padded to an even number of entries so that pairs of complex values can be
// read from shared memory with one 16-byte load:
//   dim 0:    E0[p][k0] = s0 * e^{sign i xi_{k0} r_0}, k0 = 0..M/2  (s0 = lambda_p or 1)
//   dim t>=1: Et[p][j]  = e^{sign i xi_{j-M/2} r_t}, j = 0..M
// Padding entries hold zero.
__host__ __device__ __forceinline__ int even_up(int n) { return (n + 1) & ~1; }

template <typename R>
__device__ void fill_tables(const FarArgs<R> &a, int64_t p0, int cnt, const double *c,
                            R sign, bool with_lambda, cplx<R> *E)
{
    const int seg0 = a.seg0, seg = a.seg;
    const int rowlen = seg0 + (a.d - 1) * seg;
    for (int idx = threadIdx.x; idx < cnt * rowlen; idx += blockDim.x) {
        int p = idx / rowlen, j = idx - p * rowlen;
        int t, kidx;
        bool pad;
        if (j < seg0) {
            t = 0;
            pad = j >= a.n0;
            kidx = j + a.M / 2;
        } else {
            t = 1 + (j - seg0) / seg;
            kidx = (j - seg0) % seg;
            pad = kidx >= a.n1;
        }
        cplx<R> e;
        if (pad) {
            e.x = e.y = (R)0;
        } else {
            R r = a.xs[(int64_t)t * a.N + p0 + p] - (R)c[t];
            R sn, co;
            sincos_r(sign * a.xi[kidx] * r, &sn, &co);
            e.x = co;
            e.y = sn;
            if (t == 0 && with_lambda) {
                R l = a.lam[p0 + p];
                e.x *= l;
                e.y *= l;
            }
        }
        E[idx] = e;
    }
}

__device__ __forceinline__ void ld2(const float2 *p, float2 &u, float2 &v)
{
    const float4 w = *reinterpret_cast<const float4 *>(p);
    u = make_float2(w.x, w.y);
    v = make_float2(w.z, w.w);
}
__device__ __forceinline__ void ld2(const double2 *p, double2 &u, double2 &v)
{
    u = p[0];
    v = p[1];
}

__device__ __forceinline__ void leaf_centre(const uint64_t key, int d, int D, const double *lo,
                                            double side, double *c)
{
    int k[RBF_MAX_DIM];
    decode_key(key, d, D, k);
    double w = side / (double)(1 << D);
    for (int t = 0; t < d; ++t) c[t] = lo[t] + ((double)k[t] + 0.5) * w;
}

// Shared-memory offsets of the row factors of one row (k0, k_1, .., k_{d-2}):
// o[0] = k0 in the dimension-0 segment, o[t] = seg0 + (t-1) seg + k_t.  Kept as
// scalars so that they stay in registers inside the point loop.
struct RowOff {
    int o0, o1, o2, o3, o4;
};

__device__ __forceinline__ RowOff row_offsets(int row, int d, int n1, int seg0, int seg)
{
    RowOff r;
    r.o1 = r.o2 = r.o3 = r.o4 = 0;
    // dimensions d-2 .. 1 are the fastest digits of the row index
    if (d >= 6) { r.o4 = seg0 + 3 * seg + row % n1; row /= n1; }
    if (d >= 5) { r.o3 = seg0 + 2 * seg + row % n1; row /= n1; }
    if (d >= 4) { r.o2 = seg0 + 1 * seg + row % n1; row /= n1; }
    if (d >= 3) { r.o1 = seg0 + row % n1; row /= n1; }
    r.o0 = row;
    return r;
}

// A_j[row] = E0[p][k0] prod_{1<=t<d-1} Et[p][k_t]  (1 for d == 1)
template <typename C>
__device__ __forceinline__ C row_factor(const C *Ep, int d, const RowOff &o)
{
    C A;
    if (d == 1) {
        A.x = 1;
        A.y = 0;
        return A;
    }
    A = Ep[o.o0];
    if (d >= 3) A = cmul(A, Ep[o.o1]);
    if (d >= 4) A = cmul(A, Ep[o.o2]);
    if (d >= 5) A = cmul(A, Ep[o.o3]);
    if (d >= 6) A = cmul(A, Ep[o.o4]);
    return A;
}

// ------------------------------------------------------------------ P2M ---
// Thread tile: RPT rows x NCH columns.  The NCE (>= ncol) columns are split in
// NH halves of NCH = NCE/NH (even) columns; warps alternate halves, so a half
// is warp-uniform.  Columns >= ncol are padding and are not stored.
template <int NH>
__device__ __forceinline__ void tile_coords(int &g, int &h, int &G)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    h = warp % NH;
    g = (warp / NH) * 32 + lane;
    G = blockDim.x / NH;
}

template <typename R, int NCE, int RPT, int NH, bool DENSE>
__global__ void __launch_bounds__(sizeof(R) == 4 ? far_bmax(DENSE, NCE) : 256,
                                  sizeof(R) == 4 ? far_minb(DENSE, NCE) : 1)
    k_p2m(FarArgs<R> a)
{
    using C = cplx<R>;
    constexpr int NCH = NCE / NH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *E = reinterpret_cast<C *>(smem_raw);
    const int seg0 = a.seg0, seg = a.seg;
    const int rowlen = seg0 + (a.d - 1) * seg;
    const int boff = a.d == 1 ? 0 : seg0 + (a.d - 2) * seg;
    int g, h, G;
    tile_coords<NH>(g, h, G);
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
    for (int row0 = 0; row0 < a.nrow; row0 += RPT * G) {
        int rows[RPT];
        bool act[RPT];
        RowOff ro[RPT];
        C acc[RPT][NCH];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            rows[r] = row0 + g + r * G;
            act[r] = rows[r] < a.nrow;
            ro[r] = row_offsets(act[r] ? rows[r] : 0, a.d, a.n1, seg0, seg);
#pragma unroll
            for (int q = 0; q < NCH; ++q) acc[r][q].x = acc[r][q].y = (R)0;
        }
        for (int ch = 0; ch < nchunk; ++ch) {
            const int cnt = min(a.pch, np - ch * a.pch);
            if (nchunk > 1) {
                __syncthreads();
                fill_tables<R>(a, p0 + (int64_t)ch * a.pch, cnt, c, (R)-1, true, E);
                __syncthreads();
            }
            if (!act[0]) continue;
#pragma unroll kFarUnroll
            for (int p = 0; p < cnt; ++p) {
                const C *Ep = E + p * rowlen;
                C A[RPT];
#pragma unroll
                for (int r = 0; r < RPT; ++r) A[r] = row_factor(Ep, a.d, ro[r]);
                const C *B = Ep + boff + h * NCH;
#pragma unroll
                for (int q = 0; q < NCH; q += 2) {
                    C b0, b1;
                    ld2(B + q, b0, b1);
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        cmac(acc[r][q], A[r], b0);
                        cmac(acc[r][q + 1], A[r], b1);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (!act[r]) continue;
            C *out = a.V + (int64_t)leaf * a.mstride + (int64_t)rows[r] * a.ncol + h * NCH;
#pragma unroll
            for (int q = 0; q < NCH; ++q)
                if (h * NCH + q < a.ncol) out[q] = acc[r][q];
        }
    }
}

// ------------------------------------------------------------------ L2P ---
template <typename R, int NCE, int RPT, int NH, bool DENSE>
__global__ void __launch_bounds__(sizeof(R) == 4 ? far_bmax(DENSE, NCE) : 256,
                                  sizeof(R) == 4 ? far_minb(DENSE, NCE) : 1)
    k_l2p(FarArgs<R> a)
{
    using C = cplx<R>;
    constexpr int NCH = NCE / NH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int seg0 = a.seg0, seg = a.seg;
    const int rowlen = seg0 + (a.d - 1) * seg;
    const int boff = a.d == 1 ? 0 : seg0 + (a.d - 2) * seg;
    C *E = reinterpret_cast<C *>(smem_raw);
    // partial sums: [pch][blockDim] (per thread) or [nwarp][pch] (per warp)
    R *part = reinterpret_cast<R *>(E + (size_t)a.pch * rowlen);
    const int nwarp = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int g, h, G;
    tile_coords<NH>(g, h, G);
    const int leaf = blockIdx.x;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = a.leaf_off[leaf + 1] - (int)p0;
    double c[RBF_MAX_DIM];
    leaf_centre(a.leaf_key[leaf], a.d, a.D, a.lo, a.side, c);
    const C *Lleaf = a.Lx + (int64_t)leaf * a.mstride;
    for (int ch0 = 0; ch0 < np; ch0 += a.pch) {
        const int cnt = min(a.pch, np - ch0);
        __syncthreads();
        fill_tables<R>(a, p0 + ch0, cnt, c, (R)1, false, E);
        const int npart = RBF_L2P_SMEMRED ? a.pch * (int)blockDim.x : nwarp * a.pch;
        for (int q = threadIdx.x; q < npart; q += blockDim.x) part[q] = (R)0;
        __syncthreads();
        for (int row0 = 0; row0 < a.nrow; row0 += RPT * G) {
            RowOff ro[RPT];
            C Lr[RPT][NCH];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int row = row0 + g + r * G;
                const bool act = row < a.nrow;
                ro[r] = row_offsets(act ? row : 0, a.d, a.n1, seg0, seg);
#pragma unroll
                for (int q = 0; q < NCH; ++q) {
                    const int col = h * NCH + q;
                    if (act && col < a.ncol) Lr[r][q] = Lleaf[(int64_t)row * a.ncol + col];
                    else Lr[r][q].x = Lr[r][q].y = (R)0;
                }
            }
            // adds one point's contribution v of this thread's rows to its partial sum
            auto deposit = [&](int p, R v) {
                if (RBF_L2P_SMEMRED) {
                    part[p * blockDim.x + threadIdx.x] += v;
                } else {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) part[warp * a.pch + p] += v;
                }
            };
            // Re sum_row A[row] P[row] for one point, P = this thread's column sums
            auto finish = [&](const C *Ep, const C (&P)[RPT]) {
                R v = (R)0;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    if (a.d == 1) {
                        v += P[r].x;
                    } else {
                        const C A = row_factor(Ep, a.d, ro[r]);
                        v += A.x * P[r].x - A.y * P[r].y;
                    }
                }
                return v;
            };
            int p = 0;
            if (kL2PPoints == 2 && sizeof(R) == 4) {
                // two points per step: one column sum per point and row, the two
                // points' FMA chains interleave
                for (; p + 1 < cnt; p += 2) {
                    const C *Ea = E + p * rowlen, *Eb = Ea + rowlen;
                    const C *Ba = Ea + boff + h * NCH, *Bb = Eb + boff + h * NCH;
                    C Pa[RPT], Pb[RPT];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) Pa[r].x = Pa[r].y = Pb[r].x = Pb[r].y = (R)0;
#pragma unroll
                    for (int q = 0; q < NCH; q += 2) {
                        C a0, a1, b0, b1;
                        ld2(Ba + q, a0, a1);
                        ld2(Bb + q, b0, b1);
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            cmac(Pa[r], Lr[r][q], a0);
                            cmac(Pb[r], Lr[r][q], b0);
                            cmac(Pa[r], Lr[r][q + 1], a1);
                            cmac(Pb[r], Lr[r][q + 1], b1);
                        }
                    }
                    deposit(p, finish(Ea, Pa));
                    deposit(p + 1, finish(Eb, Pb));
                }
            }
#pragma unroll kFarUnroll
            for (; p < cnt; ++p) {
                const C *Ep = E + p * rowlen;
                const C *B = Ep + boff + h * NCH;
                // four partial sums per row keep the FMA chains short
                C P4[RPT][4];
#pragma unroll
                for (int r = 0; r < RPT; ++r)
#pragma unroll
                    for (int k = 0; k < 4; ++k) P4[r][k].x = P4[r][k].y = (R)0;
#pragma unroll
                for (int q = 0; q < NCH; q += 2) {
                    C b0, b1;
                    ld2(B + q, b0, b1);
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        cmac(P4[r][(q >> 1) & 3], Lr[r][q], b0);
                        cmac(P4[r][(q >> 1) & 3], Lr[r][q + 1], b1);
                    }
                }
                C P[RPT];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    P[r].x = (P4[r][0].x + P4[r][1].x) + (P4[r][2].x + P4[r][3].x);
                    P[r].y = (P4[r][0].y + P4[r][1].y) + (P4[r][2].y + P4[r][3].y);
                }
                deposit(p, finish(Ep, P));
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            R sum = (R)0;
            if (RBF_L2P_SMEMRED) {
                // four interleaved partial sums, added in a fixed order
                const R *q = part + (size_t)p * blockDim.x;
                R s4[4] = {(R)0, (R)0, (R)0, (R)0};
                for (int t = 0; t < (int)blockDim.x; t += 4)
#pragma unroll
                    for (int k = 0; k < 4; ++k) s4[k] += q[t + k];
                sum = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            } else {
                for (int w = 0; w < nwarp; ++w) sum += part[w * a.pch + p];
            }
            a.u[p0 + ch0 + p] = sum;
        }
    }
}

// ------------------------------------------------------ L2P, FP32 Horner ---
// Along the column dimension (d-1; dimension 0 when d == 1) the phases of a
// point are powers of one unit-modulus number,
//     e^{i xi_c r} = z^(c - coff),  z = e^{i dxi r},  coff = M/2 (0 when d == 1),
// so the column sum of one mode row,  sum_c L[row][c] e^{i xi_c r},  is a
// polynomial in z.  The NCOL = 8 q + r columns are cut into q groups of 8 (the
// last one takes the r extra columns; a single group of r when q = 0).  Inside
// a group the sum is taken by Horner's rule (degree <= 14, so the rounding of z
// enters at most that often; with groups of 8 the FP32 error is that of the
// direct sum), and each group value is multiplied by the exact phase of the
// group's first column, e^{i xi_c0 r}, from the point's table.  The
// multiply-adds per mode are those of the direct sum (one complex multiply-
// add, 4 FP32 FMA), but the inner loop reads no shared memory: per point a
// thread loads z, its groups' phases and its row factor.
// A thread holds one whole mode row (NCOL <= 33 columns) in registers, loaded
// straight from global memory, and walks the leaf's points two at a time; the
// per-point sums of a warp are added by one transposed shuffle butterfly per
// four points and kept per warp.
constexpr int kHorner = 8;       // columns per Horner group (the last takes up to 7 more)
constexpr int kHornerMaxCol = 33;
constexpr int kHornerBlock = 192;  // 96 registers: three CTAs of six warps per SM
#ifndef RBF_L2P_SPLIT
#define RBF_L2P_SPLIT 1              // half a row per thread for rows of two groups or more
#endif
#ifndef RBF_L2P_BLOCK2
#define RBF_L2P_BLOCK2 256
#endif
constexpr int kHornerBlock2 = RBF_L2P_BLOCK2;
constexpr int kHornerPch = 64;     // points per table chunk

__device__ __forceinline__ float2 horner_step(float2 h, float2 z, float2 l)
{
    float2 r;
    r.x = fmaf(h.x, z.x, l.x);
    r.x = fmaf(-h.y, z.y, r.x);
    r.y = fmaf(h.x, z.y, l.y);
    r.y = fmaf(h.y, z.x, r.y);
    return r;
}

// groups of a row of NC columns: 8 columns each, the last one takes the rest
__host__ __device__ constexpr int horner_ng(int NC) { return NC >= kHorner ? NC / kHorner : 1; }
// columns held by a thread that takes groups GB .. GE-1 (from column 8 GB on)
__host__ __device__ constexpr int horner_held(int NC, int GB, int GE)
{
    return (GE >= horner_ng(NC) ? NC : kHorner * GE) - kHorner * GB;
}

// S_k (+)= ph_k * sum_{q<LEN} L[B+q] z_k^q for two points k
template <int NL, int LEN, int B, bool FIRST>
__device__ __forceinline__ void horner_group2(const float2 (&L)[NL], const float2 (&z)[2],
                                              const float2 (&ph)[2], float2 (&S)[2])
{
    float2 h[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) h[k] = L[B + LEN - 1];
#pragma unroll
    for (int q = LEN - 2; q >= 0; --q)
#pragma unroll
        for (int k = 0; k < 2; ++k) h[k] = horner_step(h[k], z[k], L[B + q]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (FIRST) S[k] = cmul(ph[k], h[k]);
        else cmac(S[k], ph[k], h[k]);
    }
}

// groups G .. GE-1 of a row whose held columns start at group GB; group g starts
// at column 8 g and its phase is rec[1 + g]
template <int NC, int GB, int GE, int G>
__device__ __forceinline__ void horner_groups(const float2 (&L)[horner_held(NC, GB, GE)],
                                              const float2 *ra, const float2 *rb,
                                              const float2 (&z)[2], float2 (&S)[2])
{
    constexpr int NG = horner_ng(NC);
    constexpr int LEN = NC < kHorner ? NC : (G + 1 < NG ? kHorner : NC - kHorner * G);
    if constexpr (G < GE) {
        const float2 ph[2] = {ra[1 + G], rb[1 + G]};
        horner_group2<horner_held(NC, GB, GE), LEN, kHorner * (G - GB), G == GB>(L, z, ph, S);
        horner_groups<NC, GB, GE, G + 1>(L, ra, rb, z, S);
    }
}

// Re(A S) for the row factor A of one point (d == 3 specialised)
template <bool D3>
__device__ __forceinline__ float row_part(const float2 *Ep, int d, const RowOff &ro,
                                          const float2 S)
{
    float2 A;
    if (D3) A = cmul(Ep[ro.o0], Ep[ro.o1]);
    else A = row_factor(Ep, d, ro);
    return A.x * S.x - A.y * S.y;
}

// the rows roff + lane, roff + lane + rstride, ... of the leaf, groups GB .. GE-1
// of each (a thread holds those columns of its row in registers); every point's
// contribution is reduced over the warp's 32 rows and added to the warp's slot
template <int NC, int GB, int GE, bool D3>
__device__ __forceinline__ void horner_rows(const FarArgs<float> &a, const float2 *E, int rowlen,
                                            int rflen, int cnt, float *part, int roff, int rstride)
{
    using C = float2;
    constexpr int NL = horner_held(NC, GB, GE);
    const int d = a.d, nrow = a.nrow;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool hi16 = lane >= 16, hi8 = (lane & 8) != 0;
    const C *Lleaf = a.Lx + (int64_t)blockIdx.x * a.mstride;
    float *wpart = part + warp * a.pch;
    for (int row0 = 0; row0 < nrow; row0 += rstride) {
        if (row0 + roff >= nrow) break;  // the whole warp is past the last row
        const int row = row0 + roff + lane;
        const bool act = row < nrow;
        C L[NL];
        const C *lrow = Lleaf + (int64_t)(act ? row : 0) * a.ncol + kHorner * GB;
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            if (act && kHorner * GB + q < a.ncol) L[q] = lrow[q];
            else L[q].x = L[q].y = 0.f;
        }
        const RowOff ro = row_offsets(act ? row : 0, d, a.n1, a.seg0, a.seg);
        for (int p = 0; p < cnt; p += 4) {
            float v[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int pa = min(p + 2 * h, cnt - 1), pb = min(p + 2 * h + 1, cnt - 1);
                const C *Ea = E + pa * rowlen, *Eb = E + pb * rowlen;
                const C z[2] = {Ea[rflen], Eb[rflen]};
                C S[2];
                horner_groups<NC, GB, GE, GB>(L, Ea + rflen, Eb + rflen, z, S);
                const float va = row_part<D3>(Ea, d, ro, S[0]);
                const float vb = row_part<D3>(Eb, d, ro, S[1]);
                v[2 * h] = act && p + 2 * h < cnt ? va : 0.f;
                v[2 * h + 1] = act && p + 2 * h + 1 < cnt ? vb : 0.f;
            }
            // warp sums of the four points: lanes < 16 keep points 0, 1 and lanes >= 16
            // points 2, 3; (lane & 8) then picks one of the pair; a butterfly over the
            // remaining 8 lanes
            const float k0 = (hi16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, hi16 ? v[0] : v[2], 16);
            const float k1 = (hi16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, hi16 ? v[1] : v[3], 16);
            float w = (hi8 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if ((lane & 7) == 0) {
                const int pk = p + (hi16 ? 2 : 0) + (hi8 ? 1 : 0);
                if (pk < cnt) wpart[pk] += w;
            }
        }
    }
}

template <int NC, bool SPLIT>
__device__ __forceinline__ void l2p_horner_body(const FarArgs<float> &a, int reclen)
{
    using C = float2;
    constexpr int NG = horner_ng(NC);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = a.d, seg0 = a.seg0, seg = a.seg;
    const int rflen = d == 1 ? 0 : seg0 + (d - 2) * seg;  // row-factor tables (dims 0..d-2)
    const int rowlen = rflen + reclen;
    const int nwarp = blockDim.x >> 5;
    C *E = reinterpret_cast<C *>(smem_raw);                                // [pch][rowlen]
    float *part = reinterpret_cast<float *>(E + (size_t)a.pch * rowlen);   // [nwarp][pch]
    const int leaf = blockIdx.x;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = a.leaf_off[leaf + 1] - (int)p0;
    double c[RBF_MAX_DIM];
    leaf_centre(a.leaf_key[leaf], d, a.D, a.lo, a.side, c);
    const int cdim = d - 1;
    const int xoff = d == 1 ? a.M / 2 : 0;  // xi index of column q is q + xoff
    for (int ch0 = 0; ch0 < np; ch0 += a.pch) {
        const int cnt = min(a.pch, np - ch0);
        __syncthreads();
        // per point: the row-factor tables, then z and the first-column phase of
        // every group
        for (int idx = threadIdx.x; idx < cnt * rowlen; idx += blockDim.x) {
            const int p = idx / rowlen, j = idx - p * rowlen;
            int t, kidx;
            bool pad;
            if (j < rflen) {
                if (j < seg0) {
                    t = 0;
                    kidx = j + a.M / 2;
                    pad = j >= a.n0;
                } else {
                    t = 1 + (j - seg0) / seg;
                    kidx = (j - seg0) % seg;
                    pad = kidx >= a.n1;
                }
            } else {
                const int q = j - rflen;
                t = cdim;
                pad = q > NG;
                kidx = q == 0 ? a.M / 2 + 1 : kHorner * (q - 1) + xoff;
            }
            C e;
            if (pad) {
                e.x = e.y = 0.f;
            } else {
                const float r = a.xs[(int64_t)t * a.N + p0 + ch0 + p] - (float)c[t];
                float sn, co;
                sincos_r(a.xi[kidx] * r, &sn, &co);
                e.x = co;
                e.y = sn;
            }
            E[idx] = e;
        }
        for (int q = threadIdx.x; q < nwarp * a.pch; q += blockDim.x) part[q] = 0.f;
        __syncthreads();
        if constexpr (!SPLIT) {
            const int roff = (threadIdx.x >> 5) * 32, rstride = blockDim.x;
            if (d == 3) horner_rows<NC, 0, NG, true>(a, E, rowlen, rflen, cnt, part, roff, rstride);
            else horner_rows<NC, 0, NG, false>(a, E, rowlen, rflen, cnt, part, roff, rstride);
        } else {
            // warp pairs share 32 rows: the even warp takes the first half of the
            // groups, the odd warp the rest (each holds half a row in registers)
            constexpr int GM = NG / 2;
            const int warp = threadIdx.x >> 5;
            const int roff = (warp >> 1) * 32, rstride = (nwarp >> 1) * 32;
            if ((warp & 1) == 0) {
                if (d == 3) horner_rows<NC, 0, GM, true>(a, E, rowlen, rflen, cnt, part, roff, rstride);
                else horner_rows<NC, 0, GM, false>(a, E, rowlen, rflen, cnt, part, roff, rstride);
            } else {
                if (d == 3) horner_rows<NC, GM, NG, true>(a, E, rowlen, rflen, cnt, part, roff, rstride);
                else horner_rows<NC, GM, NG, false>(a, E, rowlen, rflen, cnt, part, roff, rstride);
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
            float sum = 0.f;
            for (int w = 0; w < nwarp; ++w) sum += part[w * a.pch + p];
            a.u[p0 + ch0 + p] = sum;
        }
    }
}

template <int NC>
__global__ void __maxnreg__(96) k_l2p_horner(FarArgs<float> a, int reclen)
{
    l2p_horner_body<NC, false>(a, reclen);
}

#ifndef RBF_L2P_SPLIT_REGS
#define RBF_L2P_SPLIT_REGS 64
#endif
// rows of at least two groups: half a row per thread, so twice the warps fit
template <int NC>
__global__ void __maxnreg__(RBF_L2P_SPLIT_REGS) k_l2p_horner2(FarArgs<float> a, int reclen)
{
    l2p_horner_body<NC, true>(a, reclen);
}

// ------------------------------------------------------------------ M2M ---
// M2M for d <= 3, two consecutive modes per thread: every child value of the
// pair is loaded (one 16-byte load in FP32) before any arithmetic, so the
// 2^d loads of a thread are in flight together.
template <typename R, int DIM>
__global__ void __launch_bounds__(256) k_m2m_pair(int M, int n1, int nmode, int64_t ms,
                                                  const cplx<R> *sh, const int32_t *child_off,
                                                  const uint64_t *child_key, const cplx<R> *Vc,
                                                  cplx<R> *Vp)
{
    using C = cplx<R>;
    constexpr int NC = 1 << DIM;
    const int m = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
    if (m >= nmode) return;
    const bool two = m + 1 < nmode;
    const int p = blockIdx.x;
    const int c0 = child_off[p], nc = child_off[p + 1] - c0;
    C v[NC][2];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j < nc) {
            const C *src = Vc + (int64_t)(c0 + j) * ms + m;
            if (sizeof(R) == 4 && two) {
                const float4 w = *reinterpret_cast<const float4 *>(src);
                v[j][0].x = w.x;
                v[j][0].y = w.y;
                v[j][1].x = w.z;
                v[j][1].y = w.w;
            } else {
                v[j][0] = src[0];
                v[j][1] = two ? src[1] : C{(R)0, (R)0};
            }
        }
    }
    unsigned bits[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) bits[j] = j < nc ? (unsigned)(child_key[c0 + j] & (NC - 1)) : 0u;
    C out[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        // per-dimension half shift e^{-i xi_k wc/2} of mode m + e
        C P[DIM];
        int r = m + e;
#pragma unroll
        for (int t = DIM - 1; t >= 0; --t) {
            int kidx;
            if (t > 0) {
                kidx = r % n1;
                r /= n1;
            } else {
                kidx = r + M / 2;
            }
            P[t] = sh[min(kidx, n1 - 1)];
        }
        C acc{(R)0, (R)0};
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (j < nc) {
                C ph = (bits[j] & 1u) ? P[0] : cconj(P[0]);
#pragma unroll
                for (int t = 1; t < DIM; ++t) ph = cmul(ph, ((bits[j] >> t) & 1u) ? P[t] : cconj(P[t]));
                cmac(acc, ph, v[j][e]);
            }
        }
        out[e] = acc;
    }
    C *dst = Vp + (int64_t)p * ms + m;
    if (sizeof(R) == 4 && two) {
        *reinterpret_cast<float4 *>(dst) = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
    } else {
        dst[0] = out[0];
        if (two) dst[1] = out[1];
    }
}

// Parents at level l from their children at level l+1 (child width wc).
template <typename R>
__global__ void k_m2m(int d, int M, int n1, int nmode, int64_t ms, const cplx<R> *sh,
                      const int32_t *child_off, const uint64_t *child_key, const cplx<R> *Vc,
                      cplx<R> *Vp)
{
    using C = cplx<R>;
    const int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    const int p = blockIdx.x;
    // per-dimension half shift e^{-i xi_k wc/2} (table row of the child level)
    C P[RBF_MAX_DIM];
    int r = m;
    for (int t = d - 1; t >= 0; --t) {
        int kidx;
        if (t > 0) {
            kidx = r % n1;
            r /= n1;
        } else {
            kidx = r + M / 2;
        }
        P[t] = sh[kidx];
    }
    C acc;
    acc.x = acc.y = (R)0;
    const int c0 = child_off[p], c1 = child_off[p + 1];
    for (int cidx = c0; cidx < c1; ++cidx) {
        const unsigned bits = (unsigned)(child_key[cidx] & ((1u << d) - 1u));
        C ph = (bits & 1u) ? P[0] : cconj(P[0]);
        for (int t = 1; t < d; ++t) ph = cmul(ph, ((bits >> t) & 1u) ? P[t] : cconj(P[t]));
        cmac(acc, ph, Vc[(int64_t)cidx * ms + m]);
    }
    Vp[(int64_t)p * ms + m] = acc;
}

// ------------------------------------------------------------------ M2L ---
// Telescoped coupling + downsweep at the leaves (see file header).  The
// neighbours of the leaf are placed on their 3^d offset grid in shared memory
// and the offset phases are summed one dimension at a time.
template <typename R>
__global__ void k_m2l(int d, int M, int D, int n1, int64_t nmode, int64_t ms, const R *xi, const R *omegaC,
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
            C v = VD[(int64_t)bz * ms + m];
            inner.x += v.x;
            inner.y += v.y;
        }
        if (bp >= 0) cmac(inner, Q[tl], VD[(int64_t)bp * ms + m]);
        if (bm >= 0) cmac(inner, cconj(Q[tl]), VD[(int64_t)bm * ms + m]);
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
    Lx[(int64_t)a * ms + m] = out;
}

// Grouped coupling + downsweep for d <= 3: one CTA per level-(D-1) box P and a
// chunk of modes.  The 2^d children of P are the targets; their neighbour
// leaves all lie in the 4^d block of leaves around P (block coordinate
// i_t = k_t - 2 P_t + 1).  For one mode (one thread) the 3^d stencil
//     S_a = sum_{delta in {-1,0,1}^d} prod_t Q_t^{delta_t} V_{a+delta},  Q_t = e^{-i xi_t w_D}
// is summed one dimension at a time over the block, so each neighbour
// expansion is read once per CTA instead of once per target.
template <typename R, int DIM, int MP>
__global__ void RBF_M2L_BOUNDS k_m2l_grp(int M, int D, int n1, int nmode, int64_t ms,
                                                 const cplx<R> *shD,
                                                 const R *omegaC, const cplx<R> *root_ph,
                                                 const uint64_t *parent_key, const int32_t *nb4,
                                                 const cplx<R> *V0, const cplx<R> *VD,
                                                 const cplx<R> *Vzero, cplx<R> *Lx)
{
    // MP consecutive modes per thread (2: one 16-byte load of two FP32 modes)
    using C = cplx<R>;
    constexpr int NB = DIM == 1 ? 4 : (DIM == 2 ? 16 : 64);
    __shared__ const C *base[NB];   // expansion of each block position (absent: zeros)
    __shared__ int32_t nb[NB];
    const int p = blockIdx.x;
    for (int q = threadIdx.x; q < NB; q += blockDim.x) {
        const int32_t b = nb4[(int64_t)p * NB + q];
        nb[q] = b;
        base[q] = b >= 0 ? VD + (int64_t)b * ms : Vzero;
    }
    __syncthreads();
    const int m0 = MP * (blockIdx.y * blockDim.x + threadIdx.x);
    if (m0 >= nmode) return;
    // the second mode of an odd last pair reads the zero padding of the stride
    int kidx[MP][3];
    C Q[MP][3];
#pragma unroll
    for (int e = 0; e < MP; ++e) {
        int r = min(m0 + e, nmode - 1);
        for (int t = 0; t < 3; ++t) kidx[e][t] = 0;
        for (int t = DIM - 1; t >= 1; --t) {
            kidx[e][t] = r % n1;
            r /= n1;
        }
        kidx[e][0] = r + M / 2;
        // Q_t = e^{-i xi_k w_D} = (e^{-i xi_k w_D / 2})^2 from the plan's half-shift table
#pragma unroll
        for (int t = 0; t < DIM; ++t) {
            const C hq = shD[kidx[e][t]];
            Q[e][t] = cmul(hq, hq);
        }
    }
    auto ld = [&](int pos, C (&v)[MP]) {
        const C *bp = base[pos] + m0;
        if constexpr (MP == 2 && sizeof(R) == 4) {
            const float4 w = *reinterpret_cast<const float4 *>(bp);
            v[0] = make_float2(w.x, w.y);
            v[1] = make_float2(w.z, w.w);
        } else {
#pragma unroll
            for (int e = 0; e < MP; ++e) v[e] = bp[e];
        }
    };
    // 3-tap sum for targets at block positions 1 and 2 of a line v[0..3]
    auto tap = [&](const C *v, C q, C *out) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            C s = v[j + 1];
            cmac(s, cconj(q), v[j]);
            cmac(s, q, v[j + 2]);
            out[j] = s;
        }
    };
    C S[MP][8];  // targets, index j0 + 2 j1 + 4 j2 (j_t = 0, 1 <-> block position 1, 2)
    if (DIM == 1) {
        C v[MP][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            C w[MP];
            ld(i, w);
#pragma unroll
            for (int e = 0; e < MP; ++e) v[e][i] = w[e];
        }
#pragma unroll
        for (int e = 0; e < MP; ++e) tap(v[e], Q[e][0], S[e]);
    } else if (DIM == 2) {
#pragma unroll
        for (int e = 0; e < MP; ++e) {
            C s1[4][2];  // [i1][j0]
#pragma unroll
            for (int i1 = 0; i1 < 4; ++i1) {
                C v[4];
#pragma unroll
                for (int i0 = 0; i0 < 4; ++i0) {
                    C w[MP];
                    ld(i0 + 4 * i1, w);
                    v[i0] = w[e];
                }
                tap(v, Q[e][0], s1[i1]);
            }
#pragma unroll
            for (int j0 = 0; j0 < 2; ++j0) {
                C v[4], o[2];
#pragma unroll
                for (int i1 = 0; i1 < 4; ++i1) v[i1] = s1[i1][j0];
                tap(v, Q[e][1], o);
                S[e][j0] = o[0];
                S[e][j0 + 2] = o[1];
            }
        }
    } else {
        C s2[MP][4][2][2];  // [mode][i2][j1][j0]
#pragma unroll
        for (int i2 = 0; i2 < 4; ++i2) {
            C s1[MP][4][2];  // [mode][i1][j0]
#pragma unroll
            for (int i1 = 0; i1 < 4; ++i1) {
                C v[MP][4];
#pragma unroll
                for (int i0 = 0; i0 < 4; ++i0) {
                    C w[MP];
                    ld(i0 + 4 * i1 + 16 * i2, w);
#pragma unroll
                    for (int e = 0; e < MP; ++e) v[e][i0] = w[e];
                }
#pragma unroll
                for (int e = 0; e < MP; ++e) tap(v[e], Q[e][0], s1[e][i1]);
            }
#pragma unroll
            for (int e = 0; e < MP; ++e)
#pragma unroll
                for (int j0 = 0; j0 < 2; ++j0) {
                    C v[4], o[2];
#pragma unroll
                    for (int i1 = 0; i1 < 4; ++i1) v[i1] = s1[e][i1][j0];
                    tap(v, Q[e][1], o);
                    s2[e][i2][0][j0] = o[0];
                    s2[e][i2][1][j0] = o[1];
                }
        }
#pragma unroll
        for (int e = 0; e < MP; ++e)
#pragma unroll
            for (int j1 = 0; j1 < 2; ++j1)
#pragma unroll
                for (int j0 = 0; j0 < 2; ++j0) {
                    C v[4], o[2];
#pragma unroll
                    for (int i2 = 0; i2 < 4; ++i2) v[i2] = s2[e][i2][j1][j0];
                    tap(v, Q[e][2], o);
                    S[e][j0 + 2 * j1] = o[0];
                    S[e][j0 + 2 * j1 + 4] = o[1];
                }
    }
    // targets: L_a = omega C (e^{i xi.(c_a - c_0)} V_0 - S_a)
    int kp[3] = {0, 0, 0};
    {
        const uint64_t key = parent_key[p];
        for (int b = 0; b < D - 1; ++b)
#pragma unroll
            for (int t = 0; t < DIM; ++t) kp[t] |= (int)((key >> (b * DIM + t)) & 1u) << b;
    }
    const int64_t nk = (int64_t)1 << D;
    C rp[MP][3][2];
    C v0[MP];
    R w[MP];
#pragma unroll
    for (int e = 0; e < MP; ++e) {
        const int m = min(m0 + e, nmode - 1);
#pragma unroll
        for (int t = 0; t < DIM; ++t)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                rp[e][t][j] = root_ph[((int64_t)t * nk + 2 * kp[t] + j) * n1 + kidx[e][t]];
        v0[e] = V0[m];
        w[e] = m0 + e < nmode ? omegaC[m] : (R)0;  // the padding mode gets zero
    }
#pragma unroll
    for (int c = 0; c < (1 << DIM); ++c) {
        int pos = 0;
#pragma unroll
        for (int t = 0; t < DIM; ++t) pos += (((c >> t) & 1) + 1) << (2 * t);
        const int a = nb[pos];
        if (a < 0) continue;
        C out[MP];
#pragma unroll
        for (int e = 0; e < MP; ++e) {
            C ph = rp[e][0][c & 1];
#pragma unroll
            for (int t = 1; t < DIM; ++t) ph = cmul(ph, rp[e][t][(c >> t) & 1]);
            const C r = cmul(ph, v0[e]);
            out[e].x = w[e] * (r.x - S[e][c].x);
            out[e].y = w[e] * (r.y - S[e][c].y);
        }
        C *dst = Lx + (int64_t)a * ms + m0;
        if constexpr (MP == 2 && sizeof(R) == 4) {
            *reinterpret_cast<float4 *>(dst) = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
        } else {
#pragma unroll
            for (int e = 0; e < MP; ++e)
                if (m0 + e < nmode) dst[e] = out[e];
        }
    }
}

// Coupling on the whole leaf grid, for small grids (S = 2^D boxes per
// dimension, S^d <= 4096): the neighbour sum of the telescoped coupling,
//   S_a = sum_{b in N_a} e^{i xi.(c_a - c_b)} V_b,
// is a separable three-tap stencil over the grid (absent boxes hold zero),
// applied one dimension at a time to MC consecutive modes held in shared
// memory; then L_a = omega C (e^{i xi.(c_a - c_0)} V_0 - S_a).  Each leaf
// expansion is read once and each local expansion written once.
template <typename R, int S>
__global__ void __launch_bounds__(256) k_m2l_full(int d, int M, int n1, int64_t nmode, int64_t ms,
                                                  int MC, int nleaf, const R *omegaC,
                                                  const cplx<R> *shD, const cplx<R> *root_ph,
                                                  const uint64_t *leaf_key, const cplx<R> *V0,
                                                  const cplx<R> *VD, cplx<R> *Lx)
{
    using C = cplx<R>;
    constexpr int SB = S == 4 ? 2 : (S == 8 ? 3 : 4);   // bits per coordinate
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int nbox = 1;
    for (int t = 0; t < d; ++t) nbox *= S;
    C *grid = reinterpret_cast<C *>(smem_raw);                          // [nbox][MC]
    C *rph = grid + (int64_t)nbox * MC;                                  // [d][S][MC] root phases
    int *kid = reinterpret_cast<int *>(rph + d * S * MC);               // [d][MC] frequency index
    uint32_t *lc = reinterpret_cast<uint32_t *>(kid + d * MC);          // [nleaf] packed coordinates
    const int64_t m0 = (int64_t)blockIdx.x * MC;
    const int mc = (int)min((int64_t)MC, nmode - m0);
    const int D = SB;
    for (int q = threadIdx.x; q < d * MC; q += blockDim.x) {
        const int t = q / MC, mm = q - t * MC;
        int64_t r = m0 + min(mm, mc - 1);
        int k = 0;
        for (int u = d - 1; u >= 0; --u) {
            if (u == 0) {
                k = (int)r + M / 2;
            } else {
                const int dig = (int)(r % n1);
                r /= n1;
                if (u == t) k = dig;
            }
            if (u == t) break;
        }
        kid[q] = k;
    }
    // leaf coordinates k_t (SB bits each, dimension 0 lowest); grid index = the same
    // bits read as one integer
    for (int l = threadIdx.x; l < nleaf; l += blockDim.x) {
        int k[RBF_MAX_DIM];
        decode_key(leaf_key[l], d, D, k);
        uint32_t w = 0;
        for (int t = d - 1; t >= 0; --t) w = (w << SB) | (uint32_t)k[t];
        lc[l] = w;
    }
    for (int q = threadIdx.x; q < nbox * MC; q += blockDim.x) grid[q] = C{(R)0, (R)0};
    __syncthreads();
    // e^{i xi_k (c_t(k) - c_0,t)} per dimension, leaf coordinate and mode of the CTA
    for (int q = threadIdx.x; q < d * S * MC; q += blockDim.x) {
        const int t = q / (S * MC), r = q - t * S * MC, kt = r / MC, mm = r - kt * MC;
        rph[q] = root_ph[((int64_t)t * S + kt) * n1 + kid[t * MC + mm]];
    }
    // leaf expansions -> grid, eight loads in flight per thread
    {
        constexpr int U = 8;
        const int nq = nleaf * MC;
        for (int q0 = threadIdx.x; q0 < nq; q0 += U * blockDim.x) {
            C v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u * blockDim.x;
                const int l = q / MC, mm = q - l * MC;
                v[u] = (q < nq && mm < mc) ? VD[(int64_t)l * ms + m0 + mm] : C{(R)0, (R)0};
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + u * blockDim.x;
                const int l = q / MC, mm = q - l * MC;
                if (q < nq && mm < mc) grid[(int64_t)lc[l] * MC + mm] = v[u];
            }
        }
    }
    __syncthreads();
    int stride = 1;
    for (int t = 0; t < d; ++t) {
        const int nline = nbox / S;
        for (int q = threadIdx.x; q < nline * MC; q += blockDim.x) {
            const int line = q / MC, mm = q - line * MC;
            const int lo = line % stride, hi = line / stride;
            C *base = grid + ((int64_t)lo + (int64_t)hi * stride * S) * MC + mm;
            // e^{-i xi_k w_D}: factor of the neighbour one box up, conj for one box down
            const C h = shD[kid[t * MC + mm]];
            const C qf = cmul(h, h);
            C v[S];
#pragma unroll
            for (int i = 0; i < S; ++i) v[i] = base[(int64_t)i * stride * MC];
#pragma unroll
            for (int i = 0; i < S; ++i) {
                C o = v[i];
                if (i > 0) cmac(o, cconj(qf), v[i - 1]);
                if (i + 1 < S) cmac(o, qf, v[i + 1]);
                base[(int64_t)i * stride * MC] = o;
            }
        }
        stride *= S;
        __syncthreads();
    }
    for (int q = threadIdx.x; q < nleaf * MC; q += blockDim.x) {
        const int l = q / MC, mm = q - l * MC;
        if (mm >= mc) continue;
        const uint32_t w = lc[l];
        const int64_t m = m0 + mm;
        C ph = rph[(int)(w & (S - 1)) * MC + mm];
        for (int t = 1; t < d; ++t) {
            const int kt = (int)((w >> (SB * t)) & (S - 1));
            ph = cmul(ph, rph[(t * S + kt) * MC + mm]);
        }
        const C r = cmul(ph, V0[m]);
        const C sa = grid[(int64_t)w * MC + mm];
        const R wC = omegaC[m];
        C out;
        out.x = wC * (r.x - sa.x);
        out.y = wC * (r.y - sa.y);
        Lx[(int64_t)l * ms + m] = out;
    }
}

// block size: multiple of 32*NH threads, fewest idle row slots
inline int pick_block(int nrow, int rpt, int nh, int bmax)
{
    // a CTA handles one leaf in passes over its mode rows and the resident CTAs per
    // SM are fixed by the launch bounds, so the block with the fewest passes wins;
    // among equal counts the smallest (its extra threads would idle)
    const int step = 32 * nh, first = step * ((64 + step - 1) / step);
    int best = first, best_passes = 1 << 30;
    for (int bd = first; bd <= bmax; bd += step) {
        const int per = (bd / nh) * rpt;
        const int passes = (nrow + per - 1) / per;
        if (passes < best_passes) {
            best = bd;
            best_passes = passes;
        }
    }
    return best;
}

template <typename R, int NCE>
int launch_p2m_l2p(bool l2p, const FarArgs<R> &a0, int nleaf, cudaStream_t s)
{
    constexpr int RPT = sizeof(R) == 4 ? RBF_FAR_RPT : 1;
    constexpr int NH = sizeof(R) == 4 ? (NCE % (2 * RBF_FAR_NH) == 0 ? RBF_FAR_NH : 2) : far_nh64(NCE);
    constexpr int LRPT = sizeof(R) == 4 ? RBF_L2P_RPT : 1;
    constexpr int LNH = sizeof(R) == 4 ? (NCE % (2 * RBF_L2P_NH) == 0 ? RBF_L2P_NH : 2) : far_nh64(NCE);
    static_assert(NCE % (2 * NH) == 0 && NCE % (2 * LNH) == 0, "column groups must be even");
    // the column segment is read NCE entries wide; all segments of dims >= 1
    // share its length, and dim 0 is the column segment when d == 1
    FarArgs<R> a = a0;
    a.seg = NCE;
    a.seg0 = a.d == 1 ? NCE : even_up(a.n0);
    const int rowlen = a.seg0 + (a.d - 1) * a.seg;
    // dense shape for leaves of up to 96 points on average and column segments of
    // at most 36 (wider ones spill under its register bound); L2P's short chunks
    // only for leaves of up to 32 points
    bool dense = sizeof(R) == 4 && a.N <= 96 * (int64_t)nleaf && NCE <= RBF_L2P_NARROW;
    // P2M: the shape measured at plan creation, when there was a choice
    if (!l2p && a.shape != 0) dense = sizeof(R) == 4 && NCE <= RBF_L2P_NARROW && a.shape == 1;
    const bool small = a.N <= 32 * (int64_t)nleaf;
    const int want = l2p ? (dense && small ? RBF_L2P_PCH_DENSE : RBF_L2P_PCH_WIDE)
                         : (dense ? RBF_P2M_PCH_DENSE : RBF_P2M_PCH_WIDE);
    a.pch = (int)std::max<int64_t>(1, std::min<int64_t>(l2p && !RBF_L2P_SMEMRED ? 64 : want,
                                                        (64 * 1024) / ((int64_t)rowlen * sizeof(cplx<R>))));
    const int bmax = sizeof(R) == 4 ? far_bmax(dense, NCE) : 256;
    const int bd = l2p ? pick_block(a.nrow, LRPT, LNH, bmax) : pick_block(a.nrow, RPT, NH, bmax);
    size_t smem = (size_t)a.pch * rowlen * sizeof(cplx<R>);
    if (l2p) smem += (size_t)(RBF_L2P_SMEMRED ? bd : bd / 32) * a.pch * sizeof(R);
    auto go = [&](auto shape) -> int {
        constexpr bool D = decltype(shape)::value;
        if (l2p) {
            RBF_CUDA_TRY(cudaFuncSetAttribute(k_l2p<R, NCE, LRPT, LNH, D>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_l2p<R, NCE, LRPT, LNH, D><<<nleaf, bd, smem, s>>>(a);
        } else {
            RBF_CUDA_TRY(cudaFuncSetAttribute(k_p2m<R, NCE, RPT, NH, D>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_p2m<R, NCE, RPT, NH, D><<<nleaf, bd, smem, s>>>(a);
        }
        return RBF_OK;
    };
    if constexpr (sizeof(R) == 4 && NCE <= RBF_L2P_NARROW) {
        RBF_TRY(dense ? go(std::true_type()) : go(std::false_type()));
    } else {
        RBF_TRY(go(std::false_type()));
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

template <typename R>
int dispatch_p2m_l2p(bool l2p, const FarArgs<R> &a, int nleaf, cudaStream_t s)
{
    const int nc = a.ncol;
    // FP32 splits the columns in two even halves: widths are multiples of 4
    if (nc <= 12) return launch_p2m_l2p<R, 12>(l2p, a, nleaf, s);
    if (nc <= 20) return launch_p2m_l2p<R, 20>(l2p, a, nleaf, s);
    if (nc <= 28) return launch_p2m_l2p<R, 28>(l2p, a, nleaf, s);
    if (nc <= 36) return launch_p2m_l2p<R, 36>(l2p, a, nleaf, s);
    if (nc <= 44) return launch_p2m_l2p<R, 44>(l2p, a, nleaf, s);
    if (nc <= 52) return launch_p2m_l2p<R, 52>(l2p, a, nleaf, s);
    return launch_p2m_l2p<R, 68>(l2p, a, nleaf, s);
}

}  // namespace

// M2M from the leaf expansions VD up to the root (levels D-1 .. 0 of the plan)
template <typename R>
int rbf_run_m2m(rbf_tree *t, const rbf_plan *p, const cplx<R> *VD, cudaStream_t s)
{
    using C = cplx<R>;
    const int d = t->d, D = t->D;
    const int mb = 256;
    const int mchunks = ceil_div(p->nmode, mb);
    RBF_REQUIRE(mchunks < 65536, "expansion too large (%lld modes)", (long long)p->nmode);
    rbf_pass_timer tm(t, RBF_PASS_M2M, s, D);
    const int pchunks = ceil_div(p->nmode, 2 * mb);
    for (int l = D - 1; l >= 0; --l) {
        const C *child = l + 1 == D ? VD : (const C *)p->V[l + 1];
        const C *sh = (const C *)p->shift_ph + (int64_t)(l + 1) * p->n1;
        if (d <= 3) {
            dim3 grid(t->lev[l].nbox, pchunks);
#define RBF_M2M_PAIR(DD)                                                                          \
    k_m2m_pair<R, DD><<<grid, mb, 0, s>>>(p->M, p->n1, (int)p->nmode, p->mstride, sh,              \
                                          t->lev[l].child_off, t->lev[l + 1].key, child,           \
                                          (C *)p->V[l])
            if (d == 1) RBF_M2M_PAIR(1);
            else if (d == 2) RBF_M2M_PAIR(2);
            else RBF_M2M_PAIR(3);
#undef RBF_M2M_PAIR
        } else {
            dim3 grid(t->lev[l].nbox, mchunks);
            k_m2m<R><<<grid, mb, 0, s>>>(d, p->M, p->n1, (int)p->nmode, p->mstride, sh,
                                         t->lev[l].child_off, t->lev[l + 1].key, child,
                                         (C *)p->V[l]);
        }
        RBF_LAUNCH_CHECK();
    }
    return RBF_OK;
}

namespace {

// 3-D coupling by pencils: one CTA per pencil of 2 x 2 x RBF_PENCIL_Z leaves and
// chunk of 128 modes, one mode per thread.  The thread walks the planes z0 - 1 ..
// z0 + Z of the pencil's 4 x 4 (x, y) neighbourhood: each plane's 16 values are
// filtered along x (three taps) and y into the 2 x 2 plane of the pencil, a window
// of three filtered planes gives the z taps of the plane in the middle, and its four
// targets L_a = omega C (e^{i xi.(c_a - c_0)} V_0 - S_a) are written.  Every
// neighbour value is read 16 (Z + 2) / (4 Z) = 5 times per target plane instead of 8
// times by the parent-block kernel, and a target costs 8 complex MACs instead of 14.
template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? RBF_M2L_PENCIL_MINB : 3) k_m2l_pencil(int M, int D, int n1, int nmode, int64_t ms,
                                            const cplx<R> *shD, const R *omegaC,
                                            const cplx<R> *root_ph, const int4 *seg,
                                            const int32_t *pnb, const cplx<R> *V0,
                                            const cplx<R> *VD, const cplx<R> *Vzero, cplx<R> *Lx)
{
    using C = cplx<R>;
    constexpr int Z = RBF_PENCIL_Z, NP = (Z + 2) * 16;
    __shared__ const C *base[NP];   // expansion of each neighbourhood entry (absent: zeros)
    __shared__ int32_t nb[NP];
    const int sgi = blockIdx.x;
    for (int q = threadIdx.x; q < NP; q += blockDim.x) {
        const int32_t b = pnb[(int64_t)sgi * NP + q];
        nb[q] = b;
        base[q] = b >= 0 ? VD + (int64_t)b * ms : Vzero;
    }
    __syncthreads();
    const int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    int kidx[3];
    {
        int r = m;
        kidx[2] = r % n1;
        r /= n1;
        kidx[1] = r % n1;
        r /= n1;
        kidx[0] = r + M / 2;
    }
    // Q_t = e^{-i xi_k w_D} = (e^{-i xi_k w_D / 2})^2 from the plan's half-shift table
    C Q[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const C hq = shD[kidx[t]];
        Q[t] = cmul(hq, hq);
    }
    const int4 sg = seg[sgi];
    const int64_t nk = (int64_t)1 << D;
    const int x0 = 2 * sg.x, y0 = 2 * sg.y, z0 = sg.z * Z;
    // e^{i xi.(c_a - c_0)} V_0 for the pencil's four (x, y) columns; z per plane
    C RV[4];
    {
        const C v0 = V0[m];
        C px[2], py[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            px[j] = root_ph[((int64_t)0 * nk + x0 + j) * n1 + kidx[0]];
            py[j] = root_ph[((int64_t)1 * nk + y0 + j) * n1 + kidx[1]];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) RV[c] = cmul(cmul(px[c & 1], py[c >> 1]), v0);
    }
    const R w = omegaC[m];
    // 3-tap sum for targets at block positions 1 and 2 of a line v[0..3]
    auto tap = [&](const C *v, C q, C *out) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            C s = v[j + 1];
            cmac(s, cconj(q), v[j]);
            cmac(s, q, v[j + 2]);
            out[j] = s;
        }
    };
    C W0[4], W1[4], W2[4];
#pragma unroll
    for (int zz = 0; zz < Z + 2; ++zz) {
        C s1[4][2];  // [y line][x target]
#pragma unroll
        for (int i1 = 0; i1 < 4; ++i1) {
            C v[4];
#pragma unroll
            for (int i0 = 0; i0 < 4; ++i0) v[i0] = base[zz * 16 + i1 * 4 + i0][m];
            tap(v, Q[0], s1[i1]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            W0[c] = W1[c];
            W1[c] = W2[c];
        }
#pragma unroll
        for (int j0 = 0; j0 < 2; ++j0) {
            C v[4], o[2];
#pragma unroll
            for (int i1 = 0; i1 < 4; ++i1) v[i1] = s1[i1][j0];
            tap(v, Q[1], o);
            W2[j0] = o[0];
            W2[j0 + 2] = o[1];
        }
        if (zz >= 2) {
            const int pl = zz - 1;  // plane of the targets, 1 .. Z
            const C rz = root_ph[((int64_t)2 * nk + z0 + pl - 1) * n1 + kidx[2]];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int a = nb[pl * 16 + ((c >> 1) + 1) * 4 + (c & 1) + 1];
                if (a < 0) continue;
                C S = W1[c];
                cmac(S, cconj(Q[2]), W0[c]);
                cmac(S, Q[2], W2[c]);
                const C r = cmul(RV[c], rz);
                C out;
                out.x = w * (r.x - S.x);
                out.y = w * (r.y - S.y);
                Lx[(int64_t)a * ms + m] = out;
            }
        }
    }
}

}  // namespace

// coupling of all levels plus the downsweep: leaf local expansions L from the
// leaf expansions VD and the root expansion V[0] (left by rbf_run_m2m)
template <typename R>
int rbf_run_m2l(rbf_tree *t, const rbf_plan *p, const cplx<R> *VD, cplx<R> *L, cudaStream_t s)
{
    using C = cplx<R>;
    const int d = t->d, D = t->D;
    rbf_pass_timer tm(t, RBF_PASS_M2L, s);
    const C *V0 = (const C *)p->V[0];
    if (RBF_M2L_PENCIL && d == 3 && t->npz > 0) {
        k_m2l_pencil<R><<<dim3(t->npz, ceil_div(p->nmode, 128)), 128, 0, s>>>(
            p->M, D, p->n1, (int)p->nmode, p->mstride, (const C *)p->shift_ph + (int64_t)D * p->n1,
            (const R *)p->omegaC, (const C *)p->root_ph, t->pz_seg, t->pz_nb, V0, VD,
            (const C *)p->Vzero, L);
        RBF_LAUNCH_CHECK();
    } else if (d <= 3) {
        const int gb = 128;
#define RBF_M2L_GRP(DD, MP)                                                                        \
    k_m2l_grp<R, DD, MP><<<dim3(t->lev[D - 1].nbox, ceil_div(p->nmode, gb * MP)), gb, 0, s>>>(      \
        p->M, D, p->n1, (int)p->nmode, p->mstride, (const C *)p->shift_ph + (int64_t)D * p->n1,     \
        (const R *)p->omegaC, (const C *)p->root_ph, t->lev[D - 1].key, t->nb4, V0, VD,             \
        (const C *)p->Vzero, L)
        // FP32 in 3-D: RBF_M2L_MP modes per thread
        if (d == 1) {
            RBF_M2L_GRP(1, 1);
        } else if (d == 2) {
            RBF_M2L_GRP(2, 1);
        } else {
            if constexpr (sizeof(R) == 4) RBF_M2L_GRP(3, RBF_M2L_MP);
            else RBF_M2L_GRP(3, 1);
        }
#undef RBF_M2L_GRP
        RBF_LAUNCH_CHECK();
    } else if (D >= 2 && D <= 4 && d * D <= 12) {
        // whole leaf grid of S^d <= 4096 boxes: MC modes per CTA within 96 KB
        const int S = 1 << D;
        const int64_t nbox = (int64_t)1 << (d * D);
        const int MC = (int)std::max<int64_t>(1, std::min<int64_t>(16, (96 * 1024) / (nbox * (int64_t)sizeof(C))));
        const size_t smem = (size_t)nbox * MC * sizeof(C) + (size_t)d * S * MC * sizeof(C) +
                            (size_t)d * MC * sizeof(int) + (size_t)t->nleaf() * sizeof(uint32_t);
        const int nblk = ceil_div(p->nmode, MC);
#define RBF_M2L_FULL(SS)                                                                          \
    do {                                                                                          \
        RBF_CUDA_TRY(cudaFuncSetAttribute(k_m2l_full<R, SS>,                                      \
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_m2l_full<R, SS><<<nblk, 256, smem, s>>>(d, p->M, p->n1, p->nmode, p->mstride, MC,       \
                                                  t->nleaf(), (const R *)p->omegaC,              \
                                                  (const C *)p->shift_ph + (int64_t)D * p->n1,    \
                                                  (const C *)p->root_ph, t->leaf_key(), V0, VD, L); \
    } while (0)
        if (S == 4) RBF_M2L_FULL(4);
        else if (S == 8) RBF_M2L_FULL(8);
        else RBF_M2L_FULL(16);
#undef RBF_M2L_FULL
        RBF_LAUNCH_CHECK();
    } else {
        const int mb = 256;
        const double wD = t->side / (double)(1 << D);
        dim3 grid(t->nleaf(), ceil_div(p->nmode, mb));
        RBF_REQUIRE(grid.y < 65536, "expansion too large (%lld modes)", (long long)p->nmode);
        k_m2l<R><<<grid, mb, 0, s>>>(d, p->M, D, p->n1, p->nmode, p->mstride, (const R *)p->xi,
                                     (const R *)p->omegaC, wD, (const C *)p->root_ph, t->leaf_key(),
                                     t->near_off, t->near_idx, V0, VD, L);
        RBF_LAUNCH_CHECK();
    }
    return RBF_OK;
}

namespace {
template <typename R>
FarArgs<R> far_args(const rbf_tree *t, const rbf_plan *p)
{
    FarArgs<R> a;
    a.d = t->d;
    a.M = p->M;
    a.D = t->D;
    a.n0 = p->n0;
    a.n1 = p->n1;
    a.nrow = p->nrow;
    a.ncol = p->ncol;
    a.nmode = p->nmode;
    a.mstride = p->mstride;
    a.N = t->N;
    for (int q = 0; q < RBF_MAX_DIM; ++q) a.lo[q] = t->lo[q];
    a.side = t->side;
    a.xs = (const R *)(sizeof(R) == 8 ? (const void *)t->xs64 : (const void *)t->xs32);
    a.lam = nullptr;
    a.leaf_off = t->leaf_off;
    a.leaf_key = t->leaf_key();
    a.xi = (const R *)p->xi;
    a.V = nullptr;
    a.Lx = nullptr;
    a.u = nullptr;
    a.pch = 0;   // set per launch: as many points as fit in ~64 KB of tables, at most 64
    a.shape = p->p2m_shape;
    a.seg0 = a.seg = 0;
    return a;
}
}  // namespace

// P2M of one column into the leaf expansions V (nleaf x mstride)
template <typename R>
int rbf_run_p2m(rbf_tree *t, const rbf_plan *p, const R *lam_s, cplx<R> *V, cudaStream_t s)
{
    FarArgs<R> a = far_args<R>(t, p);
    a.lam = lam_s;
    a.V = V;
    rbf_pass_timer tm(t, RBF_PASS_P2M, s);
    return dispatch_p2m_l2p<R>(false, a, t->nleaf(), s);
}

// P2M launch shape of an FP32 plan, by measurement: both shapes (dense: five
// CTAs of up to 192 threads; wide: four of up to 256) run P2M twice on the plan's
// tree, the second run of each timed with CUDA events; the faster one is kept in
// the plan.  Both shapes accumulate every output over the points in the same
// order, so the choice changes no bit of the result.  Only where both shapes are
// built (column segments of at most 36) and the tree is large enough to time.
int rbf_tune_p2m_shape(rbf_tree *t, rbf_plan *p, cudaStream_t s)
{
    p->p2m_shape = 0;
    if (p->prec != RBF_FP32 || p->M == 0 || t->D < 2 || t->d < 2 || t->N < 16384 ||
        even_up(p->ncol) > RBF_L2P_NARROW || p->grid != RBF_GRID_SHARED)
        return RBF_OK;
    float *lam = nullptr;
    RBF_TRY(rbf_alloc(&lam, (size_t)t->N));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = RBF_OK;
    if (cudaMemsetAsync(lam, 0, (size_t)t->N * sizeof(float), s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        st = RBF_ECUDA;
    float best = INFINITY;
    int pick = 0;
    for (int shape = 1; shape <= 2 && st == RBF_OK; ++shape) {
        FarArgs<float> a = far_args<float>(t, p);
        a.lam = lam;
        a.V = (float2 *)p->V[t->D];
        a.shape = shape;
        float ms = 0.f;
        st = dispatch_p2m_l2p<float>(false, a, t->nleaf(), s);
        if (st == RBF_OK && cudaEventRecord(e0, s) != cudaSuccess) st = RBF_ECUDA;
        if (st == RBF_OK) st = dispatch_p2m_l2p<float>(false, a, t->nleaf(), s);
        if (st == RBF_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = RBF_ECUDA;
        if (st == RBF_OK && ms < best) {
            best = ms;
            pick = shape;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    rbf_free(lam);
    if (st == RBF_OK) p->p2m_shape = pick;
    return st;
}

namespace {
template <int NC>
int launch_l2p_horner(const FarArgs<float> &a0, int nleaf, cudaStream_t s)
{
    constexpr int NG = horner_ng(NC);
    constexpr bool split = RBF_L2P_SPLIT && NG >= 2;
    FarArgs<float> a = a0;
    a.seg0 = a.d == 1 ? 0 : even_up(a.n0);
    a.seg = even_up(a.n1);
    const int reclen = even_up(NG + 1);
    const int rflen = a.d == 1 ? 0 : a.seg0 + (a.d - 2) * a.seg;
    const int rowlen = rflen + reclen;
    // split: an even number of warps, 32 rows per warp pair
    const int bd = split ? std::min(kHornerBlock2, 64 * ((a.nrow + 31) / 32))
                         : std::min(kHornerBlock, 32 * ((a.nrow + 31) / 32));
    a.pch = kHornerPch;
    const size_t smem = (size_t)a.pch * (rowlen * sizeof(float2) + (bd / 32) * sizeof(float));
    if constexpr (split) {
        RBF_CUDA_TRY(cudaFuncSetAttribute(k_l2p_horner2<NC>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_l2p_horner2<NC><<<nleaf, bd, smem, s>>>(a, reclen);
    } else {
        RBF_CUDA_TRY(cudaFuncSetAttribute(k_l2p_horner<NC>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_l2p_horner<NC><<<nleaf, bd, smem, s>>>(a, reclen);
    }
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

// rows of up to 33 columns: NC = the column count rounded up to odd (at least 3);
// an even count (one dimension, M = 2 mod 4) runs with one zero column more
int l2p_horner(const FarArgs<float> &a, int nleaf, cudaStream_t s)
{
    switch (a.ncol / 2) {
        case 0:
        case 1: return launch_l2p_horner<3>(a, nleaf, s);
        case 2: return launch_l2p_horner<5>(a, nleaf, s);
        case 3: return launch_l2p_horner<7>(a, nleaf, s);
        case 4: return launch_l2p_horner<9>(a, nleaf, s);
        case 5: return launch_l2p_horner<11>(a, nleaf, s);
        case 6: return launch_l2p_horner<13>(a, nleaf, s);
        case 7: return launch_l2p_horner<15>(a, nleaf, s);
        case 8: return launch_l2p_horner<17>(a, nleaf, s);
        case 9: return launch_l2p_horner<19>(a, nleaf, s);
        case 10: return launch_l2p_horner<21>(a, nleaf, s);
        case 11: return launch_l2p_horner<23>(a, nleaf, s);
        case 12: return launch_l2p_horner<25>(a, nleaf, s);
        case 13: return launch_l2p_horner<27>(a, nleaf, s);
        case 14: return launch_l2p_horner<29>(a, nleaf, s);
        case 15: return launch_l2p_horner<31>(a, nleaf, s);
        default: return launch_l2p_horner<33>(a, nleaf, s);
    }
}
}  // namespace

// L2P of one column from the leaf local expansions L: FP32 rows of up to
// kHornerMaxCol columns by the Horner kernel; wider rows and FP64 by the table
// kernel.
template <typename R>
int rbf_run_l2p(rbf_tree *t, const rbf_plan *p, const cplx<R> *L, R *u_far, cudaStream_t s)
{
    FarArgs<R> a = far_args<R>(t, p);
    a.Lx = L;
    a.u = u_far;
    rbf_pass_timer tm(t, RBF_PASS_L2P, s);
    if constexpr (sizeof(R) == 4) {
        if (a.ncol <= kHornerMaxCol) return l2p_horner(a, t->nleaf(), s);
    }
    return dispatch_p2m_l2p<R>(true, a, t->nleaf(), s);
}

template <typename R>
int rbf_run_far(rbf_tree *t, const rbf_plan *p, const R *lam_s, R *u_far, cudaStream_t s)
{
    using C = cplx<R>;
    if (p->grid == RBF_GRID_NESTED) return rbf_run_far_nested<R>(t, p, lam_s, u_far, s);
    const int D = t->D;
    RBF_TRY(rbf_run_p2m<R>(t, p, lam_s, (C *)p->V[D], s));
    RBF_TRY(rbf_run_m2m<R>(t, p, (const C *)p->V[D], s));
    RBF_TRY(rbf_run_m2l<R>(t, p, (const C *)p->V[D], (C *)p->Lleaf, s));
    RBF_TRY(rbf_run_l2p<R>(t, p, (const C *)p->Lleaf, u_far, s));
    return RBF_OK;
}

template int rbf_run_far<float>(rbf_tree *, const rbf_plan *, const float *, float *, cudaStream_t);
template int rbf_run_m2m<float>(rbf_tree *, const rbf_plan *, const float2 *, cudaStream_t);
template int rbf_run_p2m<float>(rbf_tree *, const rbf_plan *, const float *, float2 *, cudaStream_t);
template int rbf_run_l2p<float>(rbf_tree *, const rbf_plan *, const float2 *, float *, cudaStream_t);
template int rbf_run_m2l<float>(rbf_tree *, const rbf_plan *, const float2 *, float2 *, cudaStream_t);
template int rbf_run_far<double>(rbf_tree *, const rbf_plan *, const double *, double *,
                                 cudaStream_t);
template int rbf_run_p2m<double>(rbf_tree *, const rbf_plan *, const double *, double2 *,
                                 cudaStream_t);
template int rbf_run_l2p<double>(rbf_tree *, const rbf_plan *, const double2 *, double *,
                                 cudaStream_t);
