// far_mrhs.cu -- far field of several right-hand sides, with P2M and L2P on the
// fifth-generation tensor cores (tcgen05.mma, TF32 operands in shared memory,
// FP32 accumulators in tensor memory).
//
// For G right-hand sides lambda_{.,r} the leaf aggregation of Eq. (P2M) is a
// complex matrix product over the points j of a leaf,
//     V_r[row][col] = sum_j A_j[row] W_j[col, r],
//     A_j[row]      = prod_{t<d-1} e^{-i xi_{k_t} (x_{j,t} - c_t)},
//     W_j[col, r]   = e^{-i xi_{k_{d-1}} (x_{j,d-1} - c_{d-1})} lambda_{j,r},
// and the evaluation of Eq. (46) is one as well, followed by a short reduction:
//     T_i[col, r]   = sum_row A'_i[row] L_r[row][col],
//     u_{i,r}       = Re sum_col B'_i[col] T_i[col, r],
// with A', B' the phases of the opposite sign (e^{+i xi (x_i - c)}).
//
// Each complex product runs as ONE real product whose K dimension stacks six
// slots per point (P2M) or per mode row (L2P).  With x = hi + lo, hi = tf32(x),
// lo = tf32(x - hi), the six slots hold
//     A:  re_hi  im_hi  re_hi  im_hi  re_lo  im_lo
//     Wr: wr_hi -wi_hi  wr_lo -wi_lo  wr_hi -wi_hi      (output column: real part)
//     Wi: wi_hi  wr_hi  wi_lo  wr_lo  wi_hi  wr_hi      (output column: imaginary part)
// so that a column of real parts accumulates A_re W_re - A_im W_im and a
// column of imaginary parts A_re W_im + A_im W_re, every real product taken as
// hi*hi + hi*lo + lo*hi (three-term split TF32, FP32-level accuracy).
//
// Tile: 128 rows (TMEM lanes) x 2*NT real columns (NT complex: 16, 32, 48 or
// 64), K staged 8 points (rows) = 48 TF32 values at a time in two
// shared-memory stages; one thread issues the six MMAs of a stage and commits
// them to the stage's mbarrier, all 256 threads generate the next stage
// meanwhile.  Accumulation runs in blocks of two stages per TMEM buffer, each
// block folded into FP32 registers (see tc_pipeline).  Operands are K-major
// without swizzle: 8-row x 16-byte core matrices, 128 B apart along K and
// 1536 B apart along rows.  P2M keeps the leaf's points and coefficients in
// shared memory; L2P streams the rows of the local expansions through a ring
// of shared-memory slots filled by bulk asynchronous copies (TMA).
//
// Every wait on an mbarrier is bounded; a wait that gives up sets a status bit
// (read by rbf_tc_fetch_status), the kernel skips its remaining work, waits
// once more (bounded) for its MMAs in flight, frees its tensor memory and
// returns.
#include <algorithm>

#include "rbf_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;           // tile rows = TMEM lanes
constexpr int kKS = 8;               // points (P2M) or mode rows (L2P) per stage
constexpr int kSlots = 6;
constexpr int kKStage = kSlots * kKS;          // 48 TF32 values of K per stage
constexpr int kCoreK = kKStage / 4;            // 12 core matrices along K
constexpr uint32_t kLBO = 128;                 // next core matrix along K
constexpr uint32_t kSBO = kCoreK * 128;        // next group of 8 rows
constexpr int kABytes = kRows * kKStage * 4;   // 24576
constexpr long long kWaitCycles = 4000000000LL;
constexpr int kMaxNT = 64;                     // complex columns of a tile

__device__ unsigned int g_tc_status;

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_bits(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo, both TF32
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = __uint_as_float(tf32_bits(x));
    lo = __uint_as_float(tf32_bits(x - hi));
}

// shared-memory matrix descriptor: K-major, no swizzle, version 1 (tcgen05)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M x N
inline uint32_t instr_desc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the completion of phase `parity`; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(&g_tc_status, 1u);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// 8 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}
__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// byte offset of the 16-byte group (row r, slot s, quad q) inside an operand tile
__device__ __forceinline__ uint32_t op_off(int r, int s, int q)
{
    return (uint32_t)((((r >> 3) * kCoreK + 2 * s + q) << 7) + ((r & 7) << 4));
}

// stores the six slots of a row of the A-side operand (4 consecutive K values)
__device__ __forceinline__ void put_a(unsigned char *tile, int r, int q, const float *re,
                                      const float *im)
{
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        split_tf32(re[e], rh[e], rl[e]);
        split_tf32(im[e], ih[e], il[e]);
    }
    const float4 RH = make_float4(rh[0], rh[1], rh[2], rh[3]);
    const float4 IH = make_float4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<float4 *>(tile + op_off(r, 0, q)) = RH;
    *reinterpret_cast<float4 *>(tile + op_off(r, 1, q)) = IH;
    *reinterpret_cast<float4 *>(tile + op_off(r, 2, q)) = RH;
    *reinterpret_cast<float4 *>(tile + op_off(r, 3, q)) = IH;
    *reinterpret_cast<float4 *>(tile + op_off(r, 4, q)) = make_float4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<float4 *>(tile + op_off(r, 5, q)) = make_float4(il[0], il[1], il[2], il[3]);
}

// stores the real-part row j and the imaginary-part row NT + j of the W-side operand
__device__ __forceinline__ void put_w(unsigned char *tile, int j, int NT, int q, const float *wr,
                                      const float *wi)
{
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        split_tf32(wr[e], rh[e], rl[e]);
        split_tf32(wi[e], ih[e], il[e]);
    }
    const float4 RH = make_float4(rh[0], rh[1], rh[2], rh[3]);
    const float4 RL = make_float4(rl[0], rl[1], rl[2], rl[3]);
    const float4 IH = make_float4(ih[0], ih[1], ih[2], ih[3]);
    const float4 IL = make_float4(il[0], il[1], il[2], il[3]);
    const float4 NIH = make_float4(-ih[0], -ih[1], -ih[2], -ih[3]);
    const float4 NIL = make_float4(-il[0], -il[1], -il[2], -il[3]);
    *reinterpret_cast<float4 *>(tile + op_off(j, 0, q)) = RH;
    *reinterpret_cast<float4 *>(tile + op_off(j, 1, q)) = NIH;
    *reinterpret_cast<float4 *>(tile + op_off(j, 2, q)) = RL;
    *reinterpret_cast<float4 *>(tile + op_off(j, 3, q)) = NIL;
    *reinterpret_cast<float4 *>(tile + op_off(j, 4, q)) = RH;
    *reinterpret_cast<float4 *>(tile + op_off(j, 5, q)) = NIH;
    const int n = NT + j;
    *reinterpret_cast<float4 *>(tile + op_off(n, 0, q)) = IH;
    *reinterpret_cast<float4 *>(tile + op_off(n, 1, q)) = RH;
    *reinterpret_cast<float4 *>(tile + op_off(n, 2, q)) = IL;
    *reinterpret_cast<float4 *>(tile + op_off(n, 3, q)) = RL;
    *reinterpret_cast<float4 *>(tile + op_off(n, 4, q)) = IH;
    *reinterpret_cast<float4 *>(tile + op_off(n, 5, q)) = RH;
}

__device__ __forceinline__ void decode_key(uint64_t key, int d, int l, int *k)
{
    for (int t = 0; t < d; ++t) k[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) k[t] |= (int)((key >> (b * d + t)) & 1u) << b;
}

// Table offsets of the row factors of mode row `row`: o[0] = k0 (dimension-0
// segment), o[t] = n0 + (t-1) n1 + k_t for t = 1 .. d-2.
struct RowFac {
    int o[RBF_MAX_DIM - 1];
};
__device__ __forceinline__ RowFac row_factors(int row, int d, int n0, int n1)
{
    RowFac f;
#pragma unroll
    for (int t = 0; t < RBF_MAX_DIM - 1; ++t) f.o[t] = 0;
#pragma unroll
    for (int t = RBF_MAX_DIM - 2; t >= 1; --t) {
        if (t <= d - 2) {
            f.o[t] = n0 + (t - 1) * n1 + row % n1;
            row /= n1;
        }
    }
    f.o[0] = row;
    return f;
}

// prod_{t<d-1} E[o_t]  (1 when d == 1)
__device__ __forceinline__ float2 row_phase(const float2 *E, const RowFac &f, int d)
{
    if (d == 1) return make_float2(1.0f, 0.0f);
    float2 a = E[f.o[0]];
#pragma unroll
    for (int t = 1; t < RBF_MAX_DIM - 1; ++t)
        if (t < d - 1) a = cmul(a, E[f.o[t]]);
    return a;
}

// next mode row: the fastest digit k_{d-2} first, carries towards k0
__device__ __forceinline__ void row_next(RowFac &f, int d, int n0, int n1)
{
#pragma unroll
    for (int t = RBF_MAX_DIM - 2; t >= 1; --t) {
        if (t <= d - 2) {
            const int base = n0 + (t - 1) * n1;
            if (++f.o[t] < base + n1) return;
            f.o[t] = base;
        }
    }
    ++f.o[0];
}

struct TcArgs {
    int d, M, D, n0, n1, nrow, ncol, G;
    int NT;                  // complex columns of the tile (16, 32, 48 or 64)
    int rowlen, rowpad;      // per-point table length, padded row stride (odd)
    int lcap;                // points of the largest leaf (P2M staging)
    uint32_t idesc, tcols;   // instruction descriptor, allocated TMEM columns
    int64_t mstride, N, vstride;
    double lo[RBF_MAX_DIM];
    double side;
    const float *xs;         // SoA [d][N]
    const float *lam;        // [G][N] sorted order (P2M)
    const int32_t *leaf_off;
    const uint64_t *leaf_key;
    const float *xi;         // [n1]
    float2 *V;               // P2M out: V_r = V + r * vstride, [leaf][mstride]
    const float2 *L;         // L2P in:  L_r = L + r * vstride
    float *u;                // L2P out: [G][N]
};

// e^{sign i xi_k (x - c_t)} of table entry j (dimension 0 keeps k0 = 0..M/2,
// dimensions >= 1 keep k = -M/2..M/2) for the point with coordinates x[t * xstride]
__device__ __forceinline__ float2 table_entry(const TcArgs &a, const float *x, int64_t xstride,
                                              int j, const double *c, float sign)
{
    int t, kidx;
    if (j < a.n0) {
        t = 0;
        kidx = j + a.M / 2;
    } else {
        t = 1 + (j - a.n0) / a.n1;
        kidx = (j - a.n0) % a.n1;
    }
    const float r = x[t * xstride] - (float)c[t];
    float sn, cs;
    sincosf(sign * a.xi[kidx] * r, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ void leaf_centre(const TcArgs &a, int leaf, double *c)
{
    int k[RBF_MAX_DIM];
    decode_key(a.leaf_key[leaf], a.d, a.D, k);
    const double w = a.side / (double)(1 << a.D);
    for (int t = 0; t < a.d; ++t) c[t] = a.lo[t] + ((double)k[t] + 0.5) * w;
}

// the two operand stages at the start of dynamic shared memory
struct StageLayout {
    unsigned char *stage[2];
    uint32_t wbytes;
};
__device__ __forceinline__ StageLayout stages(unsigned char *smem, int NT)
{
    StageLayout s;
    s.wbytes = (uint32_t)(2 * NT) * kKStage * 4;
    s.stage[0] = smem;
    s.stage[1] = smem + kABytes + s.wbytes;
    return s;
}

// Accumulation blocks: the MMAs of kBlock consecutive stages accumulate into
// one of two TMEM buffers (columns [buf * 2NT, buf * 2NT + 2NT)), starting from
// zero; a finished block is added into FP32 registers with round-to-nearest
// adds.  The tensor core's own accumulation rounds towards zero, so a long
// chain of MMAs into one accumulator shrinks it by about one ulp per MMA; short
// blocks keep that below 1e-6 relative.
constexpr int kBlock = 2;
__host__ __device__ __forceinline__ bool block_end(int ch, int nch)
{
    return (ch + 1) % kBlock == 0 || ch == nch - 1;
}
__device__ __forceinline__ int block_buf(int ch) { return (ch / kBlock) & 1; }

// Runs the stage pipeline over nch stages.  gen(ch, tile) writes the operands
// of stage ch and returns false when one of its waits gave up; post(ch) runs
// on all threads once every thread has finished gen(ch); flush(col0) adds the
// finished TMEM block at column col0 into registers (all warps, converged).
// Returns false when a wait gave up.
template <class Gen, class Post, class Flush>
__device__ __forceinline__ bool tc_pipeline(int nch, const StageLayout &SL, uint32_t tmem,
                                            uint32_t idesc, int NT, uint64_t *bar, Gen &&gen,
                                            Post &&post, Flush &&flush)
{
    const int tid = threadIdx.x;
    for (int ch = 0; ch < nch; ++ch) {
        const int st = ch & 1;
        bool ok = true;
        // the MMAs of stage ch-2 (and all before) are complete once its commit arrived
        if (ch >= 2) ok = mbar_wait(smem_u32(&bar[st]), ((ch - 2) >> 1) & 1);
        if (__syncthreads_or(!ok)) return false;
        if (ch >= 2 && block_end(ch - 2, nch)) {
            tc_fence_after();
            flush((uint32_t)(block_buf(ch - 2) * 2 * NT));
            tc_fence_before();
        }
        unsigned char *tile = SL.stage[st];
        ok = gen(ch, tile);
        fence_async_smem();
        if (__syncthreads_or(!ok)) return false;
        post(ch);
        if (tid == 0) {
            const uint32_t a0 = smem_u32(tile), b0 = a0 + (uint32_t)kABytes;
            const uint32_t d = tmem + (uint32_t)(block_buf(ch) * 2 * NT);
            const bool fresh = ch % kBlock == 0;
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < kSlots; ++s)
                mma_tf32(d, smem_desc(a0 + 256u * s), smem_desc(b0 + 256u * s), idesc,
                         (fresh && s == 0) ? 0u : 1u);
            mma_commit(smem_u32(&bar[st]));
        }
    }
    if (nch == 0) return true;
    const bool ok = mbar_wait(smem_u32(&bar[(nch - 1) & 1]), ((nch - 1) >> 1) & 1);
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
    if (nch >= 2 && block_end(nch - 2, nch)) flush((uint32_t)(block_buf(nch - 2) * 2 * NT));
    flush((uint32_t)(block_buf(nch - 1) * 2 * NT));
    return true;
}

// shared-memory barriers (two MMA stages + nring copy slots) and the TMEM slot
struct CtaSync {
    uint64_t *bar;    // [2] MMA stages
    uint64_t *full;   // [nring] copy slots
    uint32_t *tslot;
};
__device__ __forceinline__ CtaSync cta_sync_at(void *end, int nring)
{
    CtaSync c;
    c.bar = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(end) + 15) & ~(uintptr_t)15);
    c.full = c.bar + 2;
    c.tslot = reinterpret_cast<uint32_t *>(c.full + nring);
    return c;
}
constexpr int kSyncBytes = 16 + 8 * (2 + 8) + 16;   // alignment, barriers, TMEM slot

__device__ __forceinline__ void cta_setup(const CtaSync &cs, int nring, uint32_t tcols)
{
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&cs.bar[0]), 1);
        mbar_init(smem_u32(&cs.bar[1]), 1);
        for (int k = 0; k < nring; ++k) mbar_init(smem_u32(&cs.full[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(cs.tslot), tcols);
}

// after an abandoned pipeline: bounded wait for the last committed MMA stage
__device__ __forceinline__ void drain(const CtaSync &cs, int nch)
{
    if (threadIdx.x == 0 && nch > 0)
        (void)mbar_wait(smem_u32(&cs.bar[(nch - 1) & 1]), ((nch - 1) >> 1) & 1);
}

__device__ __forceinline__ void cta_teardown(uint32_t tmem, uint32_t tcols)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// ------------------------------------------------------------------ P2M ---
// grid (leaf, row tile, column tile); V_r[leaf][row * ncol + col].  NT = 16 NTH
// complex columns; warp w reads TMEM lanes 32 (w & 3) .. and the complex
// columns [(w >> 2) NT/2, (w >> 2 + 1) NT/2) (real and imaginary parts).  The
// leaf's coordinates and coefficients are staged in shared memory once.
template <int NTH>
__global__ void __launch_bounds__(kThreads, 1) k_p2m_tc(const TcArgs a)
{
    constexpr int NT = 16 * NTH, NH = NT / 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    const StageLayout SL = stages(smem, NT);
    unsigned char *tail = smem + 2 * (kABytes + SL.wbytes);
    float2 *E = reinterpret_cast<float2 *>(tail);                      // [kKS][rowlen]
    float *xl = reinterpret_cast<float *>(E + kKS * a.rowlen);         // [d][lcap]
    float *ll = xl + a.d * a.lcap;                                     // [G][lcap]
    const CtaSync cs = cta_sync_at(ll + a.G * a.lcap, 0);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int leaf = blockIdx.x;
    const int row0 = blockIdx.y * kRows;
    const int n0c = blockIdx.z * NT;
    const int ntot = a.ncol * a.G;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = min(a.leaf_off[leaf + 1] - (int)p0, a.lcap);
    const int nch = (np + kKS - 1) / kKS;

    double c[RBF_MAX_DIM];
    leaf_centre(a, leaf, c);
    cta_setup(cs, 0, a.tcols);
    for (int idx = tid; idx < a.d * np; idx += kThreads) {
        const int t = idx / np, p = idx - t * np;
        xl[t * a.lcap + p] = a.xs[(int64_t)t * a.N + p0 + p];
    }
    for (int idx = tid; idx < a.G * np; idx += kThreads) {
        const int r = idx / np, p = idx - r * np;
        ll[r * a.lcap + p] = a.lam[(int64_t)r * a.N + p0 + p];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *cs.tslot;

    // A side: this thread's mode row and point quad
    const int rt = tid & (kRows - 1), qa = tid >> 7;
    const int row = row0 + rt;
    const bool row_ok = row < a.nrow;
    const RowFac rf = row_factors(row_ok ? row : 0, a.d, a.n0, a.n1);
    const int ocol = a.d == 1 ? 0 : a.n0 + (a.d - 2) * a.n1;
    // accumulators: lane quarter q, column half h
    const int q = warp & 3, h = warp >> 2;
    const uint32_t tlane = tmem + ((uint32_t)(32 * q) << 16);
    float acc_re[NH], acc_im[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) acc_re[j] = acc_im[j] = 0.0f;

    auto gen = [&](int ch, unsigned char *tile) -> bool {
        const int k0 = ch * kKS;
        const int cnt = min(kKS, np - k0);
        for (int idx = tid; idx < kKS * a.rowlen; idx += kThreads) {
            const int p = idx / a.rowlen, j = idx - p * a.rowlen;
            E[idx] = p < cnt ? table_entry(a, xl + k0 + p, a.lcap, j, c, -1.0f)
                             : make_float2(0.0f, 0.0f);
        }
        __syncthreads();
        {
            float re[4], im[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 v = row_ok ? row_phase(E + (4 * qa + e) * a.rowlen, rf, a.d)
                                        : make_float2(0.0f, 0.0f);
                re[e] = v.x;
                im[e] = v.y;
            }
            put_a(tile, rt, qa, re, im);
        }
        for (int idx = tid; idx < 2 * NT; idx += kThreads) {
            const int j = idx >> 1, qq = idx & 1;
            const int n = n0c + j;
            float wr[4] = {0, 0, 0, 0}, wi[4] = {0, 0, 0, 0};
            if (n < ntot) {
                const int r = n / a.ncol, col = n - r * a.ncol;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int p = 4 * qq + e;
                    const float2 ev = E[p * a.rowlen + ocol + col];
                    const float l = p < cnt ? ll[r * a.lcap + k0 + p] : 0.0f;
                    wr[e] = ev.x * l;
                    wi[e] = ev.y * l;
                }
            }
            put_w(tile + kABytes, j, NT, qq, wr, wi);
        }
        return true;
    };
    auto post = [&](int) {};
    auto flush = [&](uint32_t col0) {
#pragma unroll
        for (int g = 0; g < NTH; ++g) {
            float re[8], im[8];
            tmem_ld8(tlane + col0 + h * NH + 8 * g, re);
            tmem_ld8(tlane + col0 + NT + h * NH + 8 * g, im);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                acc_re[8 * g + e] += re[e];
                acc_im[8 * g + e] += im[e];
            }
        }
    };
    const bool ok = tc_pipeline(nch, SL, tmem, a.idesc, NT, cs.bar, gen, post, flush);
    if (ok) {
        // registers -> shared staging [kRows][NT + 1] -> coalesced stores
        __syncthreads();
        float2 *S = reinterpret_cast<float2 *>(smem);
        const int sst = NT + 1;
        const int r = 32 * q + lane;
#pragma unroll
        for (int j = 0; j < NH; ++j) S[r * sst + h * NH + j] = make_float2(acc_re[j], acc_im[j]);
        __syncthreads();
        for (int idx = tid; idx < kRows * NT; idx += kThreads) {
            const int rr = idx / NT, j = idx - rr * NT;
            const int n = n0c + j, grow = row0 + rr;
            if (grow >= a.nrow || n >= ntot) continue;
            const int rhs = n / a.ncol, col = n - rhs * a.ncol;
            a.V[(int64_t)rhs * a.vstride + (int64_t)leaf * a.mstride + (int64_t)grow * a.ncol + col] =
                S[rr * sst + j];
        }
    } else {
        drain(cs, nch);
    }
    cta_teardown(tmem, a.tcols);
}

// ------------------------------------------------------------------ L2P ---
// grid (leaf, point tile, RHS tile); the tile's NT = 16 NTH complex columns hold
// Rg whole right-hand sides (Rg * ncol <= NT), so every u_{i,r} is finished in
// the CTA.  Each block of T is contracted with B'_i at once:
//   S_i[j] += Re(B'_i[col(j)] T_i[j]),  u_{i,r} = sum of S_i over the columns of r.
// The kKS-row slices of L_r (contiguous: rows are row-major) arrive through a
// ring of kRing shared-memory slots, kRing stages ahead of their use.
constexpr int kRing = 6;

template <int NTH>
__global__ void __launch_bounds__(kThreads, 1) k_l2p_tc(const TcArgs a, int Rg)
{
    constexpr int NT = 16 * NTH, NH = NT / 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    const StageLayout SL = stages(smem, NT);
    unsigned char *tail = smem + 2 * (kABytes + SL.wbytes);
    const int slot_c = Rg * kKS * a.ncol;                              // complex per ring slot
    float2 *ring = reinterpret_cast<float2 *>(tail);                   // [kRing][Rg][kKS][ncol]
    float2 *E = ring + kRing * slot_c;                                 // [kRows][rowpad]
    const CtaSync cs = cta_sync_at(E + kRows * a.rowpad, kRing);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int leaf = blockIdx.x;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = a.leaf_off[leaf + 1] - (int)p0;
    const int pt0 = blockIdx.y * kRows;
    if (pt0 >= np) return;   // uniform: before any allocation or barrier
    const int cnt = min(kRows, np - pt0);
    const int rg0 = blockIdx.z * Rg;
    const int rgv = min(Rg, a.G - rg0);   // right-hand sides present in the tile
    const int ncolt = Rg * a.ncol;        // columns of the tile
    const int nch = (a.nrow + kKS - 1) / kKS;

    double c[RBF_MAX_DIM];
    leaf_centre(a, leaf, c);
    cta_setup(cs, kRing, a.tcols);
    // producer: one bulk copy per right-hand side and stage (16-byte multiple;
    // the allocation of L carries a 64-byte tail for the last round-up)
    int issued = 0;   // stages whose copies were issued (thread 0)
    auto issue = [&](int ch) {
        issued = ch + 1;
        const int k = ch % kRing;
        const int rows = min(kKS, a.nrow - ch * kKS);
        const uint32_t bytes = ((uint32_t)(rows * a.ncol) * 8u + 15u) & ~15u;
        const uint32_t fb = smem_u32(&cs.full[k]);
        mbar_expect_tx(fb, bytes * (uint32_t)rgv);
        for (int r = 0; r < rgv; ++r) {
            const float2 *src = a.L + (int64_t)(rg0 + r) * a.vstride + (int64_t)leaf * a.mstride +
                                (int64_t)ch * kKS * a.ncol;
            bulk_g2s(smem_u32(ring + k * slot_c + r * kKS * a.ncol), src, bytes, fb);
        }
    };
    if (tid == 0)
        for (int ch = 0; ch < min(kRing, nch); ++ch) issue(ch);
    // per-point phase tables e^{+i xi (x - c)} of the tile's points
    for (int idx = tid; idx < kRows * a.rowlen; idx += kThreads) {
        const int p = idx / a.rowlen, j = idx - p * a.rowlen;
        E[p * a.rowpad + j] = p < cnt ? table_entry(a, a.xs + p0 + pt0 + p, a.N, j, c, 1.0f)
                                      : make_float2(0.0f, 0.0f);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *cs.tslot;

    // A side: this thread's point and mode-row quad; W side: (column, quad) pair
    const int pa = tid & (kRows - 1), qa = tid >> 7;
    const float2 *Ep = E + pa * a.rowpad;
    const int jw = tid >> 1, qw = tid & 1;
    const int rlw = jw / a.ncol, colw = jw - rlw * a.ncol;
    const bool w_val = jw < ncolt && rlw < rgv;   // column present
    // contraction with B'_i: lane quarter q (points), column half h
    const int q = warp & 3, h = warp >> 2;
    const int i = 32 * q + lane;
    const uint32_t tlane = tmem + ((uint32_t)(32 * q) << 16);
    const int ocol = a.d == 1 ? 0 : a.n0 + (a.d - 2) * a.n1;
    const float2 *B = E + i * a.rowpad + ocol;
    float acc[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) acc[j] = 0.0f;

    auto gen = [&](int ch, unsigned char *tile) -> bool {
        {
            float re[4], im[4];
            const int rw0 = ch * kKS + 4 * qa;
            RowFac rf = row_factors(min(rw0, a.nrow - 1), a.d, a.n0, a.n1);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float2 v = make_float2(0.0f, 0.0f);
                if (rw0 + e < a.nrow) {
                    v = row_phase(Ep, rf, a.d);
                    row_next(rf, a.d, a.n0, a.n1);
                }
                re[e] = v.x;
                im[e] = v.y;
            }
            put_a(tile, pa, qa, re, im);
        }
        bool ok = true;
        if (jw < NT) {
            float wr[4] = {0, 0, 0, 0}, wi[4] = {0, 0, 0, 0};
            if (w_val) {
                const int k = ch % kRing;
                ok = mbar_wait(smem_u32(&cs.full[k]), (uint32_t)(ch / kRing) & 1u);
                const float2 *sl = ring + k * slot_c + rlw * kKS * a.ncol + colw;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int rr = 4 * qw + e;
                    if (ok && ch * kKS + rr < a.nrow) {
                        const float2 v = sl[rr * a.ncol];
                        wr[e] = v.x;
                        wi[e] = v.y;
                    }
                }
            }
            put_w(tile + kABytes, jw, NT, qw, wr, wi);
        }
        return ok;
    };
    // every thread is done with slot ch % kRing: refill it for stage ch + kRing
    auto post = [&](int ch) {
        if (tid == 0 && ch + kRing < nch) issue(ch + kRing);
    };
    auto flush = [&](uint32_t col0) {
#pragma unroll
        for (int g = 0; g < NTH; ++g) {
            float re[8], im[8];
            tmem_ld8(tlane + col0 + h * NH + 8 * g, re);
            tmem_ld8(tlane + col0 + NT + h * NH + 8 * g, im);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = h * NH + 8 * g + e;
                if (j < ncolt) {
                    const float2 b = B[j % a.ncol];
                    acc[8 * g + e] = fmaf(b.x, re[e], acc[8 * g + e]);
                    acc[8 * g + e] = fmaf(-b.y, im[e], acc[8 * g + e]);
                }
            }
        }
    };
    const bool ok = tc_pipeline(nch, SL, tmem, a.idesc, NT, cs.bar, gen, post, flush);
    if (ok) {
        // per-column sums -> shared [kRows][NT + 1] -> per-RHS sums in column order
        __syncthreads();
        float *S = reinterpret_cast<float *>(smem);
        const int sst = NT + 1;
#pragma unroll
        for (int j = 0; j < NH; ++j) S[i * sst + h * NH + j] = acc[j];
        __syncthreads();
        for (int idx = tid; idx < kRows * rgv; idx += kThreads) {
            const int pi = idx % kRows, rl = idx / kRows;
            if (pi >= cnt) continue;
            float u = 0.0f;
            for (int col = 0; col < a.ncol; ++col) u += S[pi * sst + rl * a.ncol + col];
            a.u[(int64_t)(rg0 + rl) * a.N + p0 + pt0 + pi] = u;
        }
    } else {
        drain(cs, nch);
        // bounded wait for the copies in flight: the latest issued phase of each slot
        if (tid == 0)
            for (int ch = std::max(0, issued - kRing); ch < issued; ++ch)
                (void)mbar_wait(smem_u32(&cs.full[ch % kRing]), (uint32_t)(ch / kRing) & 1u);
    }
    cta_teardown(tmem, a.tcols);
}

inline uint32_t tmem_cols(int n)
{
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

TcArgs base_args(const rbf_tree *t, const rbf_plan *p, int G)
{
    TcArgs a{};
    a.d = t->d;
    a.M = p->M;
    a.D = t->D;
    a.n0 = p->n0;
    a.n1 = p->n1;
    a.nrow = p->nrow;
    a.ncol = p->ncol;
    a.G = G;
    a.rowlen = t->d == 1 ? p->n0 : p->n0 + (t->d - 1) * p->n1;
    a.rowpad = a.rowlen | 1;
    a.lcap = std::max(1, (int)t->max_leaf);
    a.mstride = p->mstride;
    a.N = t->N;
    a.vstride = (int64_t)t->nleaf() * p->mstride;
    for (int q = 0; q < RBF_MAX_DIM; ++q) a.lo[q] = t->lo[q];
    a.side = t->side;
    a.xs = t->xs32;
    a.leaf_off = t->leaf_off;
    a.leaf_key = t->leaf_key();
    a.xi = (const float *)p->xi;
    return a;
}

constexpr size_t kSmemMax = 227 * 1024;
size_t stage_bytes(int NT) { return 2 * ((size_t)kABytes + (size_t)2 * NT * kKStage * 4); }

// P2M tile: complex columns per tile (16 NTH) and shared memory
void p2m_shape(const rbf_tree *t, const rbf_plan *p, int G, int *nth, size_t *smem)
{
    const int ntot = p->ncol * G;
    int best_c = 4;
    int64_t best = INT64_MAX;
    for (int c = 1; c <= 4; ++c) {
        const int64_t tiles = (ntot + 16 * c - 1) / (16 * c);
        const int64_t cost = tiles * (16 * c + 16);   // MMA columns + per-tile generation
        if (cost < best) {
            best = cost;
            best_c = c;
        }
    }
    *nth = best_c;
    const int rowlen = t->d == 1 ? p->n0 : p->n0 + (t->d - 1) * p->n1;
    *smem = stage_bytes(16 * best_c) + (size_t)kKS * rowlen * sizeof(float2) +
            (size_t)(t->d + G) * std::max(1, (int)t->max_leaf) * sizeof(float) + kSyncBytes;
}

// L2P tile: right-hand sides per tile, complex columns (16 NTH) and shared memory
void l2p_shape(const rbf_tree *t, const rbf_plan *p, int G, int *rg, int *nth, size_t *smem)
{
    int Rg = std::max(1, std::min(G, kMaxNT / p->ncol));
    const int rtiles = (G + Rg - 1) / Rg;
    Rg = (G + rtiles - 1) / rtiles;   // balance the tiles
    *rg = Rg;
    *nth = (Rg * p->ncol + 15) / 16;
    const int rowlen = t->d == 1 ? p->n0 : p->n0 + (t->d - 1) * p->n1;
    *smem = stage_bytes(16 * *nth) + (size_t)kRing * Rg * kKS * p->ncol * sizeof(float2) +
            (size_t)kRows * (rowlen | 1) * sizeof(float2) + kSyncBytes;
}

template <int NTH>
int launch_p2m(const TcArgs &a, dim3 grid, size_t smem, cudaStream_t s)
{
    RBF_CUDA_TRY(cudaFuncSetAttribute(k_p2m_tc<NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_p2m_tc<NTH><<<grid, kThreads, smem, s>>>(a);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

template <int NTH>
int launch_l2p(const TcArgs &a, int Rg, dim3 grid, size_t smem, cudaStream_t s)
{
    RBF_CUDA_TRY(cudaFuncSetAttribute(k_l2p_tc<NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_l2p_tc<NTH><<<grid, kThreads, smem, s>>>(a, Rg);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

}  // namespace

int rbf_far_multi_supported(const rbf_plan *p) { return p->ncol <= kMaxNT; }

int rbf_run_far_multi(rbf_tree *t, const rbf_plan *p, const float *lam_s, int G, float2 *V,
                      float2 *L, float *u_far, cudaStream_t s)
{
    RBF_REQUIRE(G >= 1 && p->ncol <= kMaxNT, "rbf_run_far_multi: G=%d, %d columns", G, p->ncol);
    const int nleaf = t->nleaf();
    const int64_t vstride = (int64_t)nleaf * p->mstride;
    // The tensor-core contractions pay off when a leaf fills the K dimension
    // (P2M: points) or the M dimension (L2P: points per 128-row tile); with
    // fewer points per leaf the CUDA-core kernels run column by column.
    const double per_leaf = (double)t->N / std::max(1, nleaf);
    int nth = 0;
    size_t smem = 0;
    p2m_shape(t, p, G, &nth, &smem);
    if (per_leaf >= 64.0 && smem <= kSmemMax) {
        TcArgs a = base_args(t, p, G);
        a.lam = lam_s;
        a.V = V;
        a.NT = 16 * nth;
        a.idesc = instr_desc_tf32(kRows, 2 * a.NT);
        a.tcols = tmem_cols(4 * a.NT);
        const int ntiles = (p->ncol * G + a.NT - 1) / a.NT;
        dim3 grid(nleaf, ceil_div(p->nrow, kRows), ntiles);
        RBF_REQUIRE(grid.y < 65536 && grid.z < 65536, "rbf_run_far_multi: expansion too large");
        rbf_pass_timer tm(t, RBF_PASS_P2M, s);
        switch (nth) {
        case 1: RBF_TRY(launch_p2m<1>(a, grid, smem, s)); break;
        case 2: RBF_TRY(launch_p2m<2>(a, grid, smem, s)); break;
        case 3: RBF_TRY(launch_p2m<3>(a, grid, smem, s)); break;
        default: RBF_TRY(launch_p2m<4>(a, grid, smem, s)); break;
        }
    } else {
        for (int g = 0; g < G; ++g)
            RBF_TRY(rbf_run_p2m<float>(t, p, lam_s + g * t->N, V + g * vstride, s));
    }
    for (int g = 0; g < G; ++g) {
        RBF_TRY(rbf_run_m2m<float>(t, p, V + g * vstride, s));
        RBF_TRY(rbf_run_m2l<float>(t, p, V + g * vstride, L + g * vstride, s));
    }
    int Rg = 0;
    l2p_shape(t, p, G, &Rg, &nth, &smem);
    if (per_leaf >= 96.0 && smem <= kSmemMax) {
        TcArgs a = base_args(t, p, G);
        a.L = L;
        a.u = u_far;
        a.NT = 16 * nth;
        a.idesc = instr_desc_tf32(kRows, 2 * a.NT);
        a.tcols = tmem_cols(4 * a.NT);
        const int rtiles = (G + Rg - 1) / Rg;
        dim3 grid(nleaf, ceil_div(std::max<int>(t->max_leaf, 1), kRows), rtiles);
        RBF_REQUIRE(grid.y < 65536, "rbf_run_far_multi: leaf too large");
        rbf_pass_timer tm(t, RBF_PASS_L2P, s);
        switch (nth) {
        case 1: RBF_TRY(launch_l2p<1>(a, Rg, grid, smem, s)); break;
        case 2: RBF_TRY(launch_l2p<2>(a, Rg, grid, smem, s)); break;
        case 3: RBF_TRY(launch_l2p<3>(a, Rg, grid, smem, s)); break;
        default: RBF_TRY(launch_l2p<4>(a, Rg, grid, smem, s)); break;
        }
    } else {
        for (int g = 0; g < G; ++g)
            RBF_TRY(rbf_run_l2p<float>(t, p, L + g * vstride, u_far + g * t->N, s));
    }
    return RBF_OK;
}

int rbf_tc_fetch_status(int *flags_host)
{
    unsigned int v = 0, zero = 0;
    RBF_CUDA_TRY(cudaDeviceSynchronize());
    RBF_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(v)));
    RBF_CUDA_TRY(cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(zero)));
    if (flags_host) *flags_host = (int)v;
    return RBF_OK;
}
