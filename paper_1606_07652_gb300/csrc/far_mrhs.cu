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
// k-steps per point (P2M) or per mode row (L2P).  With x = hi + lo,
// hi = tf32(x), lo = tf32(x - hi), the six k-steps pair
//     A:  re_hi  im_hi  re_hi  im_hi  re_lo  im_lo
//     Wr: wr_hi -wi_hi  wr_lo -wi_lo  wr_hi -wi_hi      (output column: real part)
//     Wi: wi_hi  wr_hi  wi_lo  wr_lo  wi_hi  wr_hi      (output column: imaginary part)
// so that a column of real parts accumulates A_re W_re - A_im W_im and a
// column of imaginary parts A_re W_im + A_im W_re, every real product taken as
// hi*hi + hi*lo + lo*hi (three-term split TF32, FP32-level accuracy).  Only
// four slots of each operand are stored (A: re_hi im_hi re_lo im_lo; W: its
// first four); the descriptors of k-steps 2..5 point at the slots they repeat.
//
// Tile: 128 rows (TMEM lanes) x 2*NT real columns (NT complex: 16, 32, 48 or
// 64); K advances 8 points (mode rows) = 48 TF32 values per stage.  Operands
// are K-major without swizzle: 8-row x 16-byte core matrices, 128 B apart
// along K and 1536 B apart along rows.  The CTA is split by warp roles:
//   producers (8 warps)  build the operands of a ring of stages,
//   MMA (1 warp)         one lane issues the six MMAs of a stage, commits them
//                        to the stage's "empty" barrier and, at the end of an
//                        accumulation block, to the block's "full" barrier,
//   epilogue (8 warps)   add each finished block into FP32 registers,
//   copy (1 warp, L2P)   streams the mode rows of the local expansions into a
//                        ring of shared-memory slots with bulk copies (TMA).
// Roles meet only at mbarriers; every wait on one is bounded.  A wait that
// gives up sets a status bit (read by rbf_tc_fetch_status) and a shared abort
// flag; the roles then skip their remaining work (producers still pass their
// named barriers), the MMA lane waits once more (bounded) for its last
// commit, tensor memory is freed and the kernel returns.
#include <algorithm>

#include "rbf_internal.cuh"

namespace {

constexpr int kRows = 128;           // tile rows = TMEM lanes
constexpr int kKS = 8;               // points (P2M) or mode rows (L2P) per stage
constexpr int kSlots = 6;                      // MMA k-steps per stage
constexpr int kStore = 4;                      // operand slots stored per stage
constexpr int kKStage = kStore * kKS;          // 32 TF32 values of K stored per stage
constexpr int kCoreK = kKStage / 4;            // 8 core matrices along K
constexpr uint32_t kLBO = 128;                 // next core matrix along K
constexpr uint32_t kSBO = kCoreK * 128;        // next group of 8 rows
constexpr int kABytes = kRows * kKStage * 4;   // 16384
constexpr long long kWaitCycles = 4000000000LL;
constexpr uint32_t kSuspendNs = 200000;       // try_wait suspend-time hint
#ifndef RBF_TC_BACKOFF_NS
#define RBF_TC_BACKOFF_NS 64
#endif
constexpr unsigned kBackoffNs = RBF_TC_BACKOFF_NS;   // sleep after a failed try_wait
constexpr int kMaxNT = 64;                     // complex columns of a tile

__device__ unsigned int g_tc_status;

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// x = hi + lo: hi = x rounded to TF32 (nearest, ties away: add half of the 13
// dropped bits, clear them), lo = x - hi exactly; the MMA reads lo's top 19 bits
// (truncation, at most 2^-21 |x|), so x is carried to FP32-level accuracy
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
    lo = x - hi;
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

// test for the completion of phase `parity`; a thread whose phase is not complete
// is suspended (up to the hint, in ns) instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
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

// stores the four slots of a row of the A-side operand (4 consecutive K values):
// re_hi, im_hi, re_lo, im_lo
__device__ __forceinline__ void put_a(unsigned char *tile, int r, int q, const float *re,
                                      const float *im)
{
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        split_tf32(re[e], rh[e], rl[e]);
        split_tf32(im[e], ih[e], il[e]);
    }
    *reinterpret_cast<float4 *>(tile + op_off(r, 0, q)) = make_float4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<float4 *>(tile + op_off(r, 1, q)) = make_float4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<float4 *>(tile + op_off(r, 2, q)) = make_float4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<float4 *>(tile + op_off(r, 3, q)) = make_float4(il[0], il[1], il[2], il[3]);
}

// stores one row of the W-side operand for complex column j: half 0 = the
// real-part row j (wr_hi, -wi_hi, wr_lo, -wi_lo), half 1 = the imaginary-part
// row NT + j (wi_hi, wr_hi, wi_lo, wr_lo)
__device__ __forceinline__ void put_w_half(unsigned char *tile, int j, int NT, int q, int half,
                                           const float *wr, const float *wi)
{
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        split_tf32(wr[e], rh[e], rl[e]);
        split_tf32(wi[e], ih[e], il[e]);
    }
    if (half == 0) {
        *reinterpret_cast<float4 *>(tile + op_off(j, 0, q)) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4 *>(tile + op_off(j, 1, q)) = make_float4(-ih[0], -ih[1], -ih[2], -ih[3]);
        *reinterpret_cast<float4 *>(tile + op_off(j, 2, q)) = make_float4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<float4 *>(tile + op_off(j, 3, q)) = make_float4(-il[0], -il[1], -il[2], -il[3]);
    } else {
        const int n = NT + j;
        *reinterpret_cast<float4 *>(tile + op_off(n, 0, q)) = make_float4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<float4 *>(tile + op_off(n, 1, q)) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4 *>(tile + op_off(n, 2, q)) = make_float4(il[0], il[1], il[2], il[3]);
        *reinterpret_cast<float4 *>(tile + op_off(n, 3, q)) = make_float4(rl[0], rl[1], rl[2], rl[3]);
    }
}

__device__ __forceinline__ void decode_key(uint64_t key, int d, int l, int *k)
{
    for (int t = 0; t < d; ++t) k[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) k[t] |= (int)((key >> (b * d + t)) & 1u) << b;
}

struct TcArgs {
    int d, M, D, n0, n1, nrow, ncol, G;
    int NT;                  // complex columns of the tile (16, 32, 48 or 64)
    int rowlen, rowpad;      // per-point table length, padded row stride (odd)
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

// ---------------------------------------------------------- warp roles ----
// average points per leaf from which P2M / L2P of several columns run on the
// tensor cores (measured crossovers)
#ifndef RBF_TC_P2M_MIN
#define RBF_TC_P2M_MIN 64
#endif
#ifndef RBF_TC_L2P_MIN
#define RBF_TC_L2P_MIN 96
#endif
#ifndef RBF_TC_GROUPS
#define RBF_TC_GROUPS 3
#endif
constexpr int kGroups = RBF_TC_GROUPS;                 // producer groups of four warps
// two and three groups are tested; four (832 threads, 72 registers) ran out a bounded
// wait in testing with the cause not found, so they are not allowed
static_assert(kGroups == 2 || kGroups == 3, "RBF_TC_GROUPS must be 2 or 3");
constexpr int kProdWarps = 4 * kGroups;                // warps 0..4G-1: operand producers
constexpr int kProdThreads = 32 * kProdWarps;
constexpr int kMmaWarp = kProdWarps;                   // MMA issue (one lane)
constexpr int kEpiWarp0 = kProdWarps + 1;              // 8 warps: accumulator epilogue
constexpr int kEpiWarps = 8;
constexpr int kCopyWarp = kEpiWarp0 + kEpiWarps;       // bulk copies
constexpr int kTcThreads = 32 * (kCopyWarp + 1);
#ifndef RBF_P2M_STAGES
#define RBF_P2M_STAGES 4
#endif
#ifndef RBF_L2P_STAGES
#define RBF_L2P_STAGES 4
#endif
constexpr int kP2MStages = RBF_P2M_STAGES, kL2PStages = RBF_L2P_STAGES;
constexpr int kMaxStages = kP2MStages > kL2PStages ? kP2MStages : kL2PStages;
constexpr int kRing = 8;                               // copy-slot barriers
constexpr int kRingE = 8, kRingL = 6;                  // copy slots of P2M, L2P
// named barriers (0 = __syncthreads): all producers, epilogue, P2M producer groups
constexpr int kBarProd = 1, kBarEpi = 2, kBarGrp0 = 3;
constexpr int kPF = 48;   // prefixes per 128-row tile: 128 / n1 + 2 <= 48 for n1 >= 3

// Accumulation blocks: the MMAs of kBlock consecutive stages of a work item
// accumulate into one of two TMEM buffers (columns [buf * 2NT, buf * 2NT + 2NT)),
// starting from zero; the epilogue adds a finished block into FP32 registers
// with round-to-nearest adds.  The tensor core's own accumulation rounds
// towards zero, so a long chain of MMAs into one accumulator shrinks it by
// about one ulp per MMA; short blocks keep that below 1e-6 relative.
constexpr int kBlock = 2;
__host__ __device__ __forceinline__ bool block_end(int ch, int nch)
{
    return (ch + 1) % kBlock == 0 || ch == nch - 1;
}

struct Sync {
    uint64_t *full, *empty;   // [kMaxStages] producers -> MMA, MMA -> producers
    uint64_t *accf, *acce;    // [2] MMA -> epilogue (block done), epilogue -> MMA (drained)
    uint64_t *rfull, *rempty; // [kRing] copies landed, slot consumed
    uint32_t *tslot;
    volatile int *abort;
};
constexpr int kSyncBytes = 16 + 8 * (2 * kMaxStages + 4 + 2 * kRing) + 16;

__device__ __forceinline__ Sync sync_at(void *end)
{
    Sync y;
    uint64_t *b = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(end) + 15) & ~(uintptr_t)15);
    y.full = b;
    y.empty = b + kMaxStages;
    y.accf = b + 2 * kMaxStages;
    y.acce = y.accf + 2;
    y.rfull = y.acce + 2;
    y.rempty = y.rfull + kRing;
    y.tslot = reinterpret_cast<uint32_t *>(y.rempty + kRing);
    y.abort = reinterpret_cast<volatile int *>(y.tslot + 1);
    return y;
}

// parts: producer warps that arrive per stage (and per copy slot)
__device__ __forceinline__ void sync_init(const Sync &y, int parts)
{
    for (int k = 0; k < kMaxStages; ++k) {
        mbar_init(smem_u32(&y.full[k]), parts);
        mbar_init(smem_u32(&y.empty[k]), 1);
    }
    for (int k = 0; k < 2; ++k) {
        mbar_init(smem_u32(&y.accf[k]), 1);
        mbar_init(smem_u32(&y.acce[k]), kEpiWarps);
    }
    for (int k = 0; k < kRing; ++k) {
        mbar_init(smem_u32(&y.rfull[k]), 1);
        mbar_init(smem_u32(&y.rempty[k]), parts);
    }
    *y.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void named_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    const uint32_t b = smem_u32(bar);
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(&g_tc_status, 1u);
            *abort = 1;
            return false;
        }
        __nanosleep(kBackoffNs);   // leave the issue slots to the warps with work
    }
    return true;
}

// bounded wait used while draining after an abort
__device__ __forceinline__ void wait_bounded(uint64_t *bar, uint32_t parity)
{
    const uint32_t b = smem_u32(bar);
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity) && clock64() - t0 < kWaitCycles) {
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

// MMA lane, one work item of nch stages: six MMAs per stage into the block's
// TMEM buffer; commits to the stage's empty barrier and, at a block end, to the
// block's full barrier.  gc / gb count stages / blocks over all items.
template <int S>
__device__ __forceinline__ void mma_item(const Sync &y, int nch, int &gc, int &gb, int &last,
                                         unsigned char *smem, uint32_t sbytes, uint32_t tmem,
                                         uint32_t idesc, int NT)
{
    for (int lc = 0; lc < nch; ++lc, ++gc) {
        const int s = gc % S, buf = gb & 1;
        if (*y.abort) {
            if (block_end(lc, nch)) ++gb;
            continue;
        }
        if (lc % kBlock == 0 && gb >= 2 && !wait_or_abort(&y.acce[buf], ((gb - 2) >> 1) & 1, y.abort))
            continue;
        if (!wait_or_abort(&y.full[s], (gc / S) & 1, y.abort)) continue;
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + s * sbytes), b0 = a0 + (uint32_t)kABytes;
        const uint32_t d = tmem + (uint32_t)(buf * 2 * NT);
        const bool fresh = lc % kBlock == 0;
        // stored slots of the six k-steps: A (hi, hi, hi, hi, lo, lo), W (hi, hi, lo, lo, hi, hi)
        constexpr uint32_t sa[kSlots] = {0, 1, 0, 1, 2, 3}, sw[kSlots] = {0, 1, 2, 3, 0, 1};
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
            mma_tf32(d, smem_desc(a0 + 256u * sa[k]), smem_desc(b0 + 256u * sw[k]), idesc,
                     (fresh && k == 0) ? 0u : 1u);
        mma_commit(smem_u32(&y.empty[s]));
        if (block_end(lc, nch)) {
            mma_commit(smem_u32(&y.accf[buf]));
            ++gb;
        }
        last = gc;
    }
}

// epilogue warp, one work item: add its blocks into acc_re / acc_im (zeroed here)
template <int NTH>
__device__ __forceinline__ void epi_item(const Sync &y, int nch, int &gb, uint32_t tlane, int h,
                                         float *acc_re, float *acc_im)
{
    constexpr int NT = 16 * NTH, NH = NT / 2;
#pragma unroll
    for (int j = 0; j < NH; ++j) acc_re[j] = acc_im[j] = 0.0f;
    const int nb = (nch + kBlock - 1) / kBlock;
    for (int b = 0; b < nb; ++b, ++gb) {
        const int buf = gb & 1;
        if (*y.abort || !wait_or_abort(&y.accf[buf], (gb >> 1) & 1, y.abort)) continue;
        tc_fence_after();
        const uint32_t col0 = (uint32_t)(buf * 2 * NT);
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
        tc_fence_before();
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(smem_u32(&y.acce[buf]));
    }
}

// ---------------------------------------------------------- point tables --
// E[i][j] = e^{-i xi_k (x_{i,t} - c_t)} of every point i (sorted order) for the
// table entries j of Eq. (P2M) (dimension-0 segment k0 = 0..M/2, then
// k = -M/2..M/2 per dimension), rows padded to rowpadE (even) entries; and the
// coefficients of the group, point-major: Lt[i][r] = lambda_r[i] (gpad columns,
// a multiple of 4, zero beyond G).
__global__ void __launch_bounds__(256) k_point_tables(const TcArgs a, int rowpadE, float2 *Eg,
                                                      int gpad, float *Lt)
{
    const int leaf = blockIdx.x;
    const int64_t p0 = a.leaf_off[leaf];
    const int np = a.leaf_off[leaf + 1] - (int)p0;
    double c[RBF_MAX_DIM];
    leaf_centre(a, leaf, c);
    for (int idx = threadIdx.x; idx < np * rowpadE; idx += blockDim.x) {
        const int p = idx / rowpadE, j = idx - p * rowpadE;
        Eg[(p0 + p) * rowpadE + j] = j < a.rowlen ? table_entry(a, a.xs + p0 + p, a.N, j, c, -1.0f)
                                                  : make_float2(0.0f, 0.0f);
    }
    if (Lt)
        for (int idx = threadIdx.x; idx < np * gpad; idx += blockDim.x) {
            const int p = idx / gpad, r = idx - p * gpad;
            Lt[(p0 + p) * gpad + r] = r < a.G ? a.lam[(int64_t)r * a.N + p0 + p] : 0.0f;
        }
}

// ------------------------------------------------------------------ P2M ---
// Persistent: CTA blockIdx.x takes the work items w = blockIdx.x + k gridDim.x,
// w = (leaf * ntile1 + row tile) * ntile2 + column tile, with V_r[leaf][row *
// ncol + col] as output.  NT = 16 NTH complex columns.  Epilogue warp w reads
// TMEM lanes 32 (w & 3) .. and the complex columns [h NT/2, (h + 1) NT/2),
// h = (w - kEpiWarp0) / 4.  The copy warp streams the stage's rows of the point
// tables and coefficients into a ring of kRingE slots.  A mode row is (prefix,
// k_{d-2}) with prefix = (k0, .., k_{d-3}); the prefix products of the tile's
// prefixes are formed once per stage, so an A element costs one complex product.
template <int NTH>
__global__ void __launch_bounds__(kTcThreads, 1) k_p2m_tc(const TcArgs a, const float2 *Eg,
                                                          const float *Lt, int rowpadE, int gpad,
                                                          int ntile1, int ntile2, int nitems)
{
    constexpr int NT = 16 * NTH, NH = NT / 2, S = kP2MStages;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t wbytes = (uint32_t)(2 * NT) * kKStage * 4;
    const uint32_t sbytes = kABytes + wbytes;
    const int eslot = kKS * rowpadE, lslot = kKS * gpad;
    float2 *Er = reinterpret_cast<float2 *>(smem + S * sbytes);       // [kRingE][kKS][rowpadE]
    float *Lr = reinterpret_cast<float *>(Er + kRingE * eslot);        // [kRingE][kKS][gpad]
    float2 *PF = reinterpret_cast<float2 *>(Lr + kRingE * lslot);      // [groups][2][kKS][kPF]
    int *pfo = reinterpret_cast<int *>(PF + 2 * kGroups * kKS * kPF);  // [2][kPF][RBF_MAX_DIM]
    const Sync y = sync_at(pfo + 2 * kPF * RBF_MAX_DIM);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntot = a.ncol * a.G;
    if (tid == 0) sync_init(y, 4);
    __syncwarp();
    if (warp == 0) tmem_alloc(smem_u32(y.tslot), a.tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *y.tslot;

    int gc = 0, gb = 0;          // stages and blocks of all items handled so far (per role)
    int last = -1, issued = 0;   // last committed stage (MMA lane), stages copied (copy lane)
    int nit = 0;                 // items handled by this CTA
    for (int w = blockIdx.x; w < nitems; w += gridDim.x, ++nit) {
        const int ct = w % ntile2, rtile = (w / ntile2) % ntile1, leaf = w / (ntile2 * ntile1);
        const int row0 = rtile * kRows, n0c = ct * NT;
        const int64_t p0 = a.leaf_off[leaf];
        const int np = a.leaf_off[leaf + 1] - (int)p0;
        const int nch = (np + kKS - 1) / kKS;
        if (warp < kProdWarps) {
            // ---- producers: groups of four warps build stages in turn, so the
            // latency chains of several stages overlap
            const int grp = warp >> 2, gt = tid & 127;
            const int rlast = min(row0 + kRows, a.nrow) - 1;
            const int qbase = a.d >= 3 ? row0 / a.n1 : 0;
            const int npf = a.d >= 3 ? rlast / a.n1 - qbase + 1 : 0;
            const int row = row0 + gt;
            const bool row_ok = row < a.nrow;
            const int qloc = a.d >= 3 && row_ok ? row / a.n1 - qbase : 0;
            const int oe = a.d >= 3 ? a.n0 + (a.d - 3) * a.n1 + (row_ok ? row % a.n1 : 0)
                                    : (row_ok ? row : 0);
            const int ocol = a.d == 1 ? 0 : a.n0 + (a.d - 2) * a.n1;
            // table offsets of the tile's prefixes, one buffer per item parity (every
            // producer finished the item before last at the previous item's barrier)
            int *pfi = pfo + (nit & 1) * kPF * RBF_MAX_DIM;
            for (int q = tid; q < npf; q += kProdThreads) {
                int Q = qbase + q;
                for (int t = a.d - 3; t >= 1; --t) {
                    pfi[q * RBF_MAX_DIM + t] = a.n0 + (t - 1) * a.n1 + Q % a.n1;
                    Q /= a.n1;
                }
                pfi[q * RBF_MAX_DIM] = Q;
            }
            named_bar(kBarProd, kProdThreads);
            for (int lc = grp; lc < nch; lc += kGroups) {
                const int gcc = gc + lc;
                const int s = gcc % S, k = gcc % kRingE;
                if (gcc >= S && !*y.abort) (void)wait_or_abort(&y.empty[s], ((gcc - S) / S) & 1, y.abort);
                if (!*y.abort) (void)wait_or_abort(&y.rfull[k], (uint32_t)(gcc / kRingE) & 1u, y.abort);
                const int cnt = min(kKS, np - lc * kKS);
                const float2 *Ec = Er + k * eslot;
                const float *Lc = Lr + k * lslot;
                float2 *PFc = PF + (grp * 2 + ((lc / kGroups) & 1)) * kKS * kPF;
                if (!*y.abort)
                    for (int idx = gt; idx < kKS * npf; idx += 128) {
                        const int p = idx / npf, q = idx - p * npf;
                        float2 v = make_float2(0.0f, 0.0f);
                        if (p < cnt) {
                            const float2 *Epp = Ec + p * rowpadE;
                            const int *o = pfi + q * RBF_MAX_DIM;
                            v = Epp[o[0]];
                            for (int t = 1; t <= a.d - 3; ++t) v = cmul(v, Epp[o[t]]);
                        }
                        PFc[p * kPF + q] = v;
                    }
                named_bar(kBarGrp0 + grp, 128);
                if (!*y.abort) {
                    unsigned char *tile = smem + s * sbytes;
#pragma unroll
                    for (int qa = 0; qa < 2; ++qa) {
                        float re[4], im[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int p = 4 * qa + e;
                            float2 v = make_float2(0.0f, 0.0f);
                            if (row_ok && p < cnt) {
                                if (a.d >= 3) v = cmul(PFc[p * kPF + qloc], Ec[p * rowpadE + oe]);
                                else if (a.d == 2) v = Ec[p * rowpadE + oe];
                                else v = make_float2(1.0f, 0.0f);
                            }
                            re[e] = v.x;
                            im[e] = v.y;
                        }
                        put_a(tile, gt, qa, re, im);
                    }
                    // W rows: one (column, point quad, half) per item
                    for (int idx = gt; idx < 4 * NT; idx += 128) {
                        const int j = idx >> 2, qq = (idx >> 1) & 1, half = idx & 1;
                        const int n = n0c + j;
                        float wr[4] = {0, 0, 0, 0}, wi[4] = {0, 0, 0, 0};
                        if (n < ntot) {
                            const int r = n / a.ncol, col = n - r * a.ncol;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int p = 4 * qq + e;
                                if (p < cnt) {
                                    const float2 ev = Ec[p * rowpadE + ocol + col];
                                    const float l = Lc[p * gpad + r];
                                    wr[e] = ev.x * l;
                                    wi[e] = ev.y * l;
                                }
                            }
                        }
                        put_w_half(tile + kABytes, j, NT, qq, half, wr, wi);
                    }
                    fence_async_smem();
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&y.full[s]));
                    mbar_arrive(smem_u32(&y.rempty[k]));
                }
            }
            gc += nch;
        } else if (warp == kMmaWarp) {
            if (lane == 0) mma_item<S>(y, nch, gc, gb, last, smem, sbytes, tmem, a.idesc, NT);
        } else if (warp == kCopyWarp) {
            // ---- copies of the stage's table rows (cnt * rowpadE * 8 bytes) and
            // coefficient rows (cnt * gpad * 4 bytes), multiples of 16
            if (lane == 0) {
                for (int lc = 0; lc < nch; ++lc, ++gc) {
                    const int k = gc % kRingE;
                    if (*y.abort) continue;
                    if (gc >= kRingE &&
                        !wait_or_abort(&y.rempty[k], (uint32_t)((gc - kRingE) / kRingE) & 1u, y.abort))
                        continue;
                    const int cnt = min(kKS, np - lc * kKS);
                    const int64_t pt = p0 + (int64_t)lc * kKS;
                    const uint32_t be = (uint32_t)(cnt * rowpadE) * 8u, bl = (uint32_t)(cnt * gpad) * 4u;
                    const uint32_t fb = smem_u32(&y.rfull[k]);
                    mbar_expect_tx(fb, be + bl);
                    bulk_g2s(smem_u32(Er + k * eslot), Eg + pt * rowpadE, be, fb);
                    bulk_g2s(smem_u32(Lr + k * lslot), Lt + pt * gpad, bl, fb);
                    issued = gc + 1;
                }
            }
        } else {
            // ---- epilogue: blocks -> registers -> V
            const int ew = warp - kEpiWarp0, q = warp & 3, h = ew >> 2;
            const uint32_t tlane = tmem + ((uint32_t)(32 * q) << 16);
            float acc_re[NH], acc_im[NH];
            epi_item<NTH>(y, nch, gb, tlane, h, acc_re, acc_im);
            const int row = row0 + 32 * q + lane;
            if (!*y.abort && row < a.nrow) {
                int n = n0c + h * NH;
                int rhs = n / a.ncol, col = n - rhs * a.ncol;
                float2 *out = a.V + (int64_t)leaf * a.mstride + (int64_t)row * a.ncol;
#pragma unroll
                for (int j = 0; j < NH; ++j) {
                    if (n + j < ntot)
                        out[(int64_t)rhs * a.vstride + col] = make_float2(acc_re[j], acc_im[j]);
                    if (++col == a.ncol) {
                        col = 0;
                        ++rhs;
                    }
                }
            }
        }
    }
    if (*y.abort) {   // bounded waits for the MMAs and copies still in flight
        if (warp == kMmaWarp && lane == 0 && last >= 0)
            wait_bounded(&y.empty[last % S], (uint32_t)(last / S) & 1u);
        if (warp == kCopyWarp && lane == 0)
            for (int c2 = max(0, issued - kRingE); c2 < issued; ++c2)
                wait_bounded(&y.rfull[c2 % kRingE], (uint32_t)(c2 / kRingE) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tcols);
    }
}

// ------------------------------------------------------------------ L2P ---
// Persistent: work item w = (leaf * nptile + point tile) * nrt + RHS tile; items
// whose point tile is beyond the leaf are skipped by every role.  The tile's NT
// = 16 NTH complex columns hold Rg whole right-hand sides (Rg * ncol <= NT), so
// every u_{i,r} is finished in the CTA.  The kKS-row slices of L_r
// (contiguous: rows are row-major) arrive through a ring of kRingL slots filled
// by the copy warp.  At the end of an item the epilogue contracts T with
// B'_i = conj(E_{d-1}[i]) (from the point tables) and sums the columns of each
// right-hand side in column order.
template <int NTH>
__global__ void __launch_bounds__(kTcThreads, 1) k_l2p_tc(const TcArgs a, const float2 *Eg,
                                                          int rowpadE, int Rg, int nptile, int nrt,
                                                          int nitems)
{
    constexpr int NT = 16 * NTH, NH = NT / 2, S = kL2PStages;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t wbytes = (uint32_t)(2 * NT) * kKStage * 4;
    const uint32_t sbytes = kABytes + wbytes;
    const int slot_c = Rg * kKS * a.ncol;                              // complex per ring slot
    float2 *ring = reinterpret_cast<float2 *>(smem + S * sbytes);      // [kRingL][Rg][kKS][ncol]
    float2 *E = ring + kRingL * slot_c;                                // [kRows][rowpad]
    float *Sg = reinterpret_cast<float *>(E + kRows * a.rowpad);       // [kRows][2][Rg]
    const Sync y = sync_at(Sg + kRows * 2 * Rg);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncolt = Rg * a.ncol;        // columns of the tile
    const int nch = (a.nrow + kKS - 1) / kKS;
    if (tid == 0) sync_init(y, 4);
    __syncwarp();
    if (warp == 0) tmem_alloc(smem_u32(y.tslot), a.tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *y.tslot;

    int gc = 0, gb = 0;          // stages and blocks of all items handled so far (per role)
    int last = -1, issued = 0;   // last committed stage (MMA lane), stages copied (copy lane)
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const int rt_ = w % nrt, ptile = (w / nrt) % nptile, leaf = w / (nrt * nptile);
        const int64_t p0 = a.leaf_off[leaf];
        const int np = a.leaf_off[leaf + 1] - (int)p0;
        const int pt0 = ptile * kRows;
        if (pt0 >= np) continue;   // same decision in every role
        const int cnt = min(kRows, np - pt0);
        const int rg0 = rt_ * Rg;
        const int rgv = min(Rg, a.G - rg0);
        if (warp < kProdWarps) {
            // ---- producers: per-point phases e^{+i xi (x - c)} of the item, then stages
            double c[RBF_MAX_DIM];
            leaf_centre(a, leaf, c);
            named_bar(kBarProd, kProdThreads);   // every producer is done with the previous item
            for (int idx = tid; idx < kRows * a.rowlen; idx += kProdThreads) {
                const int p = idx / a.rowlen, j = idx - p * a.rowlen;
                E[p * a.rowpad + j] = p < cnt ? table_entry(a, a.xs + p0 + pt0 + p, a.N, j, c, 1.0f)
                                              : make_float2(0.0f, 0.0f);
            }
            named_bar(kBarProd, kProdThreads);
            // groups of four warps take stages in turn; thread gt of a group
            // owns point gt (all 8 mode rows of a stage) and up to two W rows
            const int grp = warp >> 2, gt = tid & 127;
            const float2 *Ep = E + gt * a.rowpad;
            const float2 *Elast = Ep + (a.d >= 3 ? a.n0 + (a.d - 3) * a.n1 : 0);
            // mode row = (prefix digits dg, k_{d-2} = kl), advanced row by row
            int dg[RBF_MAX_DIM - 2] = {0, 0, 0, 0};
            int kl = 0;
            float2 pf = make_float2(1.0f, 0.0f);
            // (fixed-size unrolled loops keep the digits in registers)
            auto prefix_from_digits = [&]() {
                float2 v = Ep[dg[0]];
#pragma unroll
                for (int t = 1; t < RBF_MAX_DIM - 2; ++t)
                    if (t <= a.d - 3) v = cmul(v, Ep[a.n0 + (t - 1) * a.n1 + dg[t]]);
                return v;
            };
            auto advance = [&](int rows) {   // kl += rows with carries into the prefix
                bool moved = false;
                kl += rows;
                while (kl >= a.n1) {
                    kl -= a.n1;
                    moved = true;
                    bool carry = true;
#pragma unroll
                    for (int t = RBF_MAX_DIM - 3; t >= 1; --t) {
                        if (t <= a.d - 3 && carry) {
                            if (++dg[t] == a.n1) dg[t] = 0;
                            else carry = false;
                        }
                    }
                    if (carry) ++dg[0];
                }
                return moved;
            };
            if (a.d >= 3) {
                int Q = (grp * kKS) / a.n1;
                kl = grp * kKS - Q * a.n1;
#pragma unroll
                for (int t = RBF_MAX_DIM - 3; t >= 1; --t) {
                    if (t <= a.d - 3) {
                        dg[t] = Q % a.n1;
                        Q /= a.n1;
                    }
                }
                dg[0] = Q;
                if (grp * kKS < a.nrow) pf = prefix_from_digits();
            }
            for (int lc = grp; lc < nch; lc += kGroups) {
                const int gcc = gc + lc;
                const int s = gcc % S, k = gcc % kRingL;
                if (gcc >= S && !*y.abort) (void)wait_or_abort(&y.empty[s], ((gcc - S) / S) & 1, y.abort);
                unsigned char *tile = smem + s * sbytes;
                const bool ready = !*y.abort && wait_or_abort(&y.rfull[k], (uint32_t)(gcc / kRingL) & 1u, y.abort);
                if (ready)
                    for (int idx = gt; idx < 4 * NT; idx += 128) {
                        const int jw = idx >> 2, qw = (idx >> 1) & 1, hw = idx & 1;
                        const int rlw = jw / a.ncol, colw = jw - rlw * a.ncol;
                        float wr[4] = {0, 0, 0, 0}, wi[4] = {0, 0, 0, 0};
                        if (jw < ncolt && rlw < rgv) {
                            const float2 *sl = ring + k * slot_c + rlw * kKS * a.ncol + colw;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int rr = 4 * qw + e;
                                if (lc * kKS + rr < a.nrow) {
                                    const float2 v = sl[rr * a.ncol];
                                    wr[e] = v.x;
                                    wi[e] = v.y;
                                }
                            }
                        }
                        put_w_half(tile + kABytes, jw, NT, qw, hw, wr, wi);
                    }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&y.rempty[k]));
                if (!*y.abort) {
#pragma unroll
                    for (int qa = 0; qa < 2; ++qa) {
                        float re[4], im[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int rw = lc * kKS + 4 * qa + e;
                            float2 v = make_float2(0.0f, 0.0f);
                            if (rw < a.nrow) {
                                if (a.d >= 3) {
                                    v = cmul(pf, Elast[kl]);
                                    if (advance(1) && rw + 1 < a.nrow) pf = prefix_from_digits();
                                } else if (a.d == 2) {
                                    v = Ep[rw];
                                } else {
                                    v = make_float2(1.0f, 0.0f);
                                }
                            }
                            re[e] = v.x;
                            im[e] = v.y;
                        }
                        put_a(tile, gt, qa, re, im);
                    }
                    fence_async_smem();
                }
                // skip the other groups' stages
                if (a.d >= 3 && advance((kGroups - 1) * kKS) && (lc + kGroups) * kKS < a.nrow)
                    pf = prefix_from_digits();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&y.full[s]));
            }
            gc += nch;
        } else if (warp == kMmaWarp) {
            if (lane == 0) mma_item<S>(y, nch, gc, gb, last, smem, sbytes, tmem, a.idesc, NT);
        } else if (warp == kCopyWarp) {
            // ---- copies: one bulk copy per right-hand side and stage (16-byte
            // multiple; the allocation of L carries a 64-byte tail for the round-up)
            if (lane == 0) {
                for (int lc = 0; lc < nch; ++lc, ++gc) {
                    const int k = gc % kRingL;
                    if (*y.abort) continue;
                    if (gc >= kRingL &&
                        !wait_or_abort(&y.rempty[k], (uint32_t)((gc - kRingL) / kRingL) & 1u, y.abort))
                        continue;
                    const int rows = min(kKS, a.nrow - lc * kKS);
                    const uint32_t bytes = ((uint32_t)(rows * a.ncol) * 8u + 15u) & ~15u;
                    const uint32_t fb = smem_u32(&y.rfull[k]);
                    mbar_expect_tx(fb, bytes * (uint32_t)rgv);
                    for (int r = 0; r < rgv; ++r) {
                        const float2 *src = a.L + (int64_t)(rg0 + r) * a.vstride +
                                            (int64_t)leaf * a.mstride + (int64_t)lc * kKS * a.ncol;
                        bulk_g2s(smem_u32(ring + k * slot_c + r * kKS * a.ncol), src, bytes, fb);
                    }
                    issued = gc + 1;
                }
            }
        } else {
            // ---- epilogue
            const int ew = warp - kEpiWarp0, q = warp & 3, h = ew >> 2;
            const int i = 32 * q + lane;
            const uint32_t tlane = tmem + ((uint32_t)(32 * q) << 16);
            float acc_re[NH], acc_im[NH];
            epi_item<NTH>(y, nch, gb, tlane, h, acc_re, acc_im);
            // S_i[h][r] = sum over this half's columns of r of Re(B'_i[col] T_i[col, r])
            const int ocol = a.d == 1 ? 0 : a.n0 + (a.d - 2) * a.n1;
            float *Si = Sg + (i * 2 + h) * Rg;
            for (int r = 0; r < Rg; ++r) Si[r] = 0.0f;
            if (!*y.abort && i < cnt) {
                const float2 *B = Eg + (p0 + pt0 + i) * rowpadE + ocol;   // conj gives B'
                int j = h * NH, rl = j / a.ncol, col = j - rl * a.ncol;
#pragma unroll
                for (int jj = 0; jj < NH; ++jj, ++j) {
                    if (j < ncolt) {
                        const float2 bb = B[col];   // B' = (bb.x, -bb.y)
                        Si[rl] += fmaf(bb.x, acc_re[jj], bb.y * acc_im[jj]);
                    }
                    if (++col == a.ncol) {
                        col = 0;
                        ++rl;
                    }
                }
            }
            named_bar(kBarEpi, 32 * kEpiWarps);
            if (!*y.abort) {
                const int et = tid - 32 * kEpiWarp0;
                for (int idx = et; idx < kRows * rgv; idx += 32 * kEpiWarps) {
                    const int pi = idx % kRows, rl = idx / kRows;
                    if (pi < cnt)
                        a.u[(int64_t)(rg0 + rl) * a.N + p0 + pt0 + pi] =
                            Sg[(pi * 2) * Rg + rl] + Sg[(pi * 2 + 1) * Rg + rl];
                }
            }
            named_bar(kBarEpi, 32 * kEpiWarps);
        }
    }
    if (*y.abort) {   // bounded waits for the MMAs and copies still in flight
        if (warp == kMmaWarp && lane == 0 && last >= 0)
            wait_bounded(&y.empty[last % S], (uint32_t)(last / S) & 1u);
        if (warp == kCopyWarp && lane == 0)
            for (int c2 = max(0, issued - kRingL); c2 < issued; ++c2)
                wait_bounded(&y.rfull[c2 % kRingL], (uint32_t)(c2 / kRingL) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tcols);
    }
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
size_t stage_bytes(int NT, int S) { return (size_t)S * ((size_t)kABytes + (size_t)2 * NT * kKStage * 4); }
inline int rowpad_even(const rbf_tree *t, const rbf_plan *p)
{
    const int rowlen = t->d == 1 ? p->n0 : p->n0 + (t->d - 1) * p->n1;
    return (rowlen + 1) & ~1;
}

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
    const int gpad = 16;   // coefficient columns of the point-major copy
    *smem = stage_bytes(16 * best_c, kP2MStages) +
            (size_t)kRingE * kKS * (rowpad_even(t, p) * sizeof(float2) + gpad * sizeof(float)) +
            (size_t)2 * kGroups * kKS * kPF * sizeof(float2) + (size_t)2 * kPF * RBF_MAX_DIM * sizeof(int) +
            kSyncBytes;
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
    *smem = stage_bytes(16 * *nth, kL2PStages) + (size_t)kRingL * Rg * kKS * p->ncol * sizeof(float2) +
            (size_t)kRows * (rowlen | 1) * sizeof(float2) + (size_t)kRows * 2 * Rg * sizeof(float) +
            kSyncBytes;
}

int num_sms()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

template <int NTH>
int launch_p2m(const TcArgs &a, const float2 *Eg, const float *Lt, int rowpadE, int gpad,
               int ntile1, int ntile2, int nitems, size_t smem, cudaStream_t s)
{
    RBF_CUDA_TRY(cudaFuncSetAttribute(k_p2m_tc<NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    const int grid = std::min(nitems, num_sms());
    k_p2m_tc<NTH><<<grid, kTcThreads, smem, s>>>(a, Eg, Lt, rowpadE, gpad, ntile1, ntile2, nitems);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

template <int NTH>
int launch_l2p(const TcArgs &a, const float2 *Eg, int rowpadE, int Rg, int nptile, int nrt,
               int nitems, size_t smem, cudaStream_t s)
{
    RBF_CUDA_TRY(cudaFuncSetAttribute(k_l2p_tc<NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    const int grid = std::min(nitems, num_sms());
    k_l2p_tc<NTH><<<grid, kTcThreads, smem, s>>>(a, Eg, rowpadE, Rg, nptile, nrt, nitems);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

}  // namespace

int rbf_far_multi_supported(const rbf_plan *p)
{
    return p->M > 0 && p->ncol <= kMaxNT && p->grid == RBF_GRID_SHARED;
}

int rbf_run_far_multi(rbf_tree *t, rbf_plan *p, const float *lam_s, int G, float2 *V, float2 *L,
                      float *u_far, cudaStream_t s)
{
    RBF_REQUIRE(G >= 1 && G <= 16 && p->ncol <= kMaxNT, "rbf_run_far_multi: G=%d, %d columns", G,
                p->ncol);
    const int nleaf = t->nleaf();
    const int64_t vstride = (int64_t)nleaf * p->mstride;
    // The tensor-core contractions pay off when a leaf fills the K dimension
    // (P2M: points) or the M dimension (L2P: points per 128-row tile); with
    // fewer points per leaf the CUDA-core kernels run column by column.
    const double per_leaf = (double)t->N / std::max(1, nleaf);
    int nth_p = 0, nth_l = 0, Rg = 0;
    size_t smem_p = 0, smem_l = 0;
    p2m_shape(t, p, G, &nth_p, &smem_p);
    l2p_shape(t, p, G, &Rg, &nth_l, &smem_l);
    const bool tc_p2m = per_leaf >= RBF_TC_P2M_MIN && smem_p <= kSmemMax;
    const bool tc_l2p = per_leaf >= RBF_TC_L2P_MIN && smem_l <= kSmemMax;
    const int rowpadE = rowpad_even(t, p);
    const int gpad = 16;   // coefficient rows of the point-major copy (G <= 16)
    if (tc_p2m || tc_l2p) {
        if (!p->mr_E) RBF_TRY(rbf_alloc(&p->mr_E, (size_t)t->N * rowpadE));
        if (tc_p2m && !p->mr_Lt) RBF_TRY(rbf_alloc(&p->mr_Lt, (size_t)t->N * gpad));
        TcArgs a = base_args(t, p, G);
        a.lam = lam_s;
        k_point_tables<<<nleaf, 256, 0, s>>>(a, rowpadE, p->mr_E, gpad, tc_p2m ? p->mr_Lt : nullptr);
        RBF_LAUNCH_CHECK();
    }
    if (tc_p2m) {
        TcArgs a = base_args(t, p, G);
        a.V = V;
        a.NT = 16 * nth_p;
        a.idesc = instr_desc_tf32(kRows, 2 * a.NT);
        a.tcols = tmem_cols(4 * a.NT);
        const int ntile1 = ceil_div(p->nrow, kRows), ntile2 = ceil_div((int64_t)p->ncol * G, a.NT);
        const int64_t nitems = (int64_t)nleaf * ntile1 * ntile2;
        RBF_REQUIRE(nitems < INT32_MAX, "rbf_run_far_multi: too many tiles");
        rbf_pass_timer tm(t, RBF_PASS_P2M, s);
        switch (nth_p) {
        case 1: RBF_TRY(launch_p2m<1>(a, p->mr_E, p->mr_Lt, rowpadE, gpad, ntile1, ntile2, (int)nitems, smem_p, s)); break;
        case 2: RBF_TRY(launch_p2m<2>(a, p->mr_E, p->mr_Lt, rowpadE, gpad, ntile1, ntile2, (int)nitems, smem_p, s)); break;
        case 3: RBF_TRY(launch_p2m<3>(a, p->mr_E, p->mr_Lt, rowpadE, gpad, ntile1, ntile2, (int)nitems, smem_p, s)); break;
        default: RBF_TRY(launch_p2m<4>(a, p->mr_E, p->mr_Lt, rowpadE, gpad, ntile1, ntile2, (int)nitems, smem_p, s)); break;
        }
    } else {
        for (int g = 0; g < G; ++g)
            RBF_TRY(rbf_run_p2m<float>(t, p, lam_s + g * t->N, V + g * vstride, s));
    }
    for (int g = 0; g < G; ++g) {
        RBF_TRY(rbf_run_m2m<float>(t, p, V + g * vstride, s));
        RBF_TRY(rbf_run_m2l<float>(t, p, V + g * vstride, L + g * vstride, s));
    }
    if (tc_l2p) {
        TcArgs a = base_args(t, p, G);
        a.L = L;
        a.u = u_far;
        a.NT = 16 * nth_l;
        a.idesc = instr_desc_tf32(kRows, 2 * a.NT);
        a.tcols = tmem_cols(4 * a.NT);
        const int nrt = (G + Rg - 1) / Rg;
        const int nptile = ceil_div(std::max<int>(t->max_leaf, 1), kRows);
        const int64_t nitems = (int64_t)nleaf * nptile * nrt;
        RBF_REQUIRE(nitems < INT32_MAX, "rbf_run_far_multi: too many tiles");
        rbf_pass_timer tm(t, RBF_PASS_L2P, s);
        switch (nth_l) {
        case 1: RBF_TRY(launch_l2p<1>(a, p->mr_E, rowpadE, Rg, nptile, nrt, (int)nitems, smem_l, s)); break;
        case 2: RBF_TRY(launch_l2p<2>(a, p->mr_E, rowpadE, Rg, nptile, nrt, (int)nitems, smem_l, s)); break;
        case 3: RBF_TRY(launch_l2p<3>(a, p->mr_E, rowpadE, Rg, nptile, nrt, (int)nitems, smem_l, s)); break;
        default: RBF_TRY(launch_l2p<4>(a, p->mr_E, rowpadE, Rg, nptile, nrt, (int)nitems, smem_l, s)); break;
        }
    } else {
        for (int g = 0; g < G; ++g)
            RBF_TRY(rbf_run_l2p<float>(t, p, L + g * vstride, u_far + g * t->N, s));
    }
    return RBF_OK;
}

namespace {
// Failure-path self test: one thread waits, with the try-wait loop of the
// tensor-core kernels and a limit of limit_cycles, on an mbarrier that nothing
// arrives on; the wait gives up, sets status bit 2 and the kernel returns.
__global__ void k_wait_selftest(long long limit_cycles, int *gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const long long t0 = clock64();
    int g = 0;
    while (!mbar_try_wait(b, 0)) {
        if (clock64() - t0 > limit_cycles) {
            atomicOr(&g_tc_status, 2u);
            g = 1;
            break;
        }
        __nanosleep(kBackoffNs);
    }
    *gave_up = g;
}
}  // namespace

extern "C" int rbf_selftest_bounded_wait(double seconds, int *gave_up_host, void *stream)
{
    RBF_REQUIRE(gave_up_host && seconds > 0.0 && seconds <= 2.0,
                "rbf_selftest_bounded_wait: seconds must be in (0, 2]");
    int khz = 0, dev = 0;
    RBF_CUDA_TRY(cudaGetDevice(&dev));
    RBF_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long limit = (long long)(seconds * (double)khz * 1e3);
    int *flag = nullptr;
    RBF_TRY(rbf_alloc(&flag, 1));
    cudaStream_t s = (cudaStream_t)stream;
    k_wait_selftest<<<1, 32, 0, s>>>(limit, flag);
    int h = 0;
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                    cudaStreamSynchronize(s) == cudaSuccess;
    rbf_free(flag);
    if (!ok) {
        rbf_set_error("rbf_selftest_bounded_wait: CUDA failure");
        return RBF_ECUDA;
    }
    *gave_up_host = h;
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
