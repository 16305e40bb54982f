// tree.cu -- Morton tree on the device: box keys, stable LSD radix sort,
// leaf and level structure, near lists N_a (Eq. (38)) and interaction lists
// IL_l (Sec. 4.1 coupling).  Every list is produced in ascending Morton order
// so that it is bit-exact with a plain sequential construction.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "rbf_internal.cuh"

namespace {

// ----------------------------------------------------------- utilities ----
__device__ __forceinline__ uint64_t morton_encode(const int64_t *k, int d, int l)
{
    uint64_t key = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) key |= (uint64_t)((k[t] >> b) & 1) << (b * d + t);
    return key;
}

__host__ __device__ __forceinline__ void morton_decode(uint64_t key, int d, int l, int64_t *k)
{
    for (int t = 0; t < d; ++t) k[t] = 0;
    for (int b = 0; b < l; ++b)
        for (int t = 0; t < d; ++t) k[t] |= (int64_t)((key >> (b * d + t)) & 1u) << b;
}

// index of `key` in ascending keys[0..n), or -1
__device__ __forceinline__ int32_t find_key(const uint64_t *keys, int32_t n, uint64_t key)
{
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

// ---------------------------------------------------------------- keys ----
// k_t = min(max(floor(((x_t - lo_t)/side) * 2^D), 0), 2^D - 1) in IEEE FP64
// (explicit round-to-nearest intrinsics: no contraction into FMA).
// Morton key of point i: box coordinates floor((x - lo) / side * 2^D) in FP64,
// clamped to [0, 2^D - 1] (points on the upper face go to the last box).
__device__ __forceinline__ uint64_t point_key(const double *X, int64_t i, int d, int D,
                                              const double *lo, double side)
{
    int64_t k[RBF_MAX_DIM];
    double scale = (double)((int64_t)1 << D);
    int64_t kmax = ((int64_t)1 << D) - 1;
    for (int t = 0; t < d; ++t) {
        double v = __dmul_rn(__ddiv_rn(__dsub_rn(X[i * d + t], lo[t]), side), scale);
        double f = floor(v);
        int64_t q;
        if (!(f >= 0.0)) q = 0;  // also catches NaN
        else if (f >= (double)kmax) q = kmax;
        else q = (int64_t)f;
        k[t] = q;
    }
    return morton_encode(k, d, D);
}

__global__ void k_keys(const double *X, int64_t N, int d, int D, const double *lo, double side,
                       uint64_t *keys, int32_t *idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    keys[i] = point_key(X, i, d, D, lo, side);
    idx[i] = (int32_t)i;
}

// The root cube's lower corner passed by value (kernel parameter space), for
// callers that hold it only in host memory.
struct corner_t {
    double v[RBF_MAX_DIM];
};

__global__ void k_keys_corner(const double *X, int64_t N, int d, int D, corner_t lo, double side,
                              uint64_t *keys, int32_t *idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    keys[i] = point_key(X, i, d, D, lo.v, side);
    idx[i] = (int32_t)i;
}

// ---------------------------------------------------------------- scan ----
constexpr int SCAN_BS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_BS * SCAN_IPT;

__global__ void k_scan_tile(const int32_t *in, int32_t *out, int64_t n, int32_t *bsum)
{
    __shared__ int32_t wtot[SCAN_BS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    int32_t v[SCAN_IPT];
    int32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        tsum += v[k];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t tt = lane < SCAN_BS / 32 ? wtot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, tt, o);
            if (lane >= o) tt += y;
        }
        if (lane < SCAN_BS / 32) wtot[lane] = tt;
    }
    __syncthreads();
    int32_t run = x - tsum + (w > 0 ? wtot[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_BS - 1 && bsum) bsum[blockIdx.x] = run;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *boff)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[i / SCAN_TILE];
}

__global__ void k_sum_last(const int32_t *in, const int32_t *ex, int64_t n, int32_t *total)
{
    *total = ex[n - 1] + in[n - 1];
}

// ---------------------------------------------------------- radix sort ----
constexpr int RS_BS = 256;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_BS * RS_IPT;
constexpr int RS_WARPS = RS_BS / 32;

__global__ void k_rs_hist(const uint64_t *keys, int64_t n, int shift, int32_t *hist, int nblk)
{
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_IPT; ++r) {
        int64_t i = base + (int64_t)r * RS_BS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: the rank of an item among equal digits of its tile counts
// earlier rounds, earlier warps of this round and lower lanes of its warp.
__global__ void k_rs_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout,
                             int32_t *vout, int64_t n, int shift, const int32_t *offs, int nblk)
{
    __shared__ int32_t base_off[256];
    __shared__ int32_t running[256];
    __shared__ int32_t wcnt[RS_WARPS][256];
    __shared__ int32_t wpre[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base_off[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
    running[tid] = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_IPT; ++r) {
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        int64_t i = tile + (int64_t)r * RS_BS + tid;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int32_t val = valid ? vin[i] : 0;
        int digit = (int)((key >> shift) & 255u);
        int tag = valid ? digit : (0x10000 + lane);
        unsigned peers = __match_any_sync(0xffffffffu, tag);
        int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            int32_t run = running[tid];
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                wpre[w][tid] = run;
                run += wcnt[w][tid];
            }
            running[tid] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = (int64_t)base_off[digit] + wpre[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- leaf / levels ----
__global__ void k_diff_flags(const uint64_t *keys, int64_t n, int shift, int32_t *flag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift)) ? 1 : 0;
}

// first element of each run: out_key[id] = keys[i] >> shift, out_off[id] = i;
// owner[i] = id of the run containing i (may be null)
__global__ void k_runs(const uint64_t *keys, int64_t n, int shift, const int32_t *flag,
                       const int32_t *ex, uint64_t *out_key, int32_t *out_off, int32_t *owner)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t id = ex[i] + flag[i] - 1;
    if (flag[i]) {
        out_key[id] = keys[i] >> shift;
        if (out_off) out_off[id] = (int32_t)i;
    }
    if (owner) owner[i] = id;
}

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }

__global__ void k_gather_points(const double *X, const int32_t *perm, int64_t N, int d,
                                double *xs64, float *xs32)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t j = perm[i];
    for (int t = 0; t < d; ++t) {
        double v = X[j * d + t];
        xs64[(int64_t)t * N + i] = v;
        xs32[(int64_t)t * N + i] = (float)v;
    }
}

__global__ void k_max_leaf(const int32_t *off, int32_t n, int32_t *mx)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, off[i + 1] - off[i]);
}

// ------------------------------------------------------------ near lists --
// Leaves b with max_t |k_b,t - k_a,t| <= 1 (self included), ascending key.
template <bool FILL>
__global__ void k_near(const uint64_t *leaf_key, int32_t nleaf, int d, int D, int32_t *cnt,
                       const int32_t *off, int32_t *idx)
{
    int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nleaf) return;
    int64_t ka[RBF_MAX_DIM], kb[RBF_MAX_DIM];
    morton_decode(leaf_key[a], d, D, ka);
    int ncand = 1;
    for (int t = 0; t < d; ++t) ncand *= 3;
    const int64_t kmax = ((int64_t)1 << D) - 1;
    int32_t found = 0;
    int32_t base = FILL ? off[a] : 0;
    for (int c = 0; c < ncand; ++c) {
        int cc = c;
        bool inside = true;
        for (int t = 0; t < d; ++t) {
            kb[t] = ka[t] + (cc % 3) - 1;
            cc /= 3;
            inside = inside && kb[t] >= 0 && kb[t] <= kmax;
        }
        if (!inside) continue;
        int32_t b = find_key(leaf_key, nleaf, morton_encode(kb, d, D));
        if (b < 0) continue;
        if (FILL) {
            // insertion into the ascending list written so far
            int32_t pos = base + found;
            while (pos > base && idx[pos - 1] > b) {
                idx[pos] = idx[pos - 1];
                --pos;
            }
            idx[pos] = b;
        }
        ++found;
    }
    if (!FILL) cnt[a] = found;
}

// ----------------------------------------------------- interaction lists --
// IL_l(a): children of the parent's neighbours (Chebyshev <= 1 at level l-1)
// that are at Chebyshev distance >= 2 from a.  Parents are visited in
// ascending key and children in ascending child bits, so the output is in
// ascending level-l Morton order without a sort.
template <bool FILL>
__global__ void k_il(const uint64_t *key_l, int32_t n_l, const uint64_t *key_p, int32_t n_p,
                     int d, int l, int32_t *cnt, const int32_t *off, int32_t *idx)
{
    int32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_l) return;
    int64_t ka[RBF_MAX_DIM], kp[RBF_MAX_DIM], kc[RBF_MAX_DIM];
    morton_decode(key_l[a], d, l, ka);
    int ncand = 1;
    for (int t = 0; t < d; ++t) ncand *= 3;
    const int64_t pmax = ((int64_t)1 << (l - 1)) - 1;
    // existing parent neighbours, ascending key (insertion sort, <= 3^d)
    uint64_t pkeys[729];
    int np = 0;
    for (int c = 0; c < ncand; ++c) {
        int cc = c;
        bool inside = true;
        for (int t = 0; t < d; ++t) {
            kp[t] = (ka[t] >> 1) + (cc % 3) - 1;
            cc /= 3;
            inside = inside && kp[t] >= 0 && kp[t] <= pmax;
        }
        if (!inside) continue;
        uint64_t pk = morton_encode(kp, d, l - 1);
        if (find_key(key_p, n_p, pk) < 0) continue;
        int pos = np++;
        while (pos > 0 && pkeys[pos - 1] > pk) {
            pkeys[pos] = pkeys[pos - 1];
            --pos;
        }
        pkeys[pos] = pk;
    }
    int32_t found = 0;
    int32_t base = FILL ? off[a] : 0;
    const int nchild = 1 << d;
    for (int q = 0; q < np; ++q) {
        morton_decode(pkeys[q], d, l - 1, kp);
        for (int ch = 0; ch < nchild; ++ch) {
            int64_t cheb = 0;
            for (int t = 0; t < d; ++t) {
                kc[t] = 2 * kp[t] + ((ch >> t) & 1);
                int64_t df = kc[t] > ka[t] ? kc[t] - ka[t] : ka[t] - kc[t];
                cheb = df > cheb ? df : cheb;
            }
            if (cheb < 2) continue;
            int32_t b = find_key(key_l, n_l, (pkeys[q] << d) | (uint64_t)ch);
            if (b < 0) continue;
            if (FILL) idx[base + found] = b;
            ++found;
        }
    }
    if (!FILL) cnt[a] = found;
}

__global__ void k_i32_to_i64(const int32_t *in, int64_t *out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

// 4^d block of leaves around each level-(D-1) box P: block coordinate i_t
// covers leaf coordinate 2 P_t - 1 + i_t; -1 marks an empty or outside leaf.
__global__ void k_nb4(const uint64_t *pkey, int32_t np, const uint64_t *leaf_key, int32_t nleaf,
                      int d, int D, int32_t *nb4)
{
    int nb = 1;
    for (int t = 0; t < d; ++t) nb *= 4;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)np * nb) return;
    int32_t p = (int32_t)(i / nb);
    int pos = (int)(i % nb);
    int64_t kp[RBF_MAX_DIM], kl[RBF_MAX_DIM];
    morton_decode(pkey[p], d, D - 1, kp);
    const int64_t kmax = ((int64_t)1 << D) - 1;
    bool inside = true;
    for (int t = 0; t < d; ++t) {
        kl[t] = 2 * kp[t] - 1 + ((pos >> (2 * t)) & 3);
        inside = inside && kl[t] >= 0 && kl[t] <= kmax;
    }
    nb4[i] = inside ? find_key(leaf_key, nleaf, morton_encode(kl, d, D)) : -1;
}

// pencil neighbourhoods: entry (seg, plane, pos) is the leaf at x = 2X - 1 + (pos & 3),
// y = 2Y - 1 + (pos >> 2), z = Zs RBF_PENCIL_Z - 1 + plane, or -1 (empty or outside)
__global__ void k_pencil_nb(const int4 *seg, int32_t nseg, const uint64_t *leaf_key, int32_t nleaf,
                            int D, int32_t *nb)
{
    constexpr int NP = (RBF_PENCIL_Z + 2) * 16;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nseg * NP) return;
    const int4 sg = seg[i / NP];
    const int e = (int)(i % NP), plane = e / 16, pos = e % 16;
    int64_t k[3] = {2 * (int64_t)sg.x - 1 + (pos & 3), 2 * (int64_t)sg.y - 1 + (pos >> 2),
                    (int64_t)sg.z * RBF_PENCIL_Z - 1 + plane};
    const int64_t kmax = ((int64_t)1 << D) - 1;
    bool inside = true;
    for (int t = 0; t < 3; ++t) inside = inside && k[t] >= 0 && k[t] <= kmax;
    nb[i] = inside ? find_key(leaf_key, nleaf, morton_encode(k, 3, D)) : -1;
}

}  // namespace

// pencils of the 3-D coupling: every (X, Y, Zs) that holds a level-(D-1) box
static int build_pencils(rbf_tree *t, cudaStream_t s)
{
    const int D = t->D;
    const int32_t np = t->lev[D - 1].nbox;
    std::vector<uint64_t> pk(np);
    RBF_CUDA_TRY(cudaMemcpyAsync(pk.data(), t->lev[D - 1].key, np * sizeof(uint64_t),
                                 cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<uint64_t> code(np);
    const int zb = RBF_PENCIL_Z / 2;  // parents per pencil along z
    for (int32_t i = 0; i < np; ++i) {
        int64_t k[3];
        morton_decode(pk[i], 3, D - 1, k);
        code[i] = ((uint64_t)(k[2] / zb) << 42) | ((uint64_t)k[1] << 21) | (uint64_t)k[0];
    }
    std::sort(code.begin(), code.end());
    code.erase(std::unique(code.begin(), code.end()), code.end());
    std::vector<int4> seg(code.size());
    const uint64_t m21 = (1ull << 21) - 1;
    for (size_t i = 0; i < code.size(); ++i)
        seg[i] = make_int4((int)(code[i] & m21), (int)((code[i] >> 21) & m21), (int)(code[i] >> 42), 0);
    t->npz = (int32_t)seg.size();
    const int64_t n = (int64_t)t->npz * (RBF_PENCIL_Z + 2) * 16;
    RBF_TRY(rbf_alloc(&t->pz_seg, seg.size()));
    RBF_TRY(rbf_alloc(&t->pz_nb, n));
    RBF_CUDA_TRY(cudaMemcpyAsync(t->pz_seg, seg.data(), seg.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s));
    k_pencil_nb<<<ceil_div(n, 256), 256, 0, s>>>(t->pz_seg, t->npz, t->lev[D].key, t->nleaf(), D,
                                                 t->pz_nb);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));  // seg goes out of scope
    return RBF_OK;
}

// ----------------------------------------------------------- host side ----
int rbf_scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_host,
                           cudaStream_t s)
{
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return RBF_OK;
    }
    int64_t nblk = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *bsum = nullptr, *boff = nullptr;
    if (nblk > 1) {
        RBF_TRY(rbf_alloc(&bsum, nblk));
        RBF_TRY(rbf_alloc(&boff, nblk));
    }
    k_scan_tile<<<(unsigned)nblk, SCAN_BS, 0, s>>>(in, out, n, bsum);
    RBF_LAUNCH_CHECK();
    if (nblk > 1) {
        RBF_TRY(rbf_scan_exclusive_i32(bsum, boff, nblk, nullptr, s));
        k_scan_add<<<ceil_div(n, 256), 256, 0, s>>>(out, n, boff);
        RBF_LAUNCH_CHECK();
    }
    if (total_host) {
        int32_t *tot = nullptr;
        RBF_TRY(rbf_alloc(&tot, 1));
        k_sum_last<<<1, 1, 0, s>>>(in, out, n, tot);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaMemcpyAsync(total_host, tot, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        rbf_free(tot);
    }
    if (nblk > 1) {
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        rbf_free(bsum);
        rbf_free(boff);
    }
    return RBF_OK;
}

int rbf_radix_sort_pairs(uint64_t *keys, int32_t *vals, int64_t n, int nbits, cudaStream_t s)
{
    if (nbits <= 0 || n <= 1) return RBF_OK;
    int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    uint64_t *k2 = nullptr;
    int32_t *v2 = nullptr, *hist = nullptr, *offs = nullptr;
    RBF_TRY(rbf_alloc(&k2, n));
    RBF_TRY(rbf_alloc(&v2, n));
    RBF_TRY(rbf_alloc(&hist, (size_t)256 * nblk));
    RBF_TRY(rbf_alloc(&offs, (size_t)256 * nblk));
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = (nbits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<nblk, RS_BS, 0, s>>>(ka, n, shift, hist, nblk);
        RBF_LAUNCH_CHECK();
        RBF_TRY(rbf_scan_exclusive_i32(hist, offs, (int64_t)256 * nblk, nullptr, s));
        k_rs_scatter<<<nblk, RS_BS, 0, s>>>(ka, va, kb, vb, n, shift, offs, nblk);
        RBF_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        RBF_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        RBF_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(k2);
    rbf_free(v2);
    rbf_free(hist);
    rbf_free(offs);
    return RBF_OK;
}

// Compact the runs of (keys >> shift) in an ascending key array.
static int compact_runs(const uint64_t *keys, int64_t n, int shift, uint64_t **out_key,
                        int32_t **out_off, int32_t *owner, int32_t *nrun, cudaStream_t s)
{
    int32_t *flag = nullptr, *ex = nullptr;
    RBF_TRY(rbf_alloc(&flag, n));
    RBF_TRY(rbf_alloc(&ex, n));
    k_diff_flags<<<ceil_div(n, 256), 256, 0, s>>>(keys, n, shift, flag);
    RBF_LAUNCH_CHECK();
    RBF_TRY(rbf_scan_exclusive_i32(flag, ex, n, nrun, s));
    RBF_TRY(rbf_alloc(out_key, (size_t)*nrun));
    if (out_off) RBF_TRY(rbf_alloc(out_off, (size_t)*nrun + 1));
    k_runs<<<ceil_div(n, 256), 256, 0, s>>>(keys, n, shift, flag, ex, *out_key,
                                            out_off ? *out_off : nullptr, owner);
    RBF_LAUNCH_CHECK();
    if (out_off) {
        k_set_i32<<<1, 1, 0, s>>>(*out_off + *nrun, (int32_t)n);
        RBF_LAUNCH_CHECK();
    }
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(flag);
    rbf_free(ex);
    return RBF_OK;
}

static int build_impl(rbf_tree *t, const double *X, cudaStream_t s)
{
    const int64_t N = t->N;
    const int d = t->d, D = t->D;
    double *lo_d = nullptr;
    RBF_TRY(rbf_alloc(&lo_d, d));
    RBF_CUDA_TRY(cudaMemcpyAsync(lo_d, t->lo, d * sizeof(double), cudaMemcpyHostToDevice, s));
    RBF_TRY(rbf_alloc(&t->keys, N));
    RBF_TRY(rbf_alloc(&t->perm, N));
    k_keys<<<ceil_div(N, 256), 256, 0, s>>>(X, N, d, D, lo_d, t->side, t->keys, t->perm);
    RBF_LAUNCH_CHECK();
    RBF_TRY(rbf_radix_sort_pairs(t->keys, t->perm, N, d * D, s));
    rbf_free(lo_d);

    RBF_TRY(rbf_alloc(&t->xs64, (size_t)N * d));
    RBF_TRY(rbf_alloc(&t->xs32, (size_t)N * d));
    k_gather_points<<<ceil_div(N, 256), 256, 0, s>>>(X, t->perm, N, d, t->xs64, t->xs32);
    RBF_LAUNCH_CHECK();

    // leaves = runs of equal keys
    int32_t nleaf = 0;
    RBF_TRY(compact_runs(t->keys, N, 0, &t->lev[D].key, &t->leaf_off, nullptr, &nleaf, s));
    t->lev[D].nbox = nleaf;
    {
        int32_t *mx = nullptr;
        RBF_TRY(rbf_alloc(&mx, 1));
        RBF_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(int32_t), s));
        k_max_leaf<<<ceil_div(nleaf, 256), 256, 0, s>>>(t->leaf_off, nleaf, mx);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaMemcpyAsync(&t->max_leaf, mx, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        rbf_free(mx);
    }
    // coarser levels: runs of key >> d over the finer level's boxes
    for (int l = D - 1; l >= 0; --l) {
        rbf_level &fine = t->lev[l + 1], &coarse = t->lev[l];
        RBF_TRY(rbf_alloc(&fine.parent, fine.nbox));
        int32_t nb = 0;
        RBF_TRY(compact_runs(fine.key, fine.nbox, d, &coarse.key, &coarse.child_off, fine.parent,
                             &nb, s));
        coarse.nbox = nb;
    }
    // near lists
    int32_t *cnt = nullptr;
    RBF_TRY(rbf_alloc(&cnt, nleaf));
    RBF_TRY(rbf_alloc(&t->near_off, (size_t)nleaf + 1));
    k_near<false><<<ceil_div(nleaf, 128), 128, 0, s>>>(t->lev[D].key, nleaf, d, D, cnt, nullptr,
                                                      nullptr);
    RBF_LAUNCH_CHECK();
    int32_t total = 0;
    RBF_TRY(rbf_scan_exclusive_i32(cnt, t->near_off, nleaf, &total, s));
    k_set_i32<<<1, 1, 0, s>>>(t->near_off + nleaf, total);
    RBF_LAUNCH_CHECK();
    t->n_near = total;
    RBF_TRY(rbf_alloc(&t->near_idx, (size_t)std::max(total, 1)));
    k_near<true><<<ceil_div(nleaf, 128), 128, 0, s>>>(t->lev[D].key, nleaf, d, D, nullptr,
                                                     t->near_off, t->near_idx);
    RBF_LAUNCH_CHECK();
    if (D >= 2 && d <= 3) {
        const int32_t np = t->lev[D - 1].nbox;
        const int64_t n = (int64_t)np << (2 * d);
        RBF_TRY(rbf_alloc(&t->nb4, n));
        k_nb4<<<ceil_div(n, 256), 256, 0, s>>>(t->lev[D - 1].key, np, t->lev[D].key, nleaf, d, D,
                                              t->nb4);
        RBF_LAUNCH_CHECK();
    }
    if (d == 3 && D >= 3 && ((int64_t)1 << D) % RBF_PENCIL_Z == 0) RBF_TRY(build_pencils(t, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(cnt);
    return RBF_OK;
}

int rbf_build_il(rbf_tree *t, int level, cudaStream_t s)
{
    rbf_level &lv = t->lev[level];
    if (lv.n_il >= 0) return RBF_OK;
    int32_t *cnt = nullptr;
    RBF_TRY(rbf_alloc(&cnt, std::max(lv.nbox, 1)));
    RBF_TRY(rbf_alloc(&lv.il_off, (size_t)lv.nbox + 1));
    const rbf_level &par = t->lev[level - 1];
    k_il<false><<<ceil_div(lv.nbox, 64), 64, 0, s>>>(lv.key, lv.nbox, par.key, par.nbox, t->d,
                                                    level, cnt, nullptr, nullptr);
    RBF_LAUNCH_CHECK();
    int32_t total = 0;
    RBF_TRY(rbf_scan_exclusive_i32(cnt, lv.il_off, lv.nbox, &total, s));
    k_set_i32<<<1, 1, 0, s>>>(lv.il_off + lv.nbox, total);
    RBF_LAUNCH_CHECK();
    RBF_TRY(rbf_alloc(&lv.il_idx, (size_t)std::max(total, 1)));
    k_il<true><<<ceil_div(lv.nbox, 64), 64, 0, s>>>(lv.key, lv.nbox, par.key, par.nbox, t->d,
                                                   level, nullptr, lv.il_off, lv.il_idx);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(cnt);
    lv.n_il = total;
    return RBF_OK;
}

// bounding box of X, on the host after one device->host copy
static int auto_box(const double *X, int64_t N, int d, double *lo, double *side, cudaStream_t s)
{
    std::vector<double> h((size_t)N * d);
    RBF_CUDA_TRY(cudaMemcpyAsync(h.data(), X, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    double hi[RBF_MAX_DIM];
    for (int t = 0; t < d; ++t) lo[t] = hi[t] = h[t];
    for (int64_t i = 0; i < N; ++i)
        for (int t = 0; t < d; ++t) {
            double v = h[(size_t)i * d + t];
            RBF_REQUIRE(v == v, "rbf_tree_build: NaN coordinate at point %lld", (long long)i);
            lo[t] = std::min(lo[t], v);
            hi[t] = std::max(hi[t], v);
        }
    double ext = 0.0;
    for (int t = 0; t < d; ++t) ext = std::max(ext, hi[t] - lo[t]);
    *side = ext > 0.0 ? ext : 1.0;
    return RBF_OK;
}

extern "C" int rbf_tree_build(const double *X, int64_t N, int d, const double *lo_host, double side,
                              int depth, void *stream, rbf_tree **out)
{
    RBF_REQUIRE(out != nullptr, "rbf_tree_build: out is NULL");
    *out = nullptr;
    RBF_REQUIRE(X != nullptr, "rbf_tree_build: X is NULL");
    RBF_REQUIRE(N >= 1 && N < ((int64_t)1 << 31), "rbf_tree_build: N=%lld out of range",
                (long long)N);
    RBF_REQUIRE(d >= 1 && d <= RBF_MAX_DIM, "rbf_tree_build: d=%d out of range", d);
    cudaStream_t s = (cudaStream_t)stream;
    rbf_tree *t = new rbf_tree();
    t->N = N;
    t->d = d;
    int st = RBF_OK;
    if (lo_host) {
        if (!(side > 0.0)) {
            delete t;
            RBF_REQUIRE(false, "rbf_tree_build: side must be > 0");
        }
        for (int q = 0; q < d; ++q) t->lo[q] = lo_host[q];
        t->side = side;
    } else {
        st = auto_box(X, N, d, t->lo, &t->side, s);
        if (st != RBF_OK) {
            delete t;
            return st;
        }
    }
    if (depth < 0) {
        double lv = std::log((double)N / 32.0) / std::log((double)(1 << d));
        depth = (int)std::lround(lv);
        depth = std::max(2, std::min(depth, RBF_MAX_DEPTH));
        while (depth > 0 && d * depth > 63) --depth;
    }
    if (depth > RBF_MAX_DEPTH || d * depth > 63) {
        delete t;
        RBF_REQUIRE(false, "rbf_tree_build: depth=%d too large for d=%d", depth, d);
    }
    t->D = depth;
    st = build_impl(t, X, s);
    if (st != RBF_OK) {
        rbf_tree_free(t);
        return st;
    }
    *out = t;
    return RBF_OK;
}

extern "C" int rbf_tree_get_info(const rbf_tree *t, rbf_tree_info *info)
{
    RBF_REQUIRE(t && info, "rbf_tree_get_info: NULL argument");
    info->N = t->N;
    info->d = t->d;
    info->depth = t->D;
    for (int q = 0; q < RBF_MAX_DIM; ++q) info->lo[q] = q < t->d ? t->lo[q] : 0.0;
    info->side = t->side;
    info->n_leaf = t->lev[t->D].nbox;
    info->n_near = t->n_near;
    info->max_leaf_points = t->max_leaf;
    for (int l = 0; l <= RBF_MAX_DEPTH; ++l) info->n_box[l] = l <= t->D ? t->lev[l].nbox : 0;
    return RBF_OK;
}

static int copy_i32_as_i64(const int32_t *src, int64_t n, int64_t *dst_host, cudaStream_t s)
{
    if (!dst_host || n <= 0) return RBF_OK;
    int64_t *tmp = nullptr;
    RBF_TRY(rbf_alloc(&tmp, n));
    k_i32_to_i64<<<ceil_div(n, 256), 256, 0, s>>>(src, tmp, n);
    RBF_LAUNCH_CHECK();
    RBF_CUDA_TRY(cudaMemcpyAsync(dst_host, tmp, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    rbf_free(tmp);
    return RBF_OK;
}

extern "C" int rbf_tree_export(const rbf_tree *t, int64_t *perm, uint64_t *keys, uint64_t *leaf_key,
                               int64_t *leaf_off, int64_t *near_off, int64_t *near_idx, void *stream)
{
    RBF_REQUIRE(t != nullptr, "rbf_tree_export: tree is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t nleaf = t->nleaf();
    RBF_TRY(copy_i32_as_i64(t->perm, t->N, perm, s));
    if (keys)
        RBF_CUDA_TRY(cudaMemcpyAsync(keys, t->keys, t->N * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    if (leaf_key)
        RBF_CUDA_TRY(cudaMemcpyAsync(leaf_key, t->leaf_key(), nleaf * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, s));
    RBF_TRY(copy_i32_as_i64(t->leaf_off, (int64_t)nleaf + 1, leaf_off, s));
    RBF_TRY(copy_i32_as_i64(t->near_off, (int64_t)nleaf + 1, near_off, s));
    RBF_TRY(copy_i32_as_i64(t->near_idx, t->n_near, near_idx, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

extern "C" int rbf_tree_export_level(rbf_tree *t, int level, uint64_t *box_key, int64_t *il_off,
                                     int64_t *il_idx, int64_t *n_il_host, void *stream)
{
    RBF_REQUIRE(t != nullptr, "rbf_tree_export_level: tree is NULL");
    RBF_REQUIRE(level >= 2 && level <= t->D, "rbf_tree_export_level: level %d not in [2, %d]",
                level, t->D);
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(rbf_build_il(t, level, s));
    const rbf_level &lv = t->lev[level];
    if (n_il_host) *n_il_host = lv.n_il;
    if (box_key)
        RBF_CUDA_TRY(cudaMemcpyAsync(box_key, lv.key, lv.nbox * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, s));
    RBF_TRY(copy_i32_as_i64(lv.il_off, (int64_t)lv.nbox + 1, il_off, s));
    RBF_TRY(copy_i32_as_i64(lv.il_idx, lv.n_il, il_idx, s));
    RBF_CUDA_TRY(cudaStreamSynchronize(s));
    return RBF_OK;
}

extern "C" void rbf_tree_free(rbf_tree *t)
{
    if (!t) return;
    rbf_prof_release(t);
    rbf_precond_release(t);
    rbf_plan_free(t->plan[0]);
    rbf_plan_free(t->plan[1]);
    rbf_free(t->keys);
    rbf_free(t->perm);
    rbf_free(t->xs64);
    rbf_free(t->xs32);
    rbf_free(t->leaf_off);
    rbf_free(t->near_off);
    rbf_free(t->near_idx);
    rbf_free(t->nb4);
    rbf_free(t->pz_seg);
    rbf_free(t->pz_nb);
    for (int l = 0; l <= RBF_MAX_DEPTH; ++l) {
        rbf_free(t->lev[l].key);
        rbf_free(t->lev[l].parent);
        rbf_free(t->lev[l].child_off);
        rbf_free(t->lev[l].il_off);
        rbf_free(t->lev[l].il_idx);
    }
    rbf_free(t->scratch);
    delete t;
}

// -------------------------------------------------- allocation-free ordering --
// Morton keys and their stable radix sort with every temporary buffer in one
// file-scope device arena instead of cudaMalloc'd memory.  This entry point has
// no counterpart in the paper; it serves callers that must not allocate device
// memory at call time (see include/rbf.h).
namespace {

constexpr int64_t NOALLOC_MAX_N = (int64_t)1 << 22;
constexpr int64_t NOALLOC_MAX_BLK = (NOALLOC_MAX_N + RS_TILE - 1) / RS_TILE;
constexpr int64_t NOALLOC_HIST = 256 * NOALLOC_MAX_BLK;
constexpr int64_t NOALLOC_L1 = (NOALLOC_HIST + SCAN_TILE - 1) / SCAN_TILE;
static_assert(NOALLOC_L1 <= SCAN_TILE, "two scan levels must cover the histogram");

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_VALS = OFF_KEYS + align256(NOALLOC_MAX_N * sizeof(uint64_t));
constexpr size_t OFF_HIST = OFF_VALS + align256(NOALLOC_MAX_N * sizeof(int32_t));
constexpr size_t OFF_OFFS = OFF_HIST + align256(NOALLOC_HIST * sizeof(int32_t));
constexpr size_t OFF_BSUM = OFF_OFFS + align256(NOALLOC_HIST * sizeof(int32_t));
constexpr size_t OFF_BOFF = OFF_BSUM + align256(NOALLOC_L1 * sizeof(int32_t));
constexpr size_t ARENA_BYTES = OFF_BOFF + align256(NOALLOC_L1 * sizeof(int32_t));

// The arena: every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_arena[ARENA_BYTES];

// Driver calls that identify the current context, fetched through the runtime
// so that the library need not link libcuda.
using ctx_get_current_fn = CUresult (*)(CUcontext *);
using ctx_get_id_fn = CUresult (*)(CUcontext, unsigned long long *);

std::mutex g_arena_mu;
struct arena_slot {
    unsigned long long ctx_id = 0;  // 0: not looked up yet (context ids start at 1)
    void *addr = nullptr;
};
arena_slot g_arena_dev[256];

// Id of the context current on this thread (0 if none).
int current_context_id(unsigned long long *id)
{
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        RBF_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                      cudaEnableDefault, &q1));
        RBF_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                      cudaEnableDefault, &q2));
        RBF_REQUIRE(q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 &&
                        f2,
                    "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable");
        get_current = reinterpret_cast<ctx_get_current_fn>(f1);
        get_id = reinterpret_cast<ctx_get_id_fn>(f2);
    }
    CUcontext ctx = nullptr;
    RBF_REQUIRE(get_current(&ctx) == CUDA_SUCCESS, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx) RBF_REQUIRE(get_id(ctx, id) == CUDA_SUCCESS, "cuCtxGetId failed");
    return RBF_OK;
}

// Device address of the arena in the current device's current context.  It is
// looked up (cudaGetSymbolAddress, with that device current) on the first call
// in each context and cached; a new context on the same device (after
// cudaDeviceReset) has a new id and is looked up again.
int arena_address(unsigned char **out)
{
    int dev = 0;
    RBF_CUDA_TRY(cudaGetDevice(&dev));
    RBF_REQUIRE(dev >= 0 && dev < 256, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_arena_mu);
    unsigned long long id = 0;
    RBF_TRY(current_context_id(&id));
    arena_slot &slot = g_arena_dev[dev];
    if (id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        RBF_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_arena));  // makes the context current
        RBF_TRY(current_context_id(&id));
        RBF_REQUIRE(id != 0, "no current CUDA context after cudaGetSymbolAddress");
        slot.ctx_id = id;
        slot.addr = p;
    }
    *out = static_cast<unsigned char *>(slot.addr);
    return RBF_OK;
}

// exclusive scan of n <= NOALLOC_HIST entries with two levels of block sums
int scan_noalloc(const int32_t *in, int32_t *out, int64_t n, int32_t *bsum, int32_t *boff,
                 cudaStream_t s)
{
    const int64_t nblk = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tile<<<(unsigned)nblk, SCAN_BS, 0, s>>>(in, out, n, bsum);
    RBF_LAUNCH_CHECK();
    if (nblk > 1) {
        k_scan_tile<<<1, SCAN_BS, 0, s>>>(bsum, boff, nblk, nullptr);
        RBF_LAUNCH_CHECK();
        k_scan_add<<<ceil_div(n, 256), 256, 0, s>>>(out, n, boff);
        RBF_LAUNCH_CHECK();
    }
    return RBF_OK;
}

}  // namespace

extern "C" int rbf_morton_order_noalloc(const double *X, int64_t N, int d, const double *lo_host,
                                        double side, int depth, int32_t *perm, uint64_t *keys,
                                        void *stream)
{
    RBF_REQUIRE(X && lo_host && perm && keys, "rbf_morton_order_noalloc: NULL pointer");
    RBF_REQUIRE(N >= 1 && N <= NOALLOC_MAX_N,
                "rbf_morton_order_noalloc: N=%lld outside [1, %lld], the size of its fixed arena",
                (long long)N, (long long)NOALLOC_MAX_N);
    RBF_REQUIRE(d >= 1 && d <= RBF_MAX_DIM, "rbf_morton_order_noalloc: d=%d out of range", d);
    RBF_REQUIRE(depth >= 0 && depth <= RBF_MAX_DEPTH && d * depth <= 63,
                "rbf_morton_order_noalloc: depth=%d out of range for d=%d", depth, d);
    RBF_REQUIRE(side > 0.0, "rbf_morton_order_noalloc: side must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *arena = nullptr;
    RBF_TRY(arena_address(&arena));
    uint64_t *kalt = reinterpret_cast<uint64_t *>(arena + OFF_KEYS);
    int32_t *valt = reinterpret_cast<int32_t *>(arena + OFF_VALS);
    int32_t *hist = reinterpret_cast<int32_t *>(arena + OFF_HIST);
    int32_t *offs = reinterpret_cast<int32_t *>(arena + OFF_OFFS);
    int32_t *bsum = reinterpret_cast<int32_t *>(arena + OFF_BSUM);
    int32_t *boff = reinterpret_cast<int32_t *>(arena + OFF_BOFF);
    // every arena region below is fully written before it is read; the corner
    // travels by value in the launch, so no host memory is read after this call
    corner_t lo{};
    for (int t = 0; t < d; ++t) lo.v[t] = lo_host[t];
    k_keys_corner<<<ceil_div(N, 256), 256, 0, s>>>(X, N, d, depth, lo, side, keys, perm);
    RBF_LAUNCH_CHECK();
    const int nbits = d * depth;
    const int nblk = (int)((N + RS_TILE - 1) / RS_TILE);
    uint64_t *ka = keys, *kb = kalt;
    int32_t *va = perm, *vb = valt;
    if (N > 1) {
        for (int shift = 0; shift < nbits; shift += 8) {
            k_rs_hist<<<nblk, RS_BS, 0, s>>>(ka, N, shift, hist, nblk);
            RBF_LAUNCH_CHECK();
            RBF_TRY(scan_noalloc(hist, offs, (int64_t)256 * nblk, bsum, boff, s));
            k_rs_scatter<<<nblk, RS_BS, 0, s>>>(ka, va, kb, vb, N, shift, offs, nblk);
            RBF_LAUNCH_CHECK();
            std::swap(ka, kb);
            std::swap(va, vb);
        }
    }
    if (ka != keys) {
        RBF_CUDA_TRY(cudaMemcpyAsync(keys, ka, N * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        RBF_CUDA_TRY(cudaMemcpyAsync(perm, va, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    return RBF_OK;
}
