// mlp.cu -- the small network of the learned preconditioner: input -> 3 hidden
// layers (ReLU) -> output, BF16 weights, FP32 activations and accumulation.
// Every GEMM (forward, input gradient, weight gradient) runs on the tensor
// cores through mma.sync m16n8k16 BF16 with FP32 accumulation, from operands
// staged in shared memory; the optimiser is Adam on FP32 master weights.
#include <cuda_bf16.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cstring>

#include "rbf_internal.cuh"

struct rbf_mlp {
    int nl = 4;                 // layers
    int dims[5] = {0};          // dims[0] input ... dims[4] output
    int64_t nparam = 0;
    int64_t woff[4], boff[4];   // offsets in the flat parameter vector
    float *param = nullptr;     // FP32 master: W_l (out x in, row-major) then b_l, per layer
    float *grad = nullptr;
    float *m = nullptr, *v = nullptr;  // Adam moments
    __nv_bfloat16 *wbf = nullptr;      // BF16 copies of the weights (same offsets as param)
    int64_t step = 0;
    // activations for batches up to cap
    int64_t cap = 0;
    float *h[5] = {nullptr};    // h[0] unused (input is the caller's), h[1..3] hidden, h[4] output
    float *g0 = nullptr, *g1 = nullptr;  // gradient ping-pong (B x 128)
    float *part = nullptr;      // loss partial sums
};

namespace {

constexpr int GB_M = 64, GB_N = 64, GB_K = 32;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <typename T>
__device__ __forceinline__ __nv_bfloat16 to_bf16(T v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_bf16<float>(float v)
{
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_bf16<__nv_bfloat16>(__nv_bfloat16 v)
{
    return v;
}

// C[m][n] (+)= sum_k A(m,k) B(n,k) (+ bias[n]) (relu), with A(m,k) = A[m*sam + k*sak] and
// B(n,k) = B[n*sbn + k*sbk] rounded to BF16 when staged; FP32 accumulation.
template <typename TA, typename TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(const TA *A, int64_t sam, int64_t sak, const TB *B,
                                                   int64_t sbn, int64_t sbk, float *C, int64_t ldc,
                                                   int M, int N, int K, const float *bias, int relu,
                                                   int accumulate)
{
    __shared__ __align__(16) __nv_bfloat16 As[GB_M][GB_K + 8];
    __shared__ __align__(16) __nv_bfloat16 Bs[GB_N][GB_K + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int gq = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += GB_K) {
        for (int idx = tid; idx < GB_M * GB_K; idx += 128) {
            const int r = idx / GB_K, c = idx % GB_K;
            const int m = m0 + r, k = k0 + c;
            As[r][c] = (m < M && k < K) ? to_bf16(A[(int64_t)m * sam + (int64_t)k * sak])
                                        : __float2bfloat16_rn(0.0f);
        }
        for (int idx = tid; idx < GB_N * GB_K; idx += 128) {
            const int r = idx / GB_K, c = idx % GB_K;
            const int n = n0 + r, k = k0 + c;
            Bs[r][c] = (n < N && k < K) ? to_bf16(B[(int64_t)n * sbn + (int64_t)k * sbk])
                                        : __float2bfloat16_rn(0.0f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm * 32 + mt * 16 + gq, c = kk + tq * 2;
                af[mt][0] = pack_bf16(As[r][c], As[r][c + 1]);
                af[mt][1] = pack_bf16(As[r + 8][c], As[r + 8][c + 1]);
                af[mt][2] = pack_bf16(As[r][c + 8], As[r][c + 9]);
                af[mt][3] = pack_bf16(As[r + 8][c + 8], As[r + 8][c + 9]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = wn * 32 + nt * 8 + gq, c = kk + tq * 2;
                bfr[nt][0] = pack_bf16(Bs[n][c], Bs[n][c + 1]);
                bfr[nt][1] = pack_bf16(Bs[n][c + 8], Bs[n][c + 9]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    float *d = acc[mt][nt];
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                        : "r"(af[mt][0]), "r"(af[mt][1]), "r"(af[mt][2]), "r"(af[mt][3]),
                          "r"(bfr[nt][0]), "r"(bfr[nt][1]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + wm * 32 + mt * 16 + gq + (c >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + nt * 8 + tq * 2 + (c & 1);
                if (m >= M || n >= N) continue;
                float v = acc[mt][nt][c];
                if (bias) v += bias[n];
                if (relu) v = fmaxf(v, 0.0f);
                float *dst = C + (int64_t)m * ldc + n;
                *dst = accumulate ? *dst + v : v;
            }
}

template <typename TA, typename TB>
int gemm(const TA *A, int64_t sam, int64_t sak, const TB *B, int64_t sbn, int64_t sbk, float *C,
         int64_t ldc, int M, int N, int K, const float *bias, int relu, int accumulate, cudaStream_t s)
{
    dim3 grid(ceil_div(M, GB_M), ceil_div(N, GB_N));
    k_gemm_bf16<TA, TB><<<grid, 128, 0, s>>>(A, sam, sak, B, sbn, sbk, C, ldc, M, N, K, bias, relu,
                                             accumulate);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

__global__ void k_to_bf16(const float *in, __nv_bfloat16 *out, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// g = 2 (y - t) / (B * dout); part[block] = partial sum of (y - t)^2
__global__ void k_loss_grad(const float *y, const float *t, int64_t n, float scale, float *g,
                            float *part)
{
    __shared__ float sh[256];
    float s = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const float e = y[i] - t[i];
        if (g) g[i] = scale * e;
        s += e * e;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// gb[n] = sum_m g[m][n]  (fixed order per column)
__global__ void k_colsum(const float *g, int64_t rows, int cols, float *gb)
{
    const int n = blockIdx.x;
    __shared__ float sh[256];
    float s = 0.0f;
    for (int64_t m = threadIdx.x; m < rows; m += 256) s += g[m * cols + n];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[n] = sh[0];
}

// g *= (h > 0)   (ReLU derivative from the post-activation)
__global__ void k_relu_mask(float *g, const float *h, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(h[i] > 0.0f)) g[i] = 0.0f;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// SplitMix64 (Steele, Lea, Flood 2014) -> two uniforms -> Box-Muller normal.
__host__ __device__ inline uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

}  // namespace

static int mlp_ensure(rbf_mlp *n, int64_t B)
{
    if (B <= n->cap) return RBF_OK;
    for (int l = 1; l <= 4; ++l) {
        rbf_free(n->h[l]);
        n->h[l] = nullptr;
    }
    rbf_free(n->g0);
    rbf_free(n->g1);
    rbf_free(n->part);
    n->g0 = n->g1 = n->part = nullptr;
    n->cap = 0;
    int wmax = 0;
    for (int l = 0; l <= 4; ++l) wmax = std::max(wmax, n->dims[l]);
    for (int l = 1; l <= 4; ++l) RBF_TRY(rbf_alloc(&n->h[l], (size_t)B * n->dims[l]));
    RBF_TRY(rbf_alloc(&n->g0, (size_t)B * wmax));
    RBF_TRY(rbf_alloc(&n->g1, (size_t)B * wmax));
    RBF_TRY(rbf_alloc(&n->part, 1024));
    n->cap = B;
    return RBF_OK;
}

static int mlp_refresh_bf16(rbf_mlp *n, cudaStream_t s)
{
    k_to_bf16<<<ceil_div(n->nparam, 256), 256, 0, s>>>(n->param, n->wbf, n->nparam);
    RBF_LAUNCH_CHECK();
    return RBF_OK;
}

extern "C" int rbf_mlp_create(int d_in, int width, int d_out, uint64_t seed, rbf_mlp **out)
{
    RBF_REQUIRE(out != nullptr, "rbf_mlp_create: out is NULL");
    *out = nullptr;
    RBF_REQUIRE(d_in >= 1 && d_in <= 4096 && width >= 1 && width <= 4096 && d_out >= 1 && d_out <= 4096,
                "rbf_mlp_create: bad sizes");
    rbf_mlp *n = new rbf_mlp();
    n->dims[0] = d_in;
    n->dims[1] = n->dims[2] = n->dims[3] = width;
    n->dims[4] = d_out;
    int64_t off = 0;
    for (int l = 0; l < 4; ++l) {
        n->woff[l] = off;
        off += (int64_t)n->dims[l + 1] * n->dims[l];
        n->boff[l] = off;
        off += n->dims[l + 1];
    }
    n->nparam = off;
    // He-normal weights from a counter-based generator, zero biases (host, deterministic)
    std::vector<float> h(off, 0.0f);
    for (int l = 0; l < 4; ++l) {
        const double sd = std::sqrt(2.0 / n->dims[l]);
        const int64_t cnt = (int64_t)n->dims[l + 1] * n->dims[l];
        for (int64_t i = 0; i < cnt; ++i) {
            const uint64_t a = splitmix64(seed * 0x100000001B3ull + (uint64_t)(n->woff[l] + i) * 2);
            const uint64_t b = splitmix64(a ^ 0xD1B54A32D192ED03ull);
            const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
            h[n->woff[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
        }
    }
    int st = rbf_alloc(&n->param, off);
    if (st == RBF_OK) st = rbf_alloc(&n->grad, off);
    if (st == RBF_OK) st = rbf_alloc(&n->m, off);
    if (st == RBF_OK) st = rbf_alloc(&n->v, off);
    if (st == RBF_OK) st = rbf_alloc(&n->wbf, off);
    if (st == RBF_OK && cudaMemcpy(n->param, h.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        st = RBF_ECUDA;
    if (st == RBF_OK && (cudaMemset(n->m, 0, off * sizeof(float)) != cudaSuccess ||
                         cudaMemset(n->v, 0, off * sizeof(float)) != cudaSuccess))
        st = RBF_ECUDA;
    if (st == RBF_OK) st = mlp_refresh_bf16(n, 0);
    if (st == RBF_OK && cudaDeviceSynchronize() != cudaSuccess) st = RBF_ECUDA;
    if (st != RBF_OK) {
        rbf_mlp_free(n);
        return st;
    }
    *out = n;
    return RBF_OK;
}

extern "C" void rbf_mlp_free(rbf_mlp *n)
{
    if (!n) return;
    rbf_free(n->param);
    rbf_free(n->grad);
    rbf_free(n->m);
    rbf_free(n->v);
    rbf_free(n->wbf);
    for (int l = 1; l <= 4; ++l) rbf_free(n->h[l]);
    rbf_free(n->g0);
    rbf_free(n->g1);
    rbf_free(n->part);
    delete n;
}

// ------------------------------------------------------- checkpoints -----
// File: "RBFMLP01", int32 dims[5], int64 nparam, int64 Adam step, then the FP32
// parameters, Adam first and second moments (nparam each), little-endian.
static const char kMlpMagic[8] = {'R', 'B', 'F', 'M', 'L', 'P', '0', '1'};

extern "C" int rbf_mlp_save(const rbf_mlp *n, const char *path)
{
    RBF_REQUIRE(n && path, "rbf_mlp_save: NULL argument");
    std::vector<float> buf((size_t)n->nparam * 3);
    RBF_CUDA_TRY(cudaDeviceSynchronize());
    RBF_CUDA_TRY(cudaMemcpy(buf.data(), n->param, n->nparam * sizeof(float), cudaMemcpyDeviceToHost));
    RBF_CUDA_TRY(cudaMemcpy(buf.data() + n->nparam, n->m, n->nparam * sizeof(float),
                            cudaMemcpyDeviceToHost));
    RBF_CUDA_TRY(cudaMemcpy(buf.data() + 2 * n->nparam, n->v, n->nparam * sizeof(float),
                            cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    RBF_REQUIRE(f != nullptr, "rbf_mlp_save: cannot open %s", path);
    int32_t dims[5];
    for (int l = 0; l < 5; ++l) dims[l] = n->dims[l];
    const int64_t hdr[2] = {n->nparam, n->step};
    const bool ok = fwrite(kMlpMagic, 1, 8, f) == 8 && fwrite(dims, sizeof(dims), 1, f) == 1 &&
                    fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
                    fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    const bool closed = fclose(f) == 0;
    RBF_REQUIRE(ok && closed, "rbf_mlp_save: write to %s failed", path);
    return RBF_OK;
}

extern "C" int rbf_mlp_load(const char *path, rbf_mlp **out)
{
    RBF_REQUIRE(path && out, "rbf_mlp_load: NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    RBF_REQUIRE(f != nullptr, "rbf_mlp_load: cannot open %s", path);
    char magic[8] = {0};
    int32_t dims[5] = {0};
    int64_t hdr[2] = {0, 0};
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMlpMagic, 8) == 0 &&
              fread(dims, sizeof(dims), 1, f) == 1 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              dims[1] == dims[2] && dims[2] == dims[3] && hdr[0] > 0 && hdr[1] >= 0;
    rbf_mlp *n = nullptr;
    std::vector<float> buf;
    if (ok && rbf_mlp_create(dims[0], dims[1], dims[4], 0, &n) == RBF_OK && n->nparam == hdr[0]) {
        buf.resize((size_t)hdr[0] * 3);
        ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    } else {
        ok = false;
    }
    fclose(f);
    if (!ok) {
        rbf_mlp_free(n);
        rbf_set_error("rbf_mlp_load: %s is not a complete network checkpoint", path);
        return RBF_EINVAL;
    }
    const size_t bytes = (size_t)n->nparam * sizeof(float);
    int st = RBF_OK;
    if (cudaMemcpy(n->param, buf.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->m, buf.data() + n->nparam, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(n->v, buf.data() + 2 * n->nparam, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        rbf_set_error("rbf_mlp_load: CUDA copy failed");
        st = RBF_ECUDA;
    }
    n->step = hdr[1];
    if (st == RBF_OK) st = mlp_refresh_bf16(n, 0);
    if (st == RBF_OK && cudaDeviceSynchronize() != cudaSuccess) st = RBF_ECUDA;
    if (st != RBF_OK) {
        rbf_mlp_free(n);
        return st;
    }
    *out = n;
    return RBF_OK;
}

extern "C" int rbf_mlp_num_params(const rbf_mlp *n, int64_t *count)
{
    RBF_REQUIRE(n && count, "rbf_mlp_num_params: NULL argument");
    *count = n->nparam;
    return RBF_OK;
}

extern "C" int rbf_mlp_get_params(const rbf_mlp *n, float *host)
{
    RBF_REQUIRE(n && host, "rbf_mlp_get_params: NULL argument");
    RBF_CUDA_TRY(cudaMemcpy(host, n->param, n->nparam * sizeof(float), cudaMemcpyDeviceToHost));
    return RBF_OK;
}

extern "C" int rbf_mlp_set_params(rbf_mlp *n, const float *host)
{
    RBF_REQUIRE(n && host, "rbf_mlp_set_params: NULL argument");
    RBF_CUDA_TRY(cudaMemcpy(n->param, host, n->nparam * sizeof(float), cudaMemcpyHostToDevice));
    RBF_CUDA_TRY(cudaMemset(n->m, 0, n->nparam * sizeof(float)));
    RBF_CUDA_TRY(cudaMemset(n->v, 0, n->nparam * sizeof(float)));
    n->step = 0;
    RBF_TRY(mlp_refresh_bf16(n, 0));
    RBF_CUDA_TRY(cudaDeviceSynchronize());
    return RBF_OK;
}

// forward pass into n->h[1..4]; X is B x dims[0] FP32 (device)
static int mlp_forward_impl(rbf_mlp *n, const float *X, int64_t B, cudaStream_t s)
{
    RBF_TRY(mlp_ensure(n, B));
    const float *in = X;
    for (int l = 0; l < 4; ++l) {
        const int din = n->dims[l], dout = n->dims[l + 1];
        RBF_TRY((gemm<float, __nv_bfloat16>(in, din, 1, n->wbf + n->woff[l], din, 1, n->h[l + 1], dout,
                                           (int)B, dout, din, n->param + n->boff[l], l < 3 ? 1 : 0, 0, s)));
        in = n->h[l + 1];
    }
    return RBF_OK;
}

extern "C" int rbf_mlp_forward(rbf_mlp *n, const float *X, int64_t B, float *Y, void *stream)
{
    RBF_REQUIRE(n && X && Y && B >= 1, "rbf_mlp_forward: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(mlp_forward_impl(n, X, B, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(Y, n->h[4], B * n->dims[4] * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return RBF_OK;
}

// gradient of mean((y - t)^2) into n->grad; returns the loss on the host
static int mlp_gradient_impl(rbf_mlp *n, const float *X, const float *T, int64_t B, float *loss,
                             cudaStream_t s)
{
    RBF_TRY(mlp_forward_impl(n, X, B, s));
    const int dout = n->dims[4];
    const int64_t ny = B * dout;
    const int nb = (int)std::min<int64_t>(1024, ceil_div(ny, 256));
    k_loss_grad<<<nb, 256, 0, s>>>(n->h[4], T, ny, 2.0f / (float)ny, n->g0, n->part);
    RBF_LAUNCH_CHECK();
    float *g = n->g0, *gn = n->g1;
    for (int l = 3; l >= 0; --l) {
        const int din = n->dims[l], dl = n->dims[l + 1];
        const float *hin = l > 0 ? n->h[l] : X;
        // dW_l[o][i] = sum_m g[m][o] h_in[m][i]
        RBF_TRY((gemm<float, float>(g, 1, dl, hin, 1, din, n->grad + n->woff[l], din, dl, din, (int)B,
                                   nullptr, 0, 0, s)));
        k_colsum<<<dl, 256, 0, s>>>(g, B, dl, n->grad + n->boff[l]);
        RBF_LAUNCH_CHECK();
        if (l > 0) {
            // g_prev[m][i] = sum_o g[m][o] W_l[o][i], then the ReLU mask of h_l
            RBF_TRY((gemm<float, __nv_bfloat16>(g, dl, 1, n->wbf + n->woff[l], 1, din, gn, din, (int)B,
                                               din, dl, nullptr, 0, 0, s)));
            k_relu_mask<<<ceil_div(B * din, 256), 256, 0, s>>>(gn, n->h[l], B * din);
            RBF_LAUNCH_CHECK();
            std::swap(g, gn);
        }
    }
    if (loss) {
        std::vector<float> p(nb);
        RBF_CUDA_TRY(cudaMemcpyAsync(p.data(), n->part, nb * sizeof(float), cudaMemcpyDeviceToHost, s));
        RBF_CUDA_TRY(cudaStreamSynchronize(s));
        double sum = 0.0;
        for (float q : p) sum += q;
        *loss = (float)(sum / (double)ny);
    }
    return RBF_OK;
}

extern "C" int rbf_mlp_gradient(rbf_mlp *n, const float *X, const float *T, int64_t B, float *grad,
                                float *loss_host, void *stream)
{
    RBF_REQUIRE(n && X && T && grad && B >= 1, "rbf_mlp_gradient: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    RBF_TRY(mlp_gradient_impl(n, X, T, B, loss_host, s));
    RBF_CUDA_TRY(cudaMemcpyAsync(grad, n->grad, n->nparam * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return RBF_OK;
}

int rbf_mlp_train_step_impl(rbf_mlp *n, const float *X, const float *T, int64_t B, float lr,
                            float *loss, cudaStream_t s)
{
    RBF_TRY(mlp_gradient_impl(n, X, T, B, loss, s));
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
    k_adam<<<ceil_div(n->nparam, 256), 256, 0, s>>>(n->param, n->grad, n->m, n->v, n->nparam, lr, b1,
                                                    b2, 1e-8f, c1, c2);
    RBF_LAUNCH_CHECK();
    return mlp_refresh_bf16(n, s);
}

extern "C" int rbf_mlp_train_step(rbf_mlp *n, const float *X, const float *T, int64_t B, float lr,
                                  float *loss_host, void *stream)
{
    RBF_REQUIRE(n && X && T && B >= 1 && lr > 0.0f, "rbf_mlp_train_step: bad arguments");
    return rbf_mlp_train_step_impl(n, X, T, B, lr, loss_host, (cudaStream_t)stream);
}

int rbf_mlp_dims(const rbf_mlp *n, int *din, int *dout)
{
    *din = n->dims[0];
    *dout = n->dims[4];
    return RBF_OK;
}

int rbf_mlp_forward_dev(rbf_mlp *n, const float *X, int64_t B, const float **Y, cudaStream_t s)
{
    RBF_TRY(mlp_forward_impl(n, X, B, s));
    *Y = n->h[4];
    return RBF_OK;
}
