// peaks.cu -- measured issue rates of the arithmetic units that bound the
// kernels of this library: FP32 and FP64 fused multiply-add (P2P, P2M, L2P)
// and the multi-function unit's ex2 and rsqrt (one per near-field pair: the
// Gaussian and the inverse multiquadric).  The rates are the denominators of
// the roofline fractions the benchmark reports.  The paper has no counterpart.
//
// Each thread runs NCH independent dependency chains of one instruction, so
// that the unit, not the instruction latency, sets the pace; the grid holds
// 32 warps per SM.  The chains' results are written out so that nothing is
// removed by the compiler.
#include <algorithm>

#include "rbf_internal.cuh"

namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeBlocksPerSM = 4;

template <int KIND>
struct probe_traits;
template <>
struct probe_traits<RBF_PROBE_FFMA> {
    using T = float;
    static constexpr int NCH = 16;
    static constexpr double OPS = 2.0;  // flops per FMA
};
template <>
struct probe_traits<RBF_PROBE_DFMA> {
    using T = double;
    static constexpr int NCH = 8;
    static constexpr double OPS = 2.0;
};
template <>
struct probe_traits<RBF_PROBE_EX2> {
    using T = float;
    static constexpr int NCH = 8;
    static constexpr double OPS = 1.0;  // results per instruction
};
template <>
struct probe_traits<RBF_PROBE_RSQRT> {
    using T = float;
    static constexpr int NCH = 8;
    static constexpr double OPS = 1.0;
};

__device__ __forceinline__ float mufu_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) k_probe(int iters, double a, double b,
                                                       typename probe_traits<KIND>::T *out)
{
    using T = typename probe_traits<KIND>::T;
    constexpr int NCH = probe_traits<KIND>::NCH;
    T x[NCH];
    const T m = (T)a, c = (T)b;
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = (T)(0.5 + 1e-3 * (threadIdx.x + k));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            if (KIND == RBF_PROBE_FFMA || KIND == RBF_PROBE_DFMA)
                x[k] = fma(x[k], m, c);  // stays bounded: |m| < 1
            else if (KIND == RBF_PROBE_EX2)
                x[k] = mufu_ex2(-(float)x[k]);  // in (1/2, 1] after the first step
            else
                x[k] = mufu_rsqrt((float)x[k]);  // tends to 1
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int KIND>
int run_probe(double seconds, double *rate, cudaStream_t s)
{
    using T = typename probe_traits<KIND>::T;
    int dev = 0, nsm = 0;
    RBF_CUDA_TRY(cudaGetDevice(&dev));
    RBF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * kProbeBlocksPerSM;
    T *out = nullptr;
    RBF_TRY(rbf_alloc(&out, (size_t)grid * kProbeBlock));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = RBF_OK;
    auto timed = [&](int iters, float *ms) -> int {
        RBF_CUDA_TRY(cudaEventRecord(e0, s));
        k_probe<KIND><<<grid, kProbeBlock, 0, s>>>(iters, 0.999, 1e-4, out);
        RBF_LAUNCH_CHECK();
        RBF_CUDA_TRY(cudaEventRecord(e1, s));
        RBF_CUDA_TRY(cudaEventSynchronize(e1));
        RBF_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        return RBF_OK;
    };
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rbf_set_error("rbf_peak_probe: cudaEventCreate failed");
            status = RBF_ECUDA;
            break;
        }
        // calibrate on a short launch, then time one launch of about `seconds`
        int iters = 2048;
        float ms = 0.f;
        if ((status = timed(iters, &ms)) != RBF_OK) break;
        if ((status = timed(iters, &ms)) != RBF_OK) break;
        const double want = seconds * 1e3 / (double)(ms > 1e-3f ? ms : 1e-3f);
        iters = (int)std::min(std::max(want * iters, 2048.0), 1.0e8);
        if ((status = timed(iters, &ms)) != RBF_OK) break;
        const double ops = (double)grid * kProbeBlock * probe_traits<KIND>::NCH * (double)iters *
                           probe_traits<KIND>::OPS;
        *rate = ops / (ms * 1e-3);
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    rbf_free(out);
    return status;
}

}  // namespace

extern "C" int rbf_peak_probe(int kind, double seconds, double *rate_host, void *stream)
{
    RBF_REQUIRE(rate_host, "rbf_peak_probe: rate_host is NULL");
    RBF_REQUIRE(seconds > 0.0 && seconds <= 10.0, "rbf_peak_probe: seconds=%g outside (0, 10]",
                seconds);
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
        case RBF_PROBE_FFMA: return run_probe<RBF_PROBE_FFMA>(seconds, rate_host, s);
        case RBF_PROBE_DFMA: return run_probe<RBF_PROBE_DFMA>(seconds, rate_host, s);
        case RBF_PROBE_EX2: return run_probe<RBF_PROBE_EX2>(seconds, rate_host, s);
        case RBF_PROBE_RSQRT: return run_probe<RBF_PROBE_RSQRT>(seconds, rate_host, s);
        default: break;
    }
    RBF_REQUIRE(false, "rbf_peak_probe: unknown kind %d", kind);
}
