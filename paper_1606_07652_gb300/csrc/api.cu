// api.cu -- status codes, error messages and device allocation helpers.
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>

#include <algorithm>

#include <nvtx3/nvToolsExt.h>

#include "rbf_internal.cuh"

static thread_local char g_last_error[512] = "";

void rbf_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

int rbf_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();  // clear the sticky-free allocation error
        rbf_set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RBF_ENOMEM : RBF_ECUDA;
    }
    // test aid: with RBF_POISON set, every allocation starts as all-ones bytes (NaN
    // in FP32 and FP64), so an entry that is read before it is written shows up
    if (getenv("RBF_POISON") != nullptr) {
        e = cudaMemset(*p, 0xFF, bytes);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(*p);
            *p = nullptr;
            rbf_set_error("poisoning a new allocation failed: %s", cudaGetErrorString(e));
            return RBF_ECUDA;
        }
    }
    return RBF_OK;
}

void rbf_free(void *p)
{
    if (p) cudaFree(p);
}

extern "C" const char *rbf_strerror(int code)
{
    switch (code) {
        case RBF_OK: return "success";
        case RBF_EINVAL: return "invalid argument";
        case RBF_ENOMEM: return "device out of memory";
        case RBF_ECUDA: return "CUDA error";
        case RBF_ENOCONV: return "iterative solve did not converge";
        case RBF_ETIMEOUT: return "bounded device wait timed out";
        case RBF_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

extern "C" const char *rbf_last_error(void) { return g_last_error; }

extern "C" const char *rbf_version(void) { return "0.1.0"; }

// ---------------------------------------------------------------- profiling --
namespace {
const char *const kPassNames[RBF_PASS_COUNT] = {"rbf P2P", "rbf P2M", "rbf M2M", "rbf M2L",
                                                "rbf L2P", "rbf permute"};
}

// Every pass is also an NVTX range (header-only NVTX 3: free unless a profiler
// that collects ranges is attached).
rbf_pass_timer::rbf_pass_timer(rbf_tree *t_, int pass_, cudaStream_t s_, int launches)
    : t(t_), pass(pass_), s(s_)
{
    nvtxRangePushA(pass >= 0 && pass < RBF_PASS_COUNT ? kPassNames[pass] : "rbf pass");
    if (!t || !t->prof.on) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    t->prof.start[pass].push_back(e);
    t->prof.launches[pass] += launches;
}

rbf_pass_timer::~rbf_pass_timer()
{
    nvtxRangePop();
    if (!t || !t->prof.on) return;
    if (t->prof.stop[pass].size() >= t->prof.start[pass].size()) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    t->prof.stop[pass].push_back(e);
}

static void prof_clear(rbf_tree *t)
{
    for (int p = 0; p < RBF_PASS_COUNT; ++p) {
        for (cudaEvent_t e : t->prof.start[p]) cudaEventDestroy(e);
        for (cudaEvent_t e : t->prof.stop[p]) cudaEventDestroy(e);
        t->prof.start[p].clear();
        t->prof.stop[p].clear();
        t->prof.launches[p] = 0;
    }
}

void rbf_prof_release(rbf_tree *t) { prof_clear(t); }

extern "C" int rbf_p2m_launch_shape(const rbf_tree *t, int *shape_host)
{
    RBF_REQUIRE(t && shape_host, "rbf_p2m_launch_shape: NULL argument");
    const rbf_plan *p = t->plan[RBF_FP32];
    *shape_host = p ? p->p2m_shape : 0;
    return RBF_OK;
}

extern "C" int rbf_profile(rbf_tree *t, int enable)
{
    RBF_REQUIRE(t != nullptr, "rbf_profile: tree is NULL");
    prof_clear(t);
    t->prof.on = enable != 0;
    return RBF_OK;
}

extern "C" int rbf_profile_read(rbf_tree *t, double *ms, int64_t *launches)
{
    RBF_REQUIRE(t != nullptr, "rbf_profile_read: tree is NULL");
    for (int p = 0; p < RBF_PASS_COUNT; ++p) {
        double sum = 0.0;
        const size_t n = std::min(t->prof.start[p].size(), t->prof.stop[p].size());
        for (size_t q = 0; q < n; ++q) {
            RBF_CUDA_TRY(cudaEventSynchronize(t->prof.stop[p][q]));
            float v = 0.0f;
            RBF_CUDA_TRY(cudaEventElapsedTime(&v, t->prof.start[p][q], t->prof.stop[p][q]));
            sum += v;
        }
        if (ms) ms[p] = sum;
        if (launches) launches[p] = t->prof.launches[p];
    }
    const bool on = t->prof.on;
    prof_clear(t);
    t->prof.on = on;
    return RBF_OK;
}
