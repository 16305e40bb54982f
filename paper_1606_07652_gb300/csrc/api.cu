// api.cu -- status codes, error messages and device allocation helpers.
#include <stdarg.h>
#include <stdio.h>

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
