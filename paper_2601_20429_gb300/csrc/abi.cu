// Status strings, version and the per-thread error text of the C ABI.
#include <cuda_runtime.h>

#include <string>

#include "grtx_internal.cuh"

namespace {
thread_local std::string g_last_error;
}

int grtx_fail(int status, const std::string &msg)
{
    g_last_error = msg;
    return status;
}

int grtx_cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GRTX_ERR_OOM : GRTX_ERR_CUDA;
}

extern "C" GRTX_API const char *grtx_status_string(int status)
{
    switch (status) {
    case GRTX_OK: return "ok";
    case GRTX_ERR_INVALID_ARG: return "invalid argument";
    case GRTX_ERR_OOM: return "out of device memory";
    case GRTX_ERR_CUDA: return "CUDA error";
    case GRTX_ERR_OVERFLOW_FATAL: return "fixed limit exceeded";
    case GRTX_ERR_TIMEOUT: return "timed out";
    case GRTX_ERR_BUSY: return "busy";
    case GRTX_ERR_NOT_FOUND: return "not found";
    default: return "unknown status";
    }
}

extern "C" GRTX_API int grtx_version(void) { return GRTX_VERSION; }

extern "C" GRTX_API const char *grtx_last_error(void) { return g_last_error.c_str(); }
