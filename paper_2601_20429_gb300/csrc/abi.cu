// Status strings, version and the per-thread error text of the C ABI.
#include <cuda_runtime.h>

#include <stdint.h>

#include <mutex>
#include <string>

#include "grtx_internal.cuh"

namespace {
thread_local std::string g_last_error;

// The library's device memory pool, one per device: stream-ordered allocations whose freed
// memory stays mapped for the next build or trace (the default pool hands it back to the
// driver at every synchronisation, and mapping it again costs milliseconds per build).
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
bool g_pool_ready[64];

int library_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return grtx_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return grtx_fail(GRTX_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) return grtx_cuda_fail(e, "cudaMemPoolCreate");
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return grtx_cuda_fail(e, "cudaMemPoolSetAttribute");
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return GRTX_OK;
}
}  // namespace

int grtx_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    cudaMemPool_t pool;
    int st = library_pool(&pool);
    if (st) return st;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return grtx_fail(GRTX_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_memory_trim(int64_t keep_bytes)
{
    if (keep_bytes < 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "keep_bytes must be >= 0");
    cudaMemPool_t pool;
    int st = library_pool(&pool);
    if (st) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return grtx_cuda_fail(e, "cudaDeviceSynchronize");
    e = cudaMemPoolTrimTo(pool, (size_t)keep_bytes);
    if (e != cudaSuccess) return grtx_cuda_fail(e, "cudaMemPoolTrimTo");
    return GRTX_OK;
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
