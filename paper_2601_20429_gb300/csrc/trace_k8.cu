// Trace kernels for a k-buffer of 8 entries (one translation unit per k keeps builds parallel).
#include "trace_impl.cuh"

GRTX_INSTANTIATE_TRACE(8)
