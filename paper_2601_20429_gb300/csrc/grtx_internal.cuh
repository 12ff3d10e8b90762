// Internal declarations shared by the libgrtx translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "grtx.h"

#define GRTX_LEAF 0x80000000u
#define GRTX_NONE 0xFFFFFFFFu
#define GRTX_STACK 128         // traversal stack entries per ray; the build rejects deeper trees
#define GRTX_STACK4 192        // the same for 4-wide nodes: up to 3 per level of a tree of depth <= 64

// Record the host-side text of an error for grtx_last_error() and return the status.
int grtx_fail(int status, const std::string &msg);
int grtx_cuda_fail(cudaError_t e, const char *what);
// Stream-ordered allocation from the library's per-device pool (freed with cudaFreeAsync);
// GRTX_ERR_OOM with a message on failure, *p = NULL then.
int grtx_malloc_async(void **p, size_t bytes, cudaStream_t s);

#define GRTX_CUDA(call)                                                  \
    do {                                                                 \
        cudaError_t e__ = (call);                                        \
        if (e__ != cudaSuccess) return grtx_cuda_fail(e__, #call);       \
    } while (0)

#define GRTX_CHECK_LAUNCH(name)                                          \
    do {                                                                 \
        cudaError_t e__ = cudaGetLastError();                            \
        if (e__ != cudaSuccess) return grtx_cuda_fail(e__, name);        \
    } while (0)

// A built scene. All pointers are device memory owned by the scene.
struct grtx_scene {
    int form = 0;
    int sh_degree = 0;
    int n_coef = 1;
    int app_stride = 4;          // floats per appearance record (SH coefficients, padded to 4)
    int depth = 0;
    float alpha_min = 0.01f;
    int bvh_codes = GRTX_CODES_SIZED, bvh_builder = GRTX_BUILDER_PLOC;   // as built (for rebuilds)
    int bvh_width = 2;           // 4: nodes4 holds the 4-wide collapse of the binary tree
    int bvh_quant = 0;           // 1: the 4-wide nodes have quantised child boxes (64 bytes each)
    int64_t n = 0, n_valid = 0, n_leaves = 0, n_nodes = 0;
    float bounds[6] = {0, 0, 0, 0, 0, 0};
    float4 *nodes = nullptr;     // [n_nodes][4]: BVH2 node, see grtx_scene_export
    float4 *nodes4 = nullptr;    // [n_nodes4][8] (or [4] quantised): 4-wide nodes (bvh_width 4), see grtx_params
    int64_t n_nodes4 = 0;
    float4 *geom = nullptr;      // [n_valid][4]: rows (A_j | mu_j) + (o, -kappa^2 log2(e)/2, id, 0), leaf order
    float4 *tris = nullptr;      // proxy form: [n_leaves][3] world triangle (v0 | gidx, v1, v2)
    float *app = nullptr;        // [n_valid][app_stride] SH coefficients in leaf order
    float4 *raw = nullptr;       // [n_valid][3] raw parameters in leaf order: (mu, logit), (log-scales, 0), q
    uint32_t *gid = nullptr;     // [n] Gaussian id of each sorted Gaussian, then of each culled one
    uint32_t *leaf_ids = nullptr;// [n_leaves] Gaussian id of each leaf
    uint64_t *codes = nullptr;   // [n_leaves] sorted Morton codes
    const float4 *tpl_nodes = nullptr;   // icosphere forms: shared template BVH (not owned)
    const float4 *tpl_tris = nullptr;
    cudaStream_t stream = nullptr;
    // trace workspace (per resident ray slot checkpoint / eviction lists), grown on demand
    void *ws = nullptr;
    size_t ws_bytes = 0;
    unsigned int *d_counter = nullptr;   // ray-queue counters (2 per launch kind)
};

// Device template BVH and triangles of an icosphere form on the current device (built once).
int grtx_template_blas(int form, const float4 **nodes, const float4 **tris);

// Persistent-launch geometry of the trace kernels (filled by the trace unit).
int grtx_trace_slots(int kind, int k, int *blocks, int *threads);

// Exclusive scan of uint32 values in place (temp from grtx_scan_temp_bytes).
size_t grtx_scan_temp_bytes(int64_t m);
int grtx_scan_exclusive(uint32_t *d_data, int64_t m, void *d_temp, cudaStream_t s);

static inline int grtx_div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
