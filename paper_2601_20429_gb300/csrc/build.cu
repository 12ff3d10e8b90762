// BVH build on the GPU: Gaussian activation and instance transform, Morton codes, an LSD
// radix sort, the binary radix tree (Karras 2012), bottom-up bounds and node compaction.
// The paper builds an Embree BVH-6 on the host (Sec. V-A); this build is an LBVH so that the
// whole build stays on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "grtx_internal.cuh"

namespace {

constexpr int kThreads = 256;

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------------------------------
// Activation and instance transform (Sec. II-B parameters; Sec. IV-A unit sphere).
// ------------------------------------------------------------------------------------------
// Opacity of Gaussian i (sigmoid of its logit); it has a record and a box iff o > alpha_min.
__device__ __forceinline__ float gaussian_opacity(const float *__restrict__ logits, int64_t i)
{
    return 1.0f / (1.0f + expf(-logits[i]));
}

// Record (rows (A_j | mu_j), then (o, -kappa^2 log2(e) / 2, i, 0)) and world box of Gaussian i,
// written to geom[0..3] and bb[0..5]. A Gaussian at or below alpha_min gets a zero record
// (its test never passes) and an empty box.
__device__ __forceinline__ void prep_one(const float *__restrict__ means, const float *__restrict__ log_scales,
                                         const float *__restrict__ quats, const float *__restrict__ logits,
                                         int64_t i, float alpha_min, float4 *__restrict__ geom,
                                         float *__restrict__ bb)
{
    float o = gaussian_opacity(logits, i);
    if (!(o > alpha_min)) {
        geom[0] = geom[1] = geom[2] = geom[3] = make_float4(0, 0, 0, 0);
        bb[0] = bb[1] = bb[2] = INFINITY;
        bb[3] = bb[4] = bb[5] = -INFINITY;
        return;
    }
    float kap = sqrtf(2.0f * logf(o / alpha_min));
    float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float s[3] = {expf(log_scales[3 * i]), expf(log_scales[3 * i + 1]), expf(log_scales[3 * i + 2])};
    float w = quats[4 * i], x = quats[4 * i + 1], y = quats[4 * i + 2], z = quats[4 * i + 3];
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    // rotation matrix of the unit quaternion, row-major R[a][j]; column j = local axis j
    float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                     {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                     {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    float4 rows[3];
    for (int j = 0; j < 3; ++j) {
        float f = 1.0f / (kap * s[j]);
        rows[j] = make_float4(R[0][j] * f, R[1][j] * f, R[2][j] * f, mu[j]);
    }
    geom[0] = rows[0];
    geom[1] = rows[1];
    geom[2] = rows[2];
    geom[3] = make_float4(o, -0.5f * kap * kap * 1.4426950408889634f, __int_as_float((int)i), 0.f);
    for (int a = 0; a < 3; ++a) {
        float var = R[a][0] * R[a][0] * s[0] * s[0] + R[a][1] * R[a][1] * s[1] * s[1] +
                    R[a][2] * R[a][2] * s[2] * s[2];
        float h = kap * sqrtf(var);
        h = h * (1.0f + 1e-5f) + 1e-6f * fabsf(mu[a]);   // conservative under FP32 rounding
        bb[a] = mu[a] - h;
        bb[3 + a] = mu[a] + h;
    }
}

// Raw parameters of Gaussian i packed for the backward: (mu, logit), (log-scales, 0), q.
__device__ __forceinline__ void pack_raw(const float *__restrict__ means, const float *__restrict__ log_scales,
                                         const float *__restrict__ quats, const float *__restrict__ logits,
                                         int64_t i, float4 *__restrict__ raw)
{
    raw[0] = make_float4(means[3 * i], means[3 * i + 1], means[3 * i + 2], logits[i]);
    raw[1] = make_float4(log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2], 0.f);
    raw[2] = make_float4(quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]);
}

__global__ void k_prep(const float *__restrict__ means, const float *__restrict__ log_scales,
                       const float *__restrict__ quats, const float *__restrict__ logits, int64_t n,
                       float alpha_min, float4 *__restrict__ geom, float *__restrict__ aabb)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    prep_one(means, log_scales, quats, logits, i, alpha_min, geom + 4 * i, aabb + 6 * i);
}

// ------------------------------------------------------------------------------------------
// Centroid bounds and Morton codes.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void atomic_min_f(float *a, float v)
{
    if (v >= 0.0f) atomicMin(reinterpret_cast<int *>(a), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float *a, float v)
{
    if (v >= 0.0f) atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
    else atomicMin(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}

__global__ void k_init_bounds(float *b)
{
    if (threadIdx.x < 3) b[threadIdx.x] = INFINITY;
    else if (threadIdx.x < 6) b[threadIdx.x] = -INFINITY;
}

__device__ __forceinline__ bool box_empty(const float *bb)
{
    return !(bb[0] <= bb[3] && bb[1] <= bb[4] && bb[2] <= bb[5]);
}

__global__ void k_centroid_bounds(const float *__restrict__ aabb, int64_t n, float *__restrict__ bounds)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float *bb = aabb + 6 * i;
        if (box_empty(bb)) continue;
        for (int a = 0; a < 3; ++a) {
            float c = __fmul_rn(0.5f, __fadd_rn(bb[a], bb[3 + a]));
            lo[a] = fminf(lo[a], c);
            hi[a] = fmaxf(hi[a], c);
        }
    }
    for (int off = 16; off > 0; off >>= 1)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            if (lo[a] <= hi[a]) {
                atomic_min_f(bounds + a, lo[a]);
                atomic_max_f(bounds + 3 + a, hi[a]);
            }
        }
}

// Spread the low 21 bits of v so that bit b lands at bit 3b.
__host__ __device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float *__restrict__ aabb, int64_t n, const float *__restrict__ bounds,
                         uint64_t *__restrict__ codes, uint32_t *__restrict__ values)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *bb = aabb + 6 * i;
    if (values) values[i] = (uint32_t)i;
    if (box_empty(bb)) { codes[i] = ~0ull; return; }
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        float c = __fmul_rn(0.5f, __fadd_rn(bb[a], bb[3 + a]));
        float ext = __fsub_rn(bounds[3 + a], bounds[a]);
        float scale = ext > 0.0f ? __fdiv_rn(2097152.0f, ext) : 0.0f;
        float u = __fmul_rn(__fsub_rn(c, bounds[a]), scale);
        q[a] = u <= 0.0f ? 0u : (u >= 2097151.0f ? 2097151u : (uint32_t)u);
    }
    codes[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
}

// Spread the low 16 bits of v so that bit b lands at bit 4b.
__host__ __device__ __forceinline__ uint64_t spread4(uint32_t v)
{
    uint64_t x = v & 0xffffu;
    x = (x | (x << 24)) & 0x000000ff000000ffull;
    x = (x | (x << 12)) & 0x000f000f000f000full;
    x = (x | (x << 6)) & 0x0303030303030303ull;
    x = (x | (x << 3)) & 0x1111111111111111ull;
    return x;
}

// Size-aware code: 16 bits each of the quantised centroid and of the box diagonal on the
// positions' grid at half resolution, interleaved x, y, z, size (see grtx_morton_codes_sized).
__global__ void k_morton_sized(const float *__restrict__ aabb, int64_t n, const float *__restrict__ bounds,
                               uint64_t *__restrict__ codes, uint32_t *__restrict__ values)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *bb = aabb + 6 * i;
    if (values) values[i] = (uint32_t)i;
    if (box_empty(bb)) { codes[i] = ~0ull; return; }
    float E = 0.0f;
    uint32_t q[4];
    for (int a = 0; a < 3; ++a) {
        float c = __fmul_rn(0.5f, __fadd_rn(bb[a], bb[3 + a]));
        float ext = __fsub_rn(bounds[3 + a], bounds[a]);
        E = ext > E ? ext : E;
        float scale = ext > 0.0f ? __fdiv_rn(65536.0f, ext) : 0.0f;
        float u = __fmul_rn(__fsub_rn(c, bounds[a]), scale);
        q[a] = u <= 0.0f ? 0u : (u >= 65535.0f ? 65535u : (uint32_t)u);
    }
    float ex = __fsub_rn(bb[3], bb[0]), ey = __fsub_rn(bb[4], bb[1]), ez = __fsub_rn(bb[5], bb[2]);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    float scale_s = E > 0.0f ? __fdiv_rn(32768.0f, E) : 0.0f;
    float us = __fmul_rn(__fsqrt_rn(d2), scale_s);
    q[3] = us <= 0.0f ? 0u : (us >= 65534.0f ? 65534u : (uint32_t)us);
    codes[i] = (spread4(q[0]) << 3) | (spread4(q[1]) << 2) | (spread4(q[2]) << 1) | spread4(q[3]);
}

// ------------------------------------------------------------------------------------------
// Exclusive scan of uint32 (tiles of 4096, recursive over tile sums).
// ------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_tiles(uint32_t *__restrict__ d, int64_t m, uint32_t *__restrict__ tile_sums)
{
    __shared__ uint32_t warp_sums[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < m) ? d[base + j] : 0u;
        local += v[j];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_sums[lane];
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += t;
        }
        warp_sums[lane] = wi - w;
        if (lane == 31 && tile_sums) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_sums[wid] + incl - local;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < m) d[base + j] = run;
        run += v[j];
    }
}

__global__ void k_scan_add(uint32_t *__restrict__ d, int64_t m, const uint32_t *__restrict__ tile_off)
{
    int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    uint32_t add = tile_off[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j, i += kScanThreads)
        if (i < m) d[i] += add;
}

// ------------------------------------------------------------------------------------------
// LSD radix sort, 8-bit digits: per-tile digit histograms, a global exclusive scan laid out
// digit-major, then a stable scatter that ranks keys inside a tile with warp matching.
// ------------------------------------------------------------------------------------------
constexpr int kSortThreads = 256, kSortItems = 16, kSortTile = kSortThreads * kSortItems;

__global__ void k_sort_hist(const uint64_t *__restrict__ keys, int n, int shift, unsigned dmask,
                            uint32_t *__restrict__ counts, int n_tiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        int i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & dmask], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_sort_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                               uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int n, int shift,
                               unsigned dmask, const uint32_t *__restrict__ offsets, int n_tiles)
{
    __shared__ uint32_t wc[kSortThreads / 32][256];
    __shared__ uint32_t run[256];
    int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    run[tid] = offsets[(int64_t)tid * n_tiles + blockIdx.x];
    int base = blockIdx.x * kSortTile;
    unsigned lt_mask = (1u << lane) - 1u;
    for (int it = 0; it < kSortItems; ++it) {
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) wc[w][tid] = 0;
        __syncthreads();
        int i = base + it * kSortThreads + tid;
        bool valid = i < n;
        uint64_t k = valid ? kin[i] : 0ull;
        uint32_t v = valid ? vin[i] : 0u;
        unsigned digit = (unsigned)(k >> shift) & dmask;
        unsigned vmask = __ballot_sync(0xffffffffu, valid);
        unsigned rank = 0;
        if (valid) {
            unsigned peers = __match_any_sync(vmask, digit);
            rank = __popc(peers & lt_mask);
            if (rank == 0) wc[wid][digit] = __popc(peers);
        }
        __syncthreads();
        {
            uint32_t acc = run[tid];
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                uint32_t c = wc[w][tid];
                wc[w][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wc[wid][digit] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}

struct SortTemp {
    size_t off_keys, off_vals, off_counts, off_scan, total;
};

SortTemp sort_layout(int64_t n)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    int n_tiles = std::max(1, grtx_div_up(n, kSortTile));
    SortTemp t;
    t.off_keys = 0;
    t.off_vals = al(t.off_keys + (size_t)n * 8);
    t.off_counts = al(t.off_vals + (size_t)n * 4);
    t.off_scan = al(t.off_counts + (size_t)256 * n_tiles * 4);
    t.total = al(t.off_scan + grtx_scan_temp_bytes((int64_t)256 * n_tiles));
    return t;
}

int sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits, void *temp, cudaStream_t s)
{
    if (n <= 1) return GRTX_OK;
    SortTemp L = sort_layout(n);
    char *t = (char *)temp;
    uint64_t *k_alt = (uint64_t *)(t + L.off_keys);
    uint32_t *v_alt = (uint32_t *)(t + L.off_vals);
    uint32_t *counts = (uint32_t *)(t + L.off_counts);
    void *scan_tmp = t + L.off_scan;
    int n_tiles = grtx_div_up(n, kSortTile);
    int passes = (key_bits + 7) / 8;
    uint64_t *kin = keys, *kout = k_alt;
    uint32_t *vin = vals, *vout = v_alt;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        int bits = std::min(8, key_bits - shift);            // the last digit may be narrower
        unsigned dmask = (1u << bits) - 1u;
        k_sort_hist<<<n_tiles, kSortThreads, 0, s>>>(kin, (int)n, shift, dmask, counts, n_tiles);
        int st = grtx_scan_exclusive(counts, (int64_t)256 * n_tiles, scan_tmp, s);
        if (st != GRTX_OK) return st;
        k_sort_scatter<<<n_tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, (int)n, shift, dmask, counts, n_tiles);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    GRTX_CHECK_LAUNCH("radix sort");
    if (kin != keys) {
        GRTX_CUDA(cudaMemcpyAsync(keys, kin, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        GRTX_CUDA(cudaMemcpyAsync(vals, vin, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return GRTX_OK;
}

// ------------------------------------------------------------------------------------------
// Binary radix tree (Karras 2012) and bottom-up bounds.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int rt_delta(const uint64_t *__restrict__ k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    uint64_t a = k[i], b = k[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((unsigned)i ^ (unsigned)j));
}

__global__ void k_radix_tree(const uint64_t *__restrict__ k, int n, uint32_t *__restrict__ left,
                             uint32_t *__restrict__ right, uint32_t *__restrict__ parent)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (rt_delta(k, n, i, i + 1) - rt_delta(k, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = rt_delta(k, n, i, i - d);
    int lmax = 2;
    while (rt_delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (rt_delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = rt_delta(k, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        int t = (l + div - 1) / div;
        if (rt_delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    int gamma = i + s * d + min(d, 0);
    uint32_t L = (min(i, j) == gamma) ? (GRTX_LEAF | (uint32_t)gamma) : (uint32_t)gamma;
    uint32_t R = (max(i, j) == gamma + 1) ? (GRTX_LEAF | (uint32_t)(gamma + 1)) : (uint32_t)(gamma + 1);
    left[i] = L;
    right[i] = R;
    parent[(L & GRTX_LEAF) ? (n - 1 + (L & ~GRTX_LEAF)) : L] = (uint32_t)i;
    parent[(R & GRTX_LEAF) ? (n - 1 + (R & ~GRTX_LEAF)) : R] = (uint32_t)i;
    if (i == 0) parent[0] = GRTX_NONE;
}

__device__ __forceinline__ void load_box(uint32_t ref, const float *__restrict__ leaf_aabb,
                                         const float *node_aabb, float b[6])
{
    if (ref & GRTX_LEAF) {
        const float *p = leaf_aabb + 6 * (size_t)(ref & ~GRTX_LEAF);
        for (int c = 0; c < 6; ++c) b[c] = p[c];
    } else {
        const float *p = node_aabb + 6 * (size_t)ref;
        for (int c = 0; c < 6; ++c) b[c] = __ldcg(p + c);   // written by another thread: bypass L1
    }
}

__device__ __forceinline__ float load_slack(uint32_t ref, const float *__restrict__ leaf_slack, const float *node_slack)
{
    return (ref & GRTX_LEAF) ? leaf_slack[ref & ~GRTX_LEAF] : __ldcg(node_slack + ref);
}

// leaf_slack / node_slack (optional): a per-leaf scalar propagated as the maximum over each
// subtree (the proxy form's largest proxy diameter).
__global__ void k_refit(const uint32_t *__restrict__ left, const uint32_t *__restrict__ right,
                        const uint32_t *__restrict__ parent, const float *__restrict__ leaf_aabb, int n,
                        float *node_aabb, uint32_t *counters, const float *__restrict__ leaf_slack = nullptr,
                        float *node_slack = nullptr)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t node = parent[n - 1 + j];
    while (node != GRTX_NONE) {
        __threadfence();
        if (atomicAdd(&counters[node], 1u) == 0u) return;   // the sibling subtree is not done yet
        __threadfence();
        float a[6], b[6];
        load_box(left[node], leaf_aabb, node_aabb, a);
        load_box(right[node], leaf_aabb, node_aabb, b);
        float *out = node_aabb + 6 * (size_t)node;
        for (int c = 0; c < 3; ++c) {
            __stcg(out + c, fminf(a[c], b[c]));
            __stcg(out + 3 + c, fmaxf(a[3 + c], b[3 + c]));
        }
        if (node_slack)
            __stcg(node_slack + node, fmaxf(load_slack(left[node], leaf_slack, node_slack),
                                            load_slack(right[node], leaf_slack, node_slack)));
        node = parent[node];
    }
}

__global__ void k_depth(const uint32_t *__restrict__ parent, int n, int *__restrict__ max_depth)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int d = 0;
    uint32_t node = parent[n - 1 + j];
    while (node != GRTX_NONE && d < 100000) { ++d; node = parent[node]; }
    atomicMax(max_depth, d);
}

// BVH2 node: child 0 box, child 1 box, child refs (see grtx_scene_export).
__global__ void k_emit_nodes(const uint32_t *__restrict__ left, const uint32_t *__restrict__ right,
                             const float *__restrict__ leaf_aabb, const float *__restrict__ node_aabb, int n,
                             float4 *__restrict__ nodes, const float *__restrict__ leaf_slack,
                             const float *__restrict__ node_slack)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    float a[6], b[6];
    uint32_t L = left[i], R = right[i];
    load_box(L, leaf_aabb, node_aabb, a);
    load_box(R, leaf_aabb, node_aabb, b);
    nodes[4 * (size_t)i + 0] = make_float4(a[0], a[1], a[2], a[3]);
    nodes[4 * (size_t)i + 1] = make_float4(a[4], a[5], b[0], b[1]);
    nodes[4 * (size_t)i + 2] = make_float4(b[2], b[3], b[4], b[5]);
    float s0 = 0.f, s1 = 0.f;
    if (leaf_slack) {
        s0 = load_slack(L, leaf_slack, node_slack);
        s1 = load_slack(R, leaf_slack, node_slack);
    }
    nodes[4 * (size_t)i + 3] = make_float4(__uint_as_float(L), __uint_as_float(R), s0, s1);
}

// ------------------------------------------------------------------------------------------
// 4-wide nodes (bvh_width 4; the paper traverses a 6-wide BVH, Sec. V-A): every binary node at
// even depth becomes a node over its grandchildren (a child that is a leaf is kept as a leaf),
// so the 4-wide tree has half the depth and the same leaves. Node layout, 8 float4: lo x, lo y,
// lo z, hi x, hi y, hi z of the four children, the four child refs (bit 31: leaf slot; else a
// 4-wide node index; GRTX_NONE: empty, with an empty box), padding.
// ------------------------------------------------------------------------------------------
__global__ void k_bin_parents(const float4 *__restrict__ nodes, int n_int, uint32_t *__restrict__ parent)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const float4 r = nodes[4 * (size_t)i + 3];
    const uint32_t c[2] = {__float_as_uint(r.x), __float_as_uint(r.y)};
    for (int j = 0; j < 2; ++j)
        if (c[j] != GRTX_NONE && !(c[j] & GRTX_LEAF) && c[j] < (uint32_t)n_int) parent[c[j]] = (uint32_t)i;
}

__global__ void k_even_depth(const uint32_t *__restrict__ parent, int n_int, uint32_t *__restrict__ flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int d = 0;
    uint32_t node = (uint32_t)i;
    while (parent[node] != GRTX_NONE && d < (1 << 20)) {
        node = parent[node];
        ++d;
    }
    flag[i] = (d & 1) == 0;
}

// Quantised child boxes (bvh_quantize): per axis a lower corner o and a power-of-two step
// 2^e, and per child an 8-bit lower and upper coordinate q such that o + q * 2^e (one FMA in
// FP32, as the trace decodes it) lies below the child's lower face and above its upper face.
__device__ void quantise_axis(const float lo[4], const float hi[4], const bool used[4], float &o, uint32_t &eb,
                              uint32_t &qlo, uint32_t &qhi)
{
    float nlo = __int_as_float(0x7f800000), nhi = __int_as_float(0xff800000);
    for (int j = 0; j < 4; ++j)
        if (used[j]) {
            nlo = fminf(nlo, lo[j]);
            nhi = fmaxf(nhi, hi[j]);
        }
    o = nlo;
    int e = -126;
    const float r = (nhi - nlo) / 250.0f;
    if (r > 0.0f) {
        int ex;
        frexpf(r, &ex);                               // r < 2^ex
        e = max(-126, min(127, ex));
    }
    qlo = qhi = 0;
    for (;;) {
        const float st = __int_as_float((e + 127) << 23);
        bool fits = true;
        uint32_t ql = 0, qh = 0;
        for (int j = 0; j < 4; ++j) {
            int a, b;
            if (!used[j]) {                           // empty child: an empty decoded box
                a = 255;
                b = 0;
            } else {
                a = (int)floorf((lo[j] - o) / st);
                b = (int)ceilf((hi[j] - o) / st);
                a = max(0, min(255, a));
                b = max(0, min(255, b));
                while (a > 0 && fmaf((float)a, st, o) > lo[j]) --a;
                while (b < 255 && fmaf((float)b, st, o) < hi[j]) ++b;
                if (fmaf((float)a, st, o) > lo[j] || fmaf((float)b, st, o) < hi[j]) fits = false;
            }
            ql |= (uint32_t)a << (8 * j);
            qh |= (uint32_t)b << (8 * j);
        }
        if (fits || e >= 127) {
            qlo = ql;
            qhi = qh;
            break;
        }
        ++e;                                          // rounding pushed a face past 255 steps
    }
    eb = (uint32_t)(e + 127);
}

__global__ void k_emit_nodes4(const float4 *__restrict__ nodes, int n_int, const uint32_t *__restrict__ flag,
                              const uint32_t *__restrict__ idx, float4 *__restrict__ nodes4, int quant)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || !flag[i]) return;
    float b[6][4];
    uint32_t ref[4];
    for (int j = 0; j < 4; ++j) {
        b[0][j] = b[1][j] = b[2][j] = __int_as_float(0x7f800000);      // empty box: lo = +inf,
        b[3][j] = b[4][j] = b[5][j] = __int_as_float(0xff800000);      // hi = -inf
        ref[j] = GRTX_NONE;
    }
    int m = 0;
    // child c of binary node nd: its box (lo xyz, hi xyz) and ref
    auto child = [&](uint32_t nd, int c, float box[6], uint32_t &r) {
        const float4 n0 = nodes[4 * (size_t)nd], n1 = nodes[4 * (size_t)nd + 1], n2 = nodes[4 * (size_t)nd + 2];
        const float4 n3 = nodes[4 * (size_t)nd + 3];
        if (c == 0) {
            box[0] = n0.x; box[1] = n0.y; box[2] = n0.z; box[3] = n0.w; box[4] = n1.x; box[5] = n1.y;
            r = __float_as_uint(n3.x);
        } else {
            box[0] = n1.z; box[1] = n1.w; box[2] = n2.x; box[3] = n2.y; box[4] = n2.z; box[5] = n2.w;
            r = __float_as_uint(n3.y);
        }
    };
    auto add = [&](const float box[6], uint32_t r) {
        for (int k = 0; k < 6; ++k) b[k][m] = box[k];
        ref[m] = r;
        ++m;
    };
    for (int c = 0; c < 2; ++c) {
        float box[6];
        uint32_t r;
        child((uint32_t)i, c, box, r);
        if (r == GRTX_NONE) continue;
        if (r & GRTX_LEAF) {
            add(box, r);
            continue;
        }
        for (int g = 0; g < 2; ++g) {                // grandchildren: at even depth again
            float gb[6];
            uint32_t gr;
            child(r, g, gb, gr);
            if (gr == GRTX_NONE) continue;
            add(gb, (gr & GRTX_LEAF) ? gr : idx[gr]);
        }
    }
    if (quant) {
        // 64 bytes: (o x, o y, o z, steps as exponent bytes), then the 8-bit coordinates
        // (lo x, lo y, lo z, hi x | hi y, hi z) of the four children, then the four refs
        bool used[4];
        for (int j = 0; j < 4; ++j) used[j] = ref[j] != GRTX_NONE;
        float o[3];
        uint32_t eb[3], ql[3], qh[3];
        for (int a = 0; a < 3; ++a) quantise_axis(b[a], b[3 + a], used, o[a], eb[a], ql[a], qh[a]);
        float4 *out = nodes4 + 4 * (size_t)idx[i];
        out[0] = make_float4(o[0], o[1], o[2], __uint_as_float(eb[0] | (eb[1] << 8) | (eb[2] << 16)));
        out[1] = make_float4(__uint_as_float(ql[0]), __uint_as_float(ql[1]), __uint_as_float(ql[2]),
                             __uint_as_float(qh[0]));
        out[2] = make_float4(__uint_as_float(qh[1]), __uint_as_float(qh[2]), __uint_as_float(ref[0]),
                             __uint_as_float(ref[1]));
        out[3] = make_float4(__uint_as_float(ref[2]), __uint_as_float(ref[3]), 0.f, 0.f);
        return;
    }
    float4 *out = nodes4 + 8 * (size_t)idx[i];
    for (int k = 0; k < 6; ++k) out[k] = make_float4(b[k][0], b[k][1], b[k][2], b[k][3]);
    out[6] = make_float4(__uint_as_float(ref[0]), __uint_as_float(ref[1]), __uint_as_float(ref[2]),
                         __uint_as_float(ref[3]));
    out[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Refit for new parameters of the same Gaussians: the record, appearance and box of the
// Gaussian gid[s] at every leaf slot s < n_valid are recomputed in place; the Gaussians culled
// at build time (gid[n_valid..n)) only set *revived when one of them is now above alpha_min.
__global__ void k_refit_records(const float *__restrict__ means, const float *__restrict__ log_scales,
                                const float *__restrict__ quats, const float *__restrict__ logits,
                                const float *__restrict__ sh, int n_sh, int app_stride,
                                const uint32_t *__restrict__ gid, int64_t n_valid, int64_t n, float alpha_min,
                                float4 *__restrict__ geom, float *__restrict__ leaf_aabb, float *__restrict__ app,
                                float4 *__restrict__ raw, unsigned *__restrict__ revived)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t j = gid[s];
    if (s < n_valid) {
        prep_one(means, log_scales, quats, logits, j, alpha_min, geom + 4 * s, leaf_aabb + 6 * s);
        pack_raw(means, log_scales, quats, logits, j, raw + 3 * s);
        const float *src = sh + (size_t)j * n_sh;
        float *dst = app + (size_t)s * app_stride;
        for (int c = 0; c < app_stride; ++c) dst[c] = c < n_sh ? src[c] : 0.f;
    } else if (gaussian_opacity(logits, j) > alpha_min) {
        atomicOr(revived, 1u);
    }
}

// Left / right / parent arrays in the radix tree's layout (internal nodes 0..n-2, leaf j at
// n - 1 + j, the root's parent GRTX_NONE) read back from the compacted nodes of a tree over
// n >= 2 leaves.
__global__ void k_unpack_tree(const float4 *__restrict__ nodes, int n, uint32_t *__restrict__ left,
                              uint32_t *__restrict__ right, uint32_t *__restrict__ parent)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    float4 r = nodes[4 * (size_t)i + 3];
    uint32_t L = __float_as_uint(r.x), R = __float_as_uint(r.y);
    left[i] = L;
    right[i] = R;
    uint32_t pl = (L & GRTX_LEAF) ? (uint32_t)(n - 1) + (L & ~GRTX_LEAF) : L;
    uint32_t pr = (R & GRTX_LEAF) ? (uint32_t)(n - 1) + (R & ~GRTX_LEAF) : R;
    if (pl < (uint32_t)(2 * n - 1)) parent[pl] = (uint32_t)i;
    if (pr < (uint32_t)(2 * n - 1)) parent[pr] = (uint32_t)i;
    if (i == 0) parent[0] = GRTX_NONE;
}

// ------------------------------------------------------------------------------------------
// Locally-ordered clustering (PLOC; Meister and Bittner, IEEE TVCG 2018) over boxes in Morton
// order: each iteration every cluster finds its nearest neighbour (smallest union surface
// area, ties to the lower index) within kPlocRadius places, mutual pairs merge into a new
// node, and the clusters are compacted. The globally closest pair is always mutual, so every
// iteration merges at least one pair.
// ------------------------------------------------------------------------------------------
constexpr int kPlocBlock = 256;
constexpr int kPlocRadius = GRTX_PLOC_RADIUS;
constexpr int kPlocBatch = 8;              // rounds between host checks once few clusters are left
constexpr int kPlocBatchBelow = 65536;     // "few": below this many clusters

// Surface area of the union of two boxes, 2 (ex ey + ey ez + ez ex) with every operation
// rounded as written (no contraction), so that both members of a pair see the same value.
__device__ __forceinline__ float ploc_area(const float *a, const float *b)
{
    float e0 = __fsub_rn(fmaxf(a[3], b[3]), fminf(a[0], b[0]));
    float e1 = __fsub_rn(fmaxf(a[4], b[4]), fminf(a[1], b[1]));
    float e2 = __fsub_rn(fmaxf(a[5], b[5]), fminf(a[2], b[2]));
    float s = __fmul_rn(e0, e1);
    s = __fadd_rn(s, __fmul_rn(e1, e2));
    s = __fadd_rn(s, __fmul_rn(e2, e0));
    return __fmul_rn(2.0f, s);
}

// Device loop state of the clustering: [0] clusters left m, [1] nodes made, [2] rounds run,
// [3] error (a round that made no progress or made too many nodes). A round with m <= 1 does
// nothing, so several rounds can be enqueued between host checks.
enum { kPlocM = 0, kPlocMade = 1, kPlocRounds = 2, kPlocErr = 3 };

__global__ void k_ploc_init(uint32_t *__restrict__ id, int n, int *__restrict__ st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = GRTX_LEAF | (uint32_t)i;
    if (i == 0) {
        st[kPlocM] = n;
        st[kPlocMade] = 0;
        st[kPlocRounds] = 0;
        st[kPlocErr] = 0;
    }
}

__global__ void __launch_bounds__(kPlocBlock) k_ploc_nn(const float *__restrict__ cb, const int *__restrict__ st,
                                                        int *__restrict__ nn)
{
    __shared__ float sb[(kPlocBlock + 2 * kPlocRadius) * 6];
    const int m = st[kPlocM];
    if (m <= 1) return;
    const int b0 = blockIdx.x * kPlocBlock;
    if (b0 >= m) return;
    for (int t = threadIdx.x; t < (kPlocBlock + 2 * kPlocRadius) * 6; t += blockDim.x) {
        int g = b0 - kPlocRadius + t / 6;
        sb[t] = (g >= 0 && g < m) ? cb[6 * (size_t)g + t % 6] : 0.f;
    }
    __syncthreads();
    int i = b0 + threadIdx.x;
    if (i >= m) return;
    const float *me = sb + 6 * (threadIdx.x + kPlocRadius);
    int lo = max(i - kPlocRadius, 0), hi = min(i + kPlocRadius, m - 1);
    float best = INFINITY;
    int bj = -1;
    for (int j = lo; j <= hi; ++j) {
        if (j == i) continue;
        float a = ploc_area(me, sb + 6 * (j - b0 + kPlocRadius));
        if (a < best) {                       // ascending j: a tie keeps the lower index
            best = a;
            bj = j;
        }
    }
    nn[i] = bj;
}

// create[i]: cluster i starts a merge (mutual pair, i the lower); keep[i]: cluster i survives
// (as itself or as the merged node); tail: the two flags of the last cluster.
__global__ void k_ploc_flags(const int *__restrict__ nn, const int *__restrict__ st, uint32_t *__restrict__ create,
                             uint32_t *__restrict__ keep, uint32_t *__restrict__ tail)
{
    const int m = st[kPlocM];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (m <= 1 || i >= m) return;
    int j = nn[i];
    bool mutual = j >= 0 && nn[j] == i;
    uint32_t c = mutual && i < j, k = !(mutual && j < i);
    create[i] = c;
    keep[i] = k;
    if (i == m - 1) {
        tail[0] = c;
        tail[1] = k;
    }
}

// The round's totals (nodes created, clusters kept) and the next loop state, with the progress
// checks: every round must merge at least one pair and keep exactly m - created clusters.
__global__ void k_ploc_advance(const uint32_t *__restrict__ create_off, const uint32_t *__restrict__ keep_off,
                               const uint32_t *__restrict__ tail, int n, int *__restrict__ st)
{
    const int m = st[kPlocM];
    if (m <= 1 || st[kPlocErr]) return;
    const uint32_t created = create_off[m - 1] + tail[0];
    const uint32_t kept = keep_off[m - 1] + tail[1];
    const int made = st[kPlocMade];
    if (created == 0 || (int64_t)kept != (int64_t)m - created || (int64_t)made + created > n - 1) {
        st[kPlocErr] = 1;
        st[kPlocM] = 1;                       // stop the enqueued rounds
        return;
    }
    st[kPlocMade] = made + (int)created;
    st[kPlocM] = (int)kept;
    st[kPlocRounds] += 1;
}

__global__ void k_ploc_merge(const float *__restrict__ cb, const uint32_t *__restrict__ id, const int *__restrict__ nn,
                             const uint32_t *__restrict__ create_off, const uint32_t *__restrict__ keep_off,
                             const int *__restrict__ st, float *__restrict__ cb_out, uint32_t *__restrict__ id_out,
                             uint32_t *__restrict__ lc, uint32_t *__restrict__ rc)
{
    const int m = st[kPlocM];
    const uint32_t node_base = (uint32_t)st[kPlocMade];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (m <= 1 || i >= m) return;
    int j = nn[i];
    bool mutual = j >= 0 && nn[j] == i;
    if (mutual && j < i) return;              // merged into cluster j
    size_t w = keep_off[i];
    if (mutual) {
        uint32_t k = node_base + create_off[i];
        lc[k] = id[i];
        rc[k] = id[j];
        for (int c = 0; c < 3; ++c) {
            cb_out[6 * w + c] = fminf(cb[6 * (size_t)i + c], cb[6 * (size_t)j + c]);
            cb_out[6 * w + 3 + c] = fmaxf(cb[6 * (size_t)i + 3 + c], cb[6 * (size_t)j + 3 + c]);
        }
        id_out[w] = k;
    } else {
        for (int c = 0; c < 6; ++c) cb_out[6 * w + c] = cb[6 * (size_t)i + c];
        id_out[w] = id[i];
    }
}

// Node created k-th -> internal node n - 2 - k (the root, created last, is 0), with parents.
__global__ void k_ploc_finish(const uint32_t *__restrict__ lc, const uint32_t *__restrict__ rc, int n,
                              uint32_t *__restrict__ left, uint32_t *__restrict__ right, uint32_t *__restrict__ parent)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n - 1) return;
    uint32_t dst = (uint32_t)(n - 2 - k);
    uint32_t L = lc[k], R = rc[k];
    L = (L & GRTX_LEAF) ? L : (uint32_t)(n - 2) - L;
    R = (R & GRTX_LEAF) ? R : (uint32_t)(n - 2) - R;
    left[dst] = L;
    right[dst] = R;
    parent[(L & GRTX_LEAF) ? (n - 1 + (L & ~GRTX_LEAF)) : L] = dst;
    parent[(R & GRTX_LEAF) ? (n - 1 + (R & ~GRTX_LEAF)) : R] = dst;
    if (dst == 0) parent[0] = GRTX_NONE;
}

// ------------------------------------------------------------------------------------------
// Depth-first renumbering of a tree's internal nodes (pre-order: a node, then its left
// subtree, then its right subtree), so that every subtree occupies a contiguous range of the
// node array and a parent sits next to its left child.
// ------------------------------------------------------------------------------------------
__global__ void k_subtree_sizes(const uint32_t *__restrict__ left, const uint32_t *__restrict__ right,
                                const uint32_t *__restrict__ parent, int n, uint32_t *size, uint32_t *counters)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t node = parent[n - 1 + j];
    while (node != GRTX_NONE) {
        __threadfence();
        if (atomicAdd(&counters[node], 1u) == 0u) return;   // the sibling subtree is not done yet
        __threadfence();
        uint32_t L = left[node], R = right[node];
        uint32_t sl = (L & GRTX_LEAF) ? 0u : __ldcg(size + L);
        uint32_t sr = (R & GRTX_LEAF) ? 0u : __ldcg(size + R);
        __stcg(size + node, 1u + sl + sr);
        node = parent[node];
    }
}

// max_depth bounds the walk to the root (a clustering tree is no deeper than its rounds).
__global__ void k_preorder(const uint32_t *__restrict__ left, const uint32_t *__restrict__ parent,
                           const uint32_t *__restrict__ size, int n, int max_depth, uint32_t *__restrict__ pre)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n - 1) return;
    uint32_t idx = 0, c = (uint32_t)v;
    for (int guard = 0; guard <= max_depth; ++guard) {
        uint32_t p = parent[c];
        if (p == GRTX_NONE) break;
        uint32_t L = left[p];
        idx += 1u + ((L == c) ? 0u : ((L & GRTX_LEAF) ? 0u : size[L]));
        c = p;
    }
    pre[v] = idx;
}

__global__ void k_permute_tree(const uint32_t *__restrict__ left, const uint32_t *__restrict__ right,
                               const uint32_t *__restrict__ pre, int n, uint32_t *__restrict__ left_out,
                               uint32_t *__restrict__ right_out, uint32_t *__restrict__ parent_out)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n - 1) return;
    uint32_t d = pre[v];
    uint32_t L = left[v], R = right[v];
    L = (L & GRTX_LEAF) ? L : pre[L];
    R = (R & GRTX_LEAF) ? R : pre[R];
    left_out[d] = L;
    right_out[d] = R;
    parent_out[(L & GRTX_LEAF) ? (n - 1 + (L & ~GRTX_LEAF)) : L] = d;
    parent_out[(R & GRTX_LEAF) ? (n - 1 + (R & ~GRTX_LEAF)) : R] = d;
    if (d == 0) parent_out[0] = GRTX_NONE;
}

// One-leaf scene: a root whose second child is an empty box that no ray hits.
__global__ void k_emit_single(const float *__restrict__ leaf_aabb, float4 *__restrict__ nodes)
{
    const float *a = leaf_aabb;
    nodes[0] = make_float4(a[0], a[1], a[2], a[3]);
    nodes[1] = make_float4(a[4], a[5], INFINITY, INFINITY);
    nodes[2] = make_float4(INFINITY, -INFINITY, -INFINITY, -INFINITY);
    nodes[3] = make_float4(__uint_as_float(GRTX_LEAF | 0u), __uint_as_float(GRTX_NONE), 0.f, 0.f);
}

__global__ void k_count_valid(const uint64_t *codes, int64_t n, unsigned long long *out)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += codes[i] != ~0ull;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ------------------------------------------------------------------------------------------
// Leaf-order gather of Gaussian records and appearance.
// ------------------------------------------------------------------------------------------
__global__ void k_gather_gaussians(const uint32_t *__restrict__ order, int64_t n_valid,
                                   const float4 *__restrict__ geom_in, const float *__restrict__ aabb_in,
                                   const float *__restrict__ sh, int n_sh, int app_stride,
                                   const float *__restrict__ means, const float *__restrict__ log_scales,
                                   const float *__restrict__ quats, const float *__restrict__ logits,
                                   float4 *__restrict__ geom, float *__restrict__ aabb,
                                   float *__restrict__ app, uint32_t *__restrict__ gid, float4 *__restrict__ raw)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_valid) return;
    uint32_t i = order[s];
    for (int r = 0; r < 4; ++r) geom[4 * s + r] = geom_in[4 * (size_t)i + r];
    for (int c = 0; c < 6; ++c) aabb[6 * s + c] = aabb_in[6 * (size_t)i + c];
    const float *src = sh + (size_t)i * n_sh;
    float *dst = app + (size_t)s * app_stride;
    for (int c = 0; c < app_stride; ++c) dst[c] = c < n_sh ? src[c] : 0.f;
    gid[s] = i;
    pack_raw(means, log_scales, quats, logits, i, raw + 3 * s);
}

// ------------------------------------------------------------------------------------------
// Proxy form: 20-triangle icosahedron around each Gaussian (Sec. III-C Observation I).
// ------------------------------------------------------------------------------------------
__constant__ float c_ico_v[12][3];
__constant__ int c_ico_f[20][3];

__global__ void k_proxy_expand(const float4 *__restrict__ geom_sorted, const float *__restrict__ means,
                               const float *__restrict__ log_scales, const float *__restrict__ quats,
                               const uint32_t *__restrict__ gid, int64_t n_valid, float ico_circ,
                               float4 *__restrict__ tris, float *__restrict__ tri_aabb, float *__restrict__ tri_slack)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_valid) return;
    uint32_t i = gid[s];
    float4 g3 = geom_sorted[4 * s + 3];
    float kap = sqrtf(-2.0f * g3.y / 1.4426950408889634f);
    float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float sc[3] = {expf(log_scales[3 * i]) * kap, expf(log_scales[3 * i + 1]) * kap,
                   expf(log_scales[3 * i + 2]) * kap};
    float w = quats[4 * i], x = quats[4 * i + 1], y = quats[4 * i + 2], z = quats[4 * i + 3];
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                     {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                     {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    // every point of the proxy lies within kappa * max(s) * circumradius of the mean
    float diam = 2.0f * ico_circ * fmaxf(sc[0], fmaxf(sc[1], sc[2])) * (1.0f + 1e-4f);
    float V[12][3];
    for (int v = 0; v < 12; ++v)
        for (int a = 0; a < 3; ++a)
            V[v][a] = mu[a] + R[a][0] * sc[0] * c_ico_v[v][0] + R[a][1] * sc[1] * c_ico_v[v][1] +
                      R[a][2] * sc[2] * c_ico_v[v][2];
    for (int f = 0; f < 20; ++f) {
        const float *p0 = V[c_ico_f[f][0]], *p1 = V[c_ico_f[f][1]], *p2 = V[c_ico_f[f][2]];
        size_t t = (size_t)s * 20 + f;
        tris[3 * t + 0] = make_float4(p0[0], p0[1], p0[2], __uint_as_float((uint32_t)s));
        tris[3 * t + 1] = make_float4(p1[0], p1[1], p1[2], 0.f);
        tris[3 * t + 2] = make_float4(p2[0], p2[1], p2[2], 0.f);
        tri_slack[t] = diam;
        float *bb = tri_aabb + 6 * t;
        for (int a = 0; a < 3; ++a) {
            float lo = fminf(p0[a], fminf(p1[a], p2[a])), hi = fmaxf(p0[a], fmaxf(p1[a], p2[a]));
            float pad = 1e-6f * (hi - lo) + 1e-7f * fabsf(lo) + 1e-7f * fabsf(hi);
            bb[a] = lo - pad;
            bb[3 + a] = hi + pad;
        }
    }
}

__global__ void k_gather_tris(const uint32_t *__restrict__ order, int64_t n, const float4 *__restrict__ tin,
                              const float *__restrict__ ain, const float *__restrict__ slack_in,
                              const uint32_t *__restrict__ gid, float4 *__restrict__ tout, float *__restrict__ aout,
                              float *__restrict__ slack_out, uint32_t *__restrict__ leaf_ids)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t src = order[t];
    slack_out[t] = slack_in[src];
    for (int r = 0; r < 3; ++r) tout[3 * t + r] = tin[3 * (size_t)src + r];
    for (int c = 0; c < 6; ++c) aout[6 * t + c] = ain[6 * (size_t)src + c];
    leaf_ids[t] = gid[__float_as_uint(tin[3 * (size_t)src].w)];
}

bool g_ico_ready[64] = {};   // proxy mesh uploaded to this device's constant memory
float g_ico_circ = 0.f;   // circumradius of the uploaded proxy in unit-sphere units

int upload_icosahedron(cudaStream_t s)
{
    // Regular icosahedron from the cyclic permutations of (0, +-1, +-phi), scaled so that its
    // inradius is 1 + 1e-3: it encloses the unit sphere with a margin for FP32 rounding.
    const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
    std::vector<std::array<double, 3>> v;
    for (int s1 = -1; s1 <= 1; s1 += 2)
        for (int s2 = -1; s2 <= 1; s2 += 2) {
            v.push_back({0.0, (double)s1, s2 * phi});
            v.push_back({(double)s1, s2 * phi, 0.0});
            v.push_back({s2 * phi, 0.0, (double)s1});
        }
    // faces: vertex triples that are pairwise at the edge length 2
    std::vector<std::array<int, 3>> f;
    auto d2 = [&](int a, int b) {
        double s = 0;
        for (int c = 0; c < 3; ++c) s += (v[a][c] - v[b][c]) * (v[a][c] - v[b][c]);
        return s;
    };
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            for (int c = b + 1; c < 12; ++c)
                if (std::fabs(d2(a, b) - 4) < 1e-9 && std::fabs(d2(b, c) - 4) < 1e-9 && std::fabs(d2(a, c) - 4) < 1e-9)
                    f.push_back({a, b, c});
    if (f.size() != 20) return grtx_fail(GRTX_ERR_CUDA, "icosahedron face enumeration failed");
    // inradius of this icosahedron: distance from the origin to a face plane
    const double* p0 = v[f[0][0]].data(); const double* p1 = v[f[0][1]].data(); const double* p2 = v[f[0][2]].data();
    double e1[3], e2[3], nrm[3];
    for (int c = 0; c < 3; ++c) { e1[c] = p1[c] - p0[c]; e2[c] = p2[c] - p0[c]; }
    nrm[0] = e1[1] * e2[2] - e1[2] * e2[1]; nrm[1] = e1[2] * e2[0] - e1[0] * e2[2]; nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double nl = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    double inr = std::fabs(nrm[0] * p0[0] + nrm[1] * p0[1] + nrm[2] * p0[2]) / nl;
    static float hv[12][3];   // static: the async copies below read them after return
    static int hf[20][3];
    for (int a = 0; a < 12; ++a)
        for (int c = 0; c < 3; ++c) hv[a][c] = (float)(v[a][c] * (1.0 + 1e-3) / inr);
    g_ico_circ = (float)(std::sqrt(1.0 + phi * phi) * (1.0 + 1e-3) / inr);
    for (int a = 0; a < 20; ++a)
        for (int c = 0; c < 3; ++c) hf[a][c] = f[a][c];
    GRTX_CUDA(cudaMemcpyToSymbolAsync(c_ico_v, hv, sizeof(hv), 0, cudaMemcpyHostToDevice, s));
    GRTX_CUDA(cudaMemcpyToSymbolAsync(c_ico_f, hf, sizeof(hf), 0, cudaMemcpyHostToDevice, s));
    return GRTX_OK;
}

// ------------------------------------------------------------------------------------------
// Stream-ordered allocation helper.
// ------------------------------------------------------------------------------------------
struct Alloc {
    cudaStream_t s;
    std::vector<void *> tmp;
    explicit Alloc(cudaStream_t st) : s(st) {}
    template <class T>
    int get(T **p, size_t count, bool temp)
    {
        size_t bytes = std::max<size_t>(count * sizeof(T), 16);
        int st = grtx_malloc_async((void **)p, bytes, s);
        if (st) return st;
        if (temp) tmp.push_back(*p);
        return GRTX_OK;
    }
    ~Alloc()
    {
        for (void *p : tmp) cudaFreeAsync(p, s);
    }
};

#define TRY(x)                         \
    do {                               \
        int st__ = (x);                \
        if (st__ != GRTX_OK) return st__; \
    } while (0)

void free_scene_arrays(grtx_scene *sc)
{
    cudaStream_t s = sc->stream;
    void *ptrs[] = {sc->nodes, sc->nodes4, sc->geom, sc->tris, sc->app, sc->raw, sc->gid, sc->leaf_ids, sc->codes,
                    sc->ws, sc->d_counter};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, s);
}

// Morton -> sort -> radix tree -> refit -> nodes over n leaf boxes (sorted in place with
// `order`). Writes sc->nodes, sc->codes, sc->depth.
int build_tree(grtx_scene *sc, Alloc &A, float *leaf_aabb, int64_t n, uint32_t *order, uint64_t *codes,
               float *bounds_dev, int code_kind)
{
    cudaStream_t s = sc->stream;
    int blocks = grtx_div_up(n, kThreads);
    k_init_bounds<<<1, 32, 0, s>>>(bounds_dev);
    k_centroid_bounds<<<std::min(blocks, 4096), kThreads, 0, s>>>(leaf_aabb, n, bounds_dev);
    if (code_kind == GRTX_CODES_CENTROID)
        k_morton<<<blocks, kThreads, 0, s>>>(leaf_aabb, n, bounds_dev, codes, order);
    else
        k_morton_sized<<<blocks, kThreads, 0, s>>>(leaf_aabb, n, bounds_dev, codes, order);
    GRTX_CHECK_LAUNCH("morton");
    void *stmp;
    TRY(A.get((char **)&stmp, sort_layout(n).total, true));
    TRY(sort_pairs(codes, order, n, 64, stmp, s));
    return GRTX_OK;
}

// PLOC tree over n >= 2 boxes in order: left/right/parent in the radix tree's layout. The loop
// state lives on the device (k_ploc_advance). The host reads it after every round while many
// clusters are left (a round then costs far more than the round trip), and after every
// kPlocBatch rounds once few are left, each launch sized by the last count it read (an upper
// bound; rounds after the last do nothing). Every round merges at least one pair, so at most
// n - 1 rounds make progress; a round that does not fails the build.
int ploc_tree(Alloc &A, const float *leaf_aabb, int64_t n, uint32_t *left, uint32_t *right, uint32_t *parent,
              cudaStream_t s, int *iterations)
{
    float *cb[2];
    uint32_t *id[2], *create, *keep, *lc, *rc, *small;
    int *nn, *st;
    void *scan_tmp;
    TRY(A.get(&cb[0], 6 * (size_t)n, true));
    TRY(A.get(&cb[1], 6 * (size_t)n, true));
    TRY(A.get(&id[0], n, true));
    TRY(A.get(&id[1], n, true));
    TRY(A.get(&nn, n, true));
    TRY(A.get(&create, n, true));
    TRY(A.get(&keep, n, true));
    TRY(A.get(&lc, n - 1, true));
    TRY(A.get(&rc, n - 1, true));
    TRY(A.get(&small, 4, true));
    TRY(A.get(&st, 4, true));
    TRY(A.get((char **)&scan_tmp, grtx_scan_temp_bytes(n), true));
    GRTX_CUDA(cudaMemcpyAsync(cb[0], leaf_aabb, sizeof(float) * 6 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    k_ploc_init<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(id[0], (int)n, st);
    int64_t m = n;                            // clusters left as last read by the host
    int cur = 0, checks = 0;
    int h[4] = {(int)n, 0, 0, 0};
    while (m > 1) {
        if (++checks > n) return grtx_fail(GRTX_ERR_OVERFLOW_FATAL, "clustering did not converge");
        const int rounds = m > kPlocBatchBelow ? 1 : kPlocBatch;
        const int blocks = grtx_div_up(m, kPlocBlock);
        for (int r = 0; r < rounds; ++r) {
            k_ploc_nn<<<blocks, kPlocBlock, 0, s>>>(cb[cur], st, nn);
            k_ploc_flags<<<blocks, kPlocBlock, 0, s>>>(nn, st, create, keep, small);
            TRY(grtx_scan_exclusive(create, m, scan_tmp, s));
            TRY(grtx_scan_exclusive(keep, m, scan_tmp, s));
            k_ploc_merge<<<blocks, kPlocBlock, 0, s>>>(cb[cur], id[cur], nn, create, keep, st, cb[cur ^ 1],
                                                       id[cur ^ 1], lc, rc);
            k_ploc_advance<<<1, 1, 0, s>>>(create, keep, small, (int)n, st);
            cur ^= 1;
        }
        GRTX_CHECK_LAUNCH("clustering");
        GRTX_CUDA(cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
        GRTX_CUDA(cudaStreamSynchronize(s));
        if (h[kPlocErr]) return grtx_fail(GRTX_ERR_OVERFLOW_FATAL, "clustering made no progress");
        if ((int64_t)h[kPlocM] >= m) return grtx_fail(GRTX_ERR_OVERFLOW_FATAL, "clustering made no progress");
        m = h[kPlocM];
    }
    if (h[kPlocMade] != n - 1) return grtx_fail(GRTX_ERR_OVERFLOW_FATAL, "clustering made a wrong number of nodes");
    k_ploc_finish<<<grtx_div_up(n - 1, kThreads), kThreads, 0, s>>>(lc, rc, (int)n, left, right, parent);
    GRTX_CHECK_LAUNCH("clustering finish");
    if (iterations) *iterations = h[kPlocRounds];
    return GRTX_OK;
}

int finish_tree(grtx_scene *sc, Alloc &A, const float *leaf_aabb_sorted, int64_t n, int builder,
                const float *leaf_slack = nullptr)
{
    cudaStream_t s = sc->stream;
    int64_t n_nodes = std::max<int64_t>(n - 1, 1);
    TRY(A.get(&sc->nodes, (size_t)n_nodes * 4, false));
    sc->n_nodes = n_nodes;
    int *d_depth;
    TRY(A.get(&d_depth, 1, true));
    GRTX_CUDA(cudaMemsetAsync(d_depth, 0, sizeof(int), s));
    if (n == 1) {
        k_emit_single<<<1, 1, 0, s>>>(leaf_aabb_sorted, sc->nodes);
    } else {
        uint32_t *left, *right, *parent, *cnt;
        float *node_aabb, *node_slack = nullptr;
        if (leaf_slack) TRY(A.get(&node_slack, n - 1, true));
        TRY(A.get(&left, n - 1, true));
        TRY(A.get(&right, n - 1, true));
        TRY(A.get(&parent, 2 * n - 1, true));
        TRY(A.get(&cnt, n - 1, true));
        TRY(A.get(&node_aabb, 6 * (n - 1), true));
        GRTX_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (n - 1), s));
        if (builder == GRTX_BUILDER_PLOC) {
            // clustering numbers nodes by creation round, scattering subtrees over the array:
            // renumber them depth-first for locality
            uint32_t *l0, *r0, *p0, *sz, *pre;
            TRY(A.get(&l0, n - 1, true));
            TRY(A.get(&r0, n - 1, true));
            TRY(A.get(&p0, 2 * n - 1, true));
            TRY(A.get(&sz, n - 1, true));
            TRY(A.get(&pre, n - 1, true));
            int rounds = 0;
            TRY(ploc_tree(A, leaf_aabb_sorted, n, l0, r0, p0, s, &rounds));
            k_subtree_sizes<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(l0, r0, p0, (int)n, sz, cnt);
            k_preorder<<<grtx_div_up(n - 1, kThreads), kThreads, 0, s>>>(l0, p0, sz, (int)n, rounds, pre);
            k_permute_tree<<<grtx_div_up(n - 1, kThreads), kThreads, 0, s>>>(l0, r0, pre, (int)n, left, right, parent);
            GRTX_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (n - 1), s));
            GRTX_CHECK_LAUNCH("depth-first renumbering");
        } else {
            k_radix_tree<<<grtx_div_up(n - 1, kThreads), kThreads, 0, s>>>(sc->codes, (int)n, left, right, parent);
        }
        k_refit<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(left, right, parent, leaf_aabb_sorted, (int)n,
                                                              node_aabb, cnt, leaf_slack, node_slack);
        k_depth<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(parent, (int)n, d_depth);
        k_emit_nodes<<<grtx_div_up(n - 1, kThreads), kThreads, 0, s>>>(left, right, leaf_aabb_sorted, node_aabb,
                                                                       (int)n, sc->nodes, leaf_slack, node_slack);
        GRTX_CHECK_LAUNCH("radix tree / refit");
    }
    int h_depth = 0;
    GRTX_CUDA(cudaMemcpyAsync(&h_depth, d_depth, sizeof(int), cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaStreamSynchronize(s));
    sc->depth = n == 1 ? 1 : h_depth;
    return GRTX_OK;
}

// World bounds of all leaves = union of the root's two child boxes (h_root: the root node).
void set_bounds(grtx_scene *sc, const float *h_root)
{
    for (int c = 0; c < 3; ++c) {
        sc->bounds[c] = std::min(h_root[c], h_root[6 + c]);
        sc->bounds[3 + c] = std::max(h_root[3 + c], h_root[9 + c]);
    }
}

// Build (or, after a refit, rebuild in place) the 4-wide nodes from the binary ones.
int collapse_wide(grtx_scene *sc, cudaStream_t s)
{
    if (sc->n_valid == 0 || sc->n_nodes == 0) return GRTX_OK;
    Alloc A(s);
    const int n_int = (int)sc->n_nodes;
    uint32_t *parent, *flag, *idx;
    char *temp;
    TRY(A.get(&parent, n_int, true));
    TRY(A.get(&flag, n_int, true));
    TRY(A.get(&idx, n_int, true));
    TRY(A.get(&temp, grtx_scan_temp_bytes(n_int), true));
    GRTX_CUDA(cudaMemsetAsync(parent, 0xff, sizeof(uint32_t) * n_int, s));
    k_bin_parents<<<grtx_div_up(n_int, kThreads), kThreads, 0, s>>>(sc->nodes, n_int, parent);
    k_even_depth<<<grtx_div_up(n_int, kThreads), kThreads, 0, s>>>(parent, n_int, flag);
    GRTX_CHECK_LAUNCH("4-wide collapse: depth parity");
    GRTX_CUDA(cudaMemcpyAsync(idx, flag, sizeof(uint32_t) * n_int, cudaMemcpyDeviceToDevice, s));
    TRY(grtx_scan_exclusive(idx, n_int, temp, s));
    uint32_t h_last[2] = {0, 0};
    GRTX_CUDA(cudaMemcpyAsync(&h_last[0], idx + n_int - 1, 4, cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaMemcpyAsync(&h_last[1], flag + n_int - 1, 4, cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaStreamSynchronize(s));
    const int64_t n4 = (int64_t)h_last[0] + h_last[1];
    if (!sc->nodes4 || n4 != sc->n_nodes4) {
        if (sc->nodes4) cudaFreeAsync(sc->nodes4, s);
        sc->nodes4 = nullptr;
        sc->n_nodes4 = 0;
        TRY(A.get(&sc->nodes4, (sc->bvh_quant ? 4 : 8) * (size_t)n4, false));
        sc->n_nodes4 = n4;
    }
    k_emit_nodes4<<<grtx_div_up(n_int, kThreads), kThreads, 0, s>>>(sc->nodes, n_int, flag, idx, sc->nodes4,
                                                                    sc->bvh_quant);
    GRTX_CHECK_LAUNCH("4-wide collapse: nodes");
    return GRTX_OK;
}

int build_scene(const grtx_gaussians *g, const grtx_params *p, int form, grtx_scene *sc)
{
    cudaStream_t s = sc->stream;
    Alloc A(s);
    int64_t n = g->n;
    sc->n = n;
    sc->form = form;
    sc->sh_degree = g->sh_degree;
    sc->n_coef = (g->sh_degree + 1) * (g->sh_degree + 1);
    int n_sh = sc->n_coef * 3;
    sc->app_stride = (n_sh + 3) & ~3;
    sc->alpha_min = p->alpha_min;
    sc->bvh_codes = p->bvh_codes;
    sc->bvh_builder = p->bvh_builder;
    sc->bvh_width = p->bvh_width == 4 ? 4 : 2;
    sc->bvh_quant = sc->bvh_width == 4 && p->bvh_quantize ? 1 : 0;
    TRY(A.get(&sc->d_counter, 8, false));
    GRTX_CUDA(cudaMemsetAsync(sc->d_counter, 0, 8 * sizeof(unsigned), s));
    if (n == 0) {
        sc->n_valid = sc->n_leaves = 0;
        sc->n_nodes = 0;
        return GRTX_OK;
    }
    float4 *geom_raw;
    float *aabb_raw, *bounds_dev;
    uint64_t *codes;
    uint32_t *order;
    TRY(A.get(&geom_raw, 4 * n, true));
    TRY(A.get(&aabb_raw, 6 * n, true));
    TRY(A.get(&bounds_dev, 6, true));
    TRY(A.get(&codes, n, true));
    TRY(A.get(&order, n, true));
    int blocks = grtx_div_up(n, kThreads);
    k_prep<<<blocks, kThreads, 0, s>>>(g->means, g->log_scales, g->quats, g->opacity_logits, n, p->alpha_min,
                                       geom_raw, aabb_raw);
    GRTX_CHECK_LAUNCH("prep");
    TRY(build_tree(sc, A, aabb_raw, n, order, codes, bounds_dev, p->bvh_codes));
    // number of valid Gaussians: their codes sort before the 2^64-1 of the empty boxes
    unsigned long long *d_nvalid;
    TRY(A.get(&d_nvalid, 1, true));
    GRTX_CUDA(cudaMemsetAsync(d_nvalid, 0, 8, s));
    k_count_valid<<<std::min(blocks, 4096), kThreads, 0, s>>>(codes, n, d_nvalid);
    unsigned long long h_nvalid = 0;
    GRTX_CUDA(cudaMemcpyAsync(&h_nvalid, d_nvalid, 8, cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaStreamSynchronize(s));
    int64_t nv = (int64_t)h_nvalid;
    sc->n_valid = nv;
    if (nv == 0) {
        sc->n_leaves = 0;
        sc->n_nodes = 0;
        return GRTX_OK;
    }
    float *leaf_aabb;
    TRY(A.get(&sc->geom, 4 * nv, false));
    TRY(A.get(&sc->app, (size_t)sc->app_stride * nv, false));
    TRY(A.get(&sc->gid, n, false));                 // leaf slots, then the culled Gaussians
    TRY(A.get(&sc->raw, 3 * nv, false));
    TRY(A.get(&leaf_aabb, 6 * nv, true));
    k_gather_gaussians<<<grtx_div_up(nv, kThreads), kThreads, 0, s>>>(order, nv, geom_raw, aabb_raw, g->sh, n_sh,
                                                                      sc->app_stride, g->means, g->log_scales,
                                                                      g->quats, g->opacity_logits, sc->geom,
                                                                      leaf_aabb, sc->app, sc->gid, sc->raw);
    GRTX_CHECK_LAUNCH("gather");
    if (n > nv)
        GRTX_CUDA(cudaMemcpyAsync(sc->gid + nv, order + nv, (size_t)(n - nv) * 4, cudaMemcpyDeviceToDevice, s));
    if (form != GRTX_FORM_PROXY20) {       // sphere and icosphere forms: one leaf per Gaussian
        if (form != GRTX_FORM_SPHERE) TRY(grtx_template_blas(form, &sc->tpl_nodes, &sc->tpl_tris));
        sc->n_leaves = nv;
        TRY(A.get(&sc->codes, nv, false));
        GRTX_CUDA(cudaMemcpyAsync(sc->codes, codes, (size_t)nv * 8, cudaMemcpyDeviceToDevice, s));
        TRY(A.get(&sc->leaf_ids, nv, false));
        GRTX_CUDA(cudaMemcpyAsync(sc->leaf_ids, sc->gid, (size_t)nv * 4, cudaMemcpyDeviceToDevice, s));
        TRY(finish_tree(sc, A, leaf_aabb, nv, p->bvh_builder));
    } else {
        int dev = 0;
        GRTX_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return grtx_fail(GRTX_ERR_INVALID_ARG, "device ordinal out of range");
        if (!g_ico_ready[dev]) {
            TRY(upload_icosahedron(s));
            g_ico_ready[dev] = true;
        }
        int64_t nt = 20 * nv;
        if (nt >= (int64_t)1 << 31) return grtx_fail(GRTX_ERR_INVALID_ARG, "too many proxy triangles");
        float4 *tris_raw;
        float *tri_aabb_raw, *tri_aabb, *slack_raw, *slack;
        uint64_t *tcodes;
        uint32_t *torder;
        TRY(A.get(&tris_raw, 3 * nt, true));
        TRY(A.get(&tri_aabb_raw, 6 * nt, true));
        TRY(A.get(&slack_raw, nt, true));
        TRY(A.get(&slack, nt, true));
        TRY(A.get(&tcodes, nt, true));
        TRY(A.get(&torder, nt, true));
        k_proxy_expand<<<grtx_div_up(nv, kThreads), kThreads, 0, s>>>(sc->geom, g->means, g->log_scales, g->quats,
                                                                      sc->gid, nv, g_ico_circ, tris_raw,
                                                                      tri_aabb_raw, slack_raw);
        GRTX_CHECK_LAUNCH("proxy expand");
        TRY(build_tree(sc, A, tri_aabb_raw, nt, torder, tcodes, bounds_dev, p->bvh_codes));
        sc->n_leaves = nt;
        TRY(A.get(&sc->tris, 3 * nt, false));
        TRY(A.get(&tri_aabb, 6 * nt, true));
        TRY(A.get(&sc->leaf_ids, nt, false));
        k_gather_tris<<<grtx_div_up(nt, kThreads), kThreads, 0, s>>>(torder, nt, tris_raw, tri_aabb_raw, slack_raw,
                                                                     sc->gid, sc->tris, tri_aabb, slack, sc->leaf_ids);
        GRTX_CHECK_LAUNCH("gather triangles");
        TRY(A.get(&sc->codes, nt, false));
        GRTX_CUDA(cudaMemcpyAsync(sc->codes, tcodes, (size_t)nt * 8, cudaMemcpyDeviceToDevice, s));
        TRY(finish_tree(sc, A, tri_aabb, nt, p->bvh_builder, slack));
    }
    float h_root[16];
    GRTX_CUDA(cudaMemcpyAsync(h_root, sc->nodes, sizeof(h_root), cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaStreamSynchronize(s));
    set_bounds(sc, h_root);
    if (sc->depth >= GRTX_STACK)
        return grtx_fail(GRTX_ERR_OVERFLOW_FATAL, "BVH depth " + std::to_string(sc->depth) +
                                                      " exceeds the traversal stack");
    if (sc->bvh_width == 4) TRY(collapse_wide(sc, s));
    return GRTX_OK;
}

// Refit of a sphere- or icosphere-form scene with n_valid >= 1 for new parameters of the same
// Gaussians: topology and leaf order kept, records / appearance / leaf boxes recomputed, node
// boxes refitted bottom-up. *revived reports a build-time-culled Gaussian that is now valid
// (the caller then rebuilds). One host round trip (flag and root box).
int refit_scene(const grtx_gaussians *g, grtx_scene *sc, cudaStream_t s, bool *revived)
{
    Alloc A(s);
    int64_t n = sc->n, nv = sc->n_valid;
    unsigned *d_flag;
    float *leaf_aabb;
    TRY(A.get(&d_flag, 1, true));
    TRY(A.get(&leaf_aabb, 6 * nv, true));
    uint32_t *left = nullptr, *right = nullptr, *parent = nullptr, *cnt = nullptr;
    float *node_aabb = nullptr;
    if (nv >= 2) {
        TRY(A.get(&left, nv - 1, true));
        TRY(A.get(&right, nv - 1, true));
        TRY(A.get(&parent, 2 * nv - 1, true));
        TRY(A.get(&cnt, nv - 1, true));
        TRY(A.get(&node_aabb, 6 * (nv - 1), true));
    }
    GRTX_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(unsigned), s));
    k_refit_records<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(
        g->means, g->log_scales, g->quats, g->opacity_logits, g->sh, sc->n_coef * 3, sc->app_stride, sc->gid, nv, n,
        sc->alpha_min, sc->geom, leaf_aabb, sc->app, sc->raw, d_flag);
    if (nv == 1) {
        k_emit_single<<<1, 1, 0, s>>>(leaf_aabb, sc->nodes);
    } else {
        k_unpack_tree<<<grtx_div_up(nv - 1, kThreads), kThreads, 0, s>>>(sc->nodes, (int)nv, left, right, parent);
        GRTX_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (nv - 1), s));
        k_refit<<<grtx_div_up(nv, kThreads), kThreads, 0, s>>>(left, right, parent, leaf_aabb, (int)nv, node_aabb,
                                                               cnt);
        k_emit_nodes<<<grtx_div_up(nv - 1, kThreads), kThreads, 0, s>>>(left, right, leaf_aabb, node_aabb, (int)nv,
                                                                        sc->nodes, nullptr, nullptr);
    }
    GRTX_CHECK_LAUNCH("refit");
    if (sc->bvh_width == 4) TRY(collapse_wide(sc, s));
    unsigned h_flag = 0;
    float h_root[16];
    GRTX_CUDA(cudaMemcpyAsync(&h_flag, d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaMemcpyAsync(h_root, sc->nodes, sizeof(h_root), cudaMemcpyDeviceToHost, s));
    GRTX_CUDA(cudaStreamSynchronize(s));
    *revived = h_flag != 0;
    set_bounds(sc, h_root);
    return GRTX_OK;
}

// Full rebuild with the scene's form, alpha_min, codes and builder; the new arrays replace the
// old ones (freed stream-ordered on s), the trace workspace is kept.
int rebuild_scene(const grtx_gaussians *g, grtx_scene *sc, cudaStream_t s)
{
    grtx_params p;
    std::memset(&p, 0, sizeof(p));
    p.alpha_min = sc->alpha_min;
    p.bvh_codes = sc->bvh_codes;
    p.bvh_builder = sc->bvh_builder;
    p.bvh_width = sc->bvh_width;
    p.bvh_quantize = sc->bvh_quant;
    grtx_scene *ns = new (std::nothrow) grtx_scene();
    if (!ns) return grtx_fail(GRTX_ERR_OOM, "host allocation failed");
    ns->stream = s;
    int st = build_scene(g, &p, sc->form, ns);
    if (st != GRTX_OK) {
        free_scene_arrays(ns);
        cudaStreamSynchronize(s);
        delete ns;
        return st;
    }
    void *ws = sc->ws;
    size_t ws_bytes = sc->ws_bytes;
    sc->ws = nullptr;
    sc->stream = s;
    free_scene_arrays(sc);
    *sc = *ns;
    sc->ws = ws;
    sc->ws_bytes = ws_bytes;
    delete ns;
    return GRTX_OK;
}

}  // namespace

size_t grtx_scan_temp_bytes(int64_t m)
{
    size_t total = 0;
    while (m > kScanTile) {
        m = (m + kScanTile - 1) / kScanTile;
        total += ((size_t)m * 4 + 255) & ~(size_t)255;
    }
    return total + 256;
}

int grtx_scan_exclusive(uint32_t *d, int64_t m, void *temp, cudaStream_t s)
{
    if (m <= 0) return GRTX_OK;
    if (m <= kScanTile) {
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(d, m, nullptr);
        return GRTX_OK;
    }
    int64_t tiles = (m + kScanTile - 1) / kScanTile;
    uint32_t *sums = (uint32_t *)temp;
    char *rest = (char *)temp + (((size_t)tiles * 4 + 255) & ~(size_t)255);
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(d, m, sums);
    int st = grtx_scan_exclusive(sums, tiles, rest, s);
    if (st != GRTX_OK) return st;
    k_scan_add<<<(unsigned)tiles, kScanThreads, 0, s>>>(d, m, sums);
    return GRTX_OK;
}

// ------------------------------------------------------------------------------------------
// ABI entry points of the build.
// ------------------------------------------------------------------------------------------
static int check_gaussians(const grtx_gaussians *g)
{
    if (!g) return grtx_fail(GRTX_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0 || g->n >= ((int64_t)1 << 31)) return grtx_fail(GRTX_ERR_INVALID_ARG, "n out of range");
    if (g->sh_degree < 0 || g->sh_degree > 3) return grtx_fail(GRTX_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "a parameter array is NULL");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_prep_gaussians(const grtx_gaussians *g, float alpha_min, float *d_geom, float *d_aabb,
                                            void *stream)
{
    int st = check_gaussians(g);
    if (st) return st;
    if (!(alpha_min > 0.f && alpha_min < 1.f)) return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_min must be in (0,1)");
    if (g->n == 0) return GRTX_OK;
    if (!d_geom || !d_aabb || ((uintptr_t)d_geom & 15)) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad output pointer");
    k_prep<<<grtx_div_up(g->n, kThreads), kThreads, 0, S(stream)>>>(g->means, g->log_scales, g->quats,
                                                                     g->opacity_logits, g->n, alpha_min,
                                                                     (float4 *)d_geom, d_aabb);
    GRTX_CHECK_LAUNCH("grtx_prep_gaussians");
    return GRTX_OK;
}

static int morton_codes_abi(const float *d_aabb, int64_t n, const float *d_bounds, float *d_bounds_out,
                            uint64_t *d_codes, void *stream, bool sized)
{
    if (n < 0 || n >= ((int64_t)1 << 31)) return grtx_fail(GRTX_ERR_INVALID_ARG, "n out of range");
    if (n == 0) return GRTX_OK;
    if (!d_aabb || !d_codes) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    cudaStream_t s = S(stream);
    const float *bounds = d_bounds;
    float *tmp = nullptr;
    if (!bounds) {
        float *b = d_bounds_out;
        if (!b) {
            int st = grtx_malloc_async((void **)&tmp, 6 * sizeof(float), s);
            if (st) return st;
            b = tmp;
        }
        k_init_bounds<<<1, 32, 0, s>>>(b);
        k_centroid_bounds<<<std::min(grtx_div_up(n, kThreads), 4096), kThreads, 0, s>>>(d_aabb, n, b);
        bounds = b;
    }
    if (sized)
        k_morton_sized<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(d_aabb, n, bounds, d_codes, nullptr);
    else
        k_morton<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(d_aabb, n, bounds, d_codes, nullptr);
    if (tmp) cudaFreeAsync(tmp, s);
    GRTX_CHECK_LAUNCH(sized ? "grtx_morton_codes_sized" : "grtx_morton_codes");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_morton_codes(const float *d_aabb, int64_t n, const float *d_bounds, float *d_bounds_out,
                                          uint64_t *d_codes, void *stream)
{
    return morton_codes_abi(d_aabb, n, d_bounds, d_bounds_out, d_codes, stream, false);
}

extern "C" GRTX_API int grtx_morton_codes_sized(const float *d_aabb, int64_t n, const float *d_bounds,
                                                float *d_bounds_out, uint64_t *d_codes, void *stream)
{
    return morton_codes_abi(d_aabb, n, d_bounds, d_bounds_out, d_codes, stream, true);
}

extern "C" GRTX_API int grtx_ploc_tree(const float *d_leaf_aabb, int64_t n, uint32_t *d_left, uint32_t *d_right,
                                       uint32_t *d_parent, int *iterations, void *stream)
{
    if (n < 2 || n >= ((int64_t)1 << 30)) return grtx_fail(GRTX_ERR_INVALID_ARG, "n must be in [2, 2^30)");
    if (!d_leaf_aabb || !d_left || !d_right || !d_parent) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    Alloc A(S(stream));
    return ploc_tree(A, d_leaf_aabb, n, d_left, d_right, d_parent, S(stream), iterations);
}

extern "C" GRTX_API int grtx_sort_pairs(uint64_t *d_keys, uint32_t *d_values, int64_t n, int key_bits, void *d_temp,
                                        size_t *temp_bytes, void *stream)
{
    if (!temp_bytes) return grtx_fail(GRTX_ERR_INVALID_ARG, "temp_bytes is NULL");
    if (n < 0 || n >= ((int64_t)1 << 31)) return grtx_fail(GRTX_ERR_INVALID_ARG, "n out of range");
    if (key_bits < 1 || key_bits > 64) return grtx_fail(GRTX_ERR_INVALID_ARG, "key_bits must be 1..64");
    size_t need = sort_layout(std::max<int64_t>(n, 1)).total;
    if (!d_temp) {
        *temp_bytes = need;
        return GRTX_OK;
    }
    if (*temp_bytes < need) return grtx_fail(GRTX_ERR_INVALID_ARG, "temp buffer too small");
    if (n > 1 && (!d_keys || !d_values)) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    return sort_pairs(d_keys, d_values, n, key_bits, d_temp, S(stream));
}

extern "C" GRTX_API int grtx_radix_tree(const uint64_t *d_sorted_keys, int64_t n, uint32_t *d_left, uint32_t *d_right,
                                        uint32_t *d_parent, void *stream)
{
    if (n < 2 || n >= ((int64_t)1 << 30)) return grtx_fail(GRTX_ERR_INVALID_ARG, "n must be in [2, 2^30)");
    if (!d_sorted_keys || !d_left || !d_right || !d_parent) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    k_radix_tree<<<grtx_div_up(n - 1, kThreads), kThreads, 0, S(stream)>>>(d_sorted_keys, (int)n, d_left, d_right,
                                                                             d_parent);
    GRTX_CHECK_LAUNCH("grtx_radix_tree");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_refit(const uint32_t *d_left, const uint32_t *d_right, const uint32_t *d_parent,
                                   const float *d_leaf_aabb, int64_t n, float *d_node_aabb, uint32_t *d_counters,
                                   void *stream)
{
    if (n < 2 || n >= ((int64_t)1 << 30)) return grtx_fail(GRTX_ERR_INVALID_ARG, "n must be in [2, 2^30)");
    if (!d_left || !d_right || !d_parent || !d_leaf_aabb || !d_node_aabb || !d_counters)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    cudaStream_t s = S(stream);
    GRTX_CUDA(cudaMemsetAsync(d_counters, 0, sizeof(uint32_t) * (n - 1), s));
    k_refit<<<grtx_div_up(n, kThreads), kThreads, 0, s>>>(d_left, d_right, d_parent, d_leaf_aabb, (int)n,
                                                           d_node_aabb, d_counters);
    GRTX_CHECK_LAUNCH("grtx_refit");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_build_bvh(const grtx_gaussians *g, const grtx_params *p, int form, void *stream,
                                       grtx_scene **out)
{
    int st = check_gaussians(g);
    if (st) return st;
    if (!p || !out) return grtx_fail(GRTX_ERR_INVALID_ARG, "params or out is NULL");
    if (form != GRTX_FORM_SPHERE && form != GRTX_FORM_PROXY20 && form != GRTX_FORM_ICO20 && form != GRTX_FORM_ICO80)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "unknown form");
    if (!(p->alpha_min > 0.f && p->alpha_min < 1.f)) return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_min must be in (0,1)");
    if (p->bvh_codes != GRTX_CODES_SIZED && p->bvh_codes != GRTX_CODES_CENTROID)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "unknown bvh_codes");
    if (p->bvh_builder != GRTX_BUILDER_PLOC && p->bvh_builder != GRTX_BUILDER_LBVH)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "unknown bvh_builder");
    if (p->bvh_width != 0 && p->bvh_width != 2 && p->bvh_width != 4)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "bvh_width must be 0, 2 or 4");
    if (p->bvh_width == 4 && form != GRTX_FORM_SPHERE)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "4-wide nodes are built for the sphere form only");
    if (p->bvh_quantize != 0 && (p->bvh_quantize != 1 || p->bvh_width != 4))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "bvh_quantize is 0, or 1 with bvh_width 4");
    grtx_scene *sc = new (std::nothrow) grtx_scene();
    if (!sc) return grtx_fail(GRTX_ERR_OOM, "host allocation failed");
    sc->stream = S(stream);
    st = build_scene(g, p, form, sc);
    if (st != GRTX_OK) {
        free_scene_arrays(sc);
        cudaStreamSynchronize(sc->stream);
        delete sc;
        return st;
    }
    *out = sc;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_scene_update(grtx_scene *sc, const grtx_gaussians *g, int mode, void *stream,
                                          int *rebuilt)
{
    if (rebuilt) *rebuilt = 0;
    if (!sc) return grtx_fail(GRTX_ERR_INVALID_ARG, "scene is NULL");
    int st = check_gaussians(g);
    if (st) return st;
    if (g->n != sc->n) return grtx_fail(GRTX_ERR_INVALID_ARG, "update needs the scene's number of Gaussians");
    if (g->sh_degree != sc->sh_degree) return grtx_fail(GRTX_ERR_INVALID_ARG, "update needs the scene's SH degree");
    if (mode != GRTX_UPDATE_REFIT && mode != GRTX_UPDATE_REBUILD)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "unknown update mode");
    if (mode == GRTX_UPDATE_REFIT && sc->form == GRTX_FORM_PROXY20)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "refit needs the sphere or an icosphere form (rebuild the proxy form)");
    cudaStream_t s = S(stream);
    sc->stream = s;
    if (mode == GRTX_UPDATE_REFIT && sc->n_valid > 0) {
        bool revived = false;
        st = refit_scene(g, sc, s, &revived);
        if (st != GRTX_OK || !revived) return st;
    }
    st = rebuild_scene(g, sc, s);
    if (st == GRTX_OK && rebuilt) *rebuilt = 1;
    return st;
}

extern "C" GRTX_API int grtx_scene_info_get(const grtx_scene *sc, grtx_scene_info *info)
{
    if (!sc || !info) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    std::memset(info, 0, sizeof(*info));
    info->n_gaussians = sc->n;
    info->n_valid = sc->n_valid;
    info->n_leaves = sc->n_leaves;
    info->n_nodes = sc->n_nodes;
    info->depth = sc->depth;
    info->form = sc->form;
    info->sh_degree = sc->sh_degree;
    info->bytes_nodes = sc->n_nodes * 64;
    info->bytes_leaves = (sc->form != GRTX_FORM_PROXY20 ? sc->n_valid * 64 : sc->n_leaves * 48 + sc->n_valid * 64) +
                         sc->n_valid * 48;      // + the raw parameters in leaf order
    info->bytes_appearance = sc->n_valid * sc->app_stride * 4;
    info->bytes_workspace = (int64_t)sc->ws_bytes;
    for (int c = 0; c < 6; ++c) info->bounds[c] = sc->bounds[c];
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_scene_export(const grtx_scene *sc, float *d_nodes, uint32_t *d_leaf_ids, uint64_t *d_codes,
                                          void *stream)
{
    if (!sc) return grtx_fail(GRTX_ERR_INVALID_ARG, "scene is NULL");
    cudaStream_t s = S(stream);
    if (d_nodes && sc->n_nodes)
        GRTX_CUDA(cudaMemcpyAsync(d_nodes, sc->nodes, (size_t)sc->n_nodes * 64, cudaMemcpyDeviceToDevice, s));
    if (d_leaf_ids && sc->n_leaves)
        GRTX_CUDA(cudaMemcpyAsync(d_leaf_ids, sc->leaf_ids, (size_t)sc->n_leaves * 4, cudaMemcpyDeviceToDevice, s));
    if (d_codes && sc->n_leaves)
        GRTX_CUDA(cudaMemcpyAsync(d_codes, sc->codes, (size_t)sc->n_leaves * 8, cudaMemcpyDeviceToDevice, s));
    return GRTX_OK;
}

extern "C" GRTX_API void grtx_scene_destroy(grtx_scene *sc)
{
    if (!sc) return;
    free_scene_arrays(sc);
    cudaStreamSynchronize(sc->stream);
    delete sc;
}
