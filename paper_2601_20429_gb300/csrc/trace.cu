// C-ABI entry points of the trace: argument checks, camera set-up, the per-slot workspace
// and the persistent launch (the kernels themselves are in trace_impl.cuh).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>

#include "trace_impl.cuh"

#define GRTX_EXTERN_TRACE(K)                                                                     \
    extern template int trace_launch<K>(const TraceArgs &, int, bool, int, int, cudaStream_t); \
    extern template int trace_occupancy<K>(int, bool, int, int *);
GRTX_EXTERN_TRACE(1)
GRTX_EXTERN_TRACE(2)
GRTX_EXTERN_TRACE(4)
GRTX_EXTERN_TRACE(8)
GRTX_EXTERN_TRACE(16)
GRTX_EXTERN_TRACE(32)

#define GRTX_EXTERN_SEGMENTS(K)                                                                          \
    extern template int serve_launch<K>(const TraceArgs &, const ServeSeg *, const unsigned *, int, int, cudaStream_t, \
                                        ServeLive);                                                                  \
    extern template int serve_occupancy<K>(int *);
GRTX_EXTERN_SEGMENTS(1)
GRTX_EXTERN_SEGMENTS(2)
GRTX_EXTERN_SEGMENTS(4)
GRTX_EXTERN_SEGMENTS(8)
GRTX_EXTERN_SEGMENTS(16)
GRTX_EXTERN_SEGMENTS(32)

int trace_single_launch(const TraceArgs &a, int form, bool instr, int blocks, cudaStream_t s);
int trace_single_occupancy(int form, bool instr, int *blocks_per_sm);

namespace {

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool valid_k(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32; }

int launch_k(int k, const TraceArgs &a, int form, bool instr, int pass, int blocks, cudaStream_t s)
{
    switch (k) {
    case 1: return trace_launch<1>(a, form, instr, pass, blocks, s);
    case 2: return trace_launch<2>(a, form, instr, pass, blocks, s);
    case 4: return trace_launch<4>(a, form, instr, pass, blocks, s);
    case 8: return trace_launch<8>(a, form, instr, pass, blocks, s);
    case 16: return trace_launch<16>(a, form, instr, pass, blocks, s);
    default: return trace_launch<32>(a, form, instr, pass, blocks, s);
    }
}

int occupancy_k(int k, int form, bool instr, int pass, int *bps)
{
    switch (k) {
    case 1: return trace_occupancy<1>(form, instr, pass, bps);
    case 2: return trace_occupancy<2>(form, instr, pass, bps);
    case 4: return trace_occupancy<4>(form, instr, pass, bps);
    case 8: return trace_occupancy<8>(form, instr, pass, bps);
    case 16: return trace_occupancy<16>(form, instr, pass, bps);
    default: return trace_occupancy<32>(form, instr, pass, bps);
    }
}

int check_params(const grtx_params *p)
{
    if (!p) return grtx_fail(GRTX_ERR_INVALID_ARG, "params is NULL");
    if (!valid_k(p->k)) return grtx_fail(GRTX_ERR_INVALID_ARG, "k must be one of 1, 2, 4, 8, 16, 32");
    if (p->traversal != GRTX_TRAVERSAL_CHECKPOINT && p->traversal != GRTX_TRAVERSAL_RESTART &&
        p->traversal != GRTX_TRAVERSAL_SINGLE)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "unknown traversal mode");
    if (!(p->T_min >= 0.f && p->T_min < 1.f)) return grtx_fail(GRTX_ERR_INVALID_ARG, "T_min must be in [0,1)");
    if (!(p->alpha_max > 0.f && p->alpha_max < 1.f)) return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_max must be in (0,1)");
    if (p->ckpt_capacity < 0 || p->evict_capacity < 0 || p->ckpt_capacity > 65536 || p->evict_capacity > 65536)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "capacities must be in [0, 65536]");
    if (p->packet_stack < 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "packet_stack must be >= 0");
    if (p->bvh_width != 0 && p->bvh_width != 2 && p->bvh_width != 4)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "bvh_width must be 0, 2 or 4");
    return GRTX_OK;
}

}  // namespace

int grtx_fill_camera(CamRef &a, unsigned &n_items_out, const grtx_camera *cam)
{
    if (!cam) return grtx_fail(GRTX_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width <= 0 || cam->height <= 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "camera size must be positive");
    if (!(cam->t_near >= 0.f) || !(cam->t_far > cam->t_near))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "need 0 <= t_near < t_far");
    a.cam_type = cam->type;
    a.width = cam->width;
    a.height = cam->height;
    a.t_near = cam->t_near;
    a.t_far = cam->t_far;
    int64_t n_items;
    if (cam->type == GRTX_CAMERA_RAYS) {
        if (!cam->ray_origins || !cam->ray_dirs) return grtx_fail(GRTX_ERR_INVALID_ARG, "ray buffers are NULL");
        a.ray_o = cam->ray_origins;
        a.ray_d = cam->ray_dirs;
        a.ray_tn = cam->ray_tnear;
        a.ray_tf = cam->ray_tfar;
        if (cam->height >= 4) {                 // an image of rays: traced in 8x4 tiles
            a.tiles_x = (cam->width + 7) / 8;
            n_items = (int64_t)a.tiles_x * ((cam->height + 3) / 4) * 32;
        } else {
            a.tiles_x = 0;
            n_items = ((int64_t)cam->width * cam->height + 31) / 32 * 32;
        }
    } else if (cam->type == GRTX_CAMERA_PINHOLE || cam->type == GRTX_CAMERA_FISHEYE) {
        if (!(cam->fov > 0.f) || (cam->type == GRTX_CAMERA_PINHOLE && !(cam->fov < 3.14159f)))
            return grtx_fail(GRTX_ERR_INVALID_ARG, "bad field of view");
        a.pos = make_float3(cam->pos[0], cam->pos[1], cam->pos[2]);
        a.right = make_float3(cam->right[0], cam->right[1], cam->right[2]);
        a.up = make_float3(cam->up[0], cam->up[1], cam->up[2]);
        a.fwd = make_float3(cam->forward[0], cam->forward[1], cam->forward[2]);
        a.tan_half = tanf(0.5f * cam->fov);
        a.aspect = (float)cam->width / (float)cam->height;
        a.fish_f = (0.5f * cam->width) / cam->fov;
        a.tiles_x = (cam->width + 7) / 8;
        int tiles_y = (cam->height + 3) / 4;
        n_items = (int64_t)a.tiles_x * tiles_y * 32;
    } else {
        return grtx_fail(GRTX_ERR_INVALID_ARG, "unknown camera type");
    }
    if (n_items >= ((int64_t)1 << 31)) return grtx_fail(GRTX_ERR_INVALID_ARG, "too many rays");
    n_items_out = (unsigned)n_items;
    return GRTX_OK;
}

namespace {

int fill_camera(TraceArgs &a, const grtx_camera *cam) { return grtx_fill_camera(a.cam, a.n_items, cam); }

// SM count of the current device (cached per device ordinal).
int sm_count()
{
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

// Per-slot lists (entries_per_slot uint2 per ray slot), grown on demand; returns the base.
int ensure_workspace(grtx_scene *sc, int n_slots, size_t entries_per_slot, cudaStream_t s, uint2 **base_out)
{
    size_t need = (size_t)n_slots * entries_per_slot * sizeof(uint2);
    if (need > sc->ws_bytes) {
        if (sc->ws) {
            GRTX_CUDA(cudaDeviceSynchronize());   // earlier traces on any stream may still use it
            GRTX_CUDA(cudaFreeAsync(sc->ws, s));
            sc->ws = nullptr;
            sc->ws_bytes = 0;
        }
        int st = grtx_malloc_async(&sc->ws, need, s);
        if (st) return st;
        sc->ws_bytes = need;
    }
    *base_out = (uint2 *)sc->ws;
    return GRTX_OK;
}

}  // namespace

SceneRef grtx_scene_ref(const grtx_scene *sc)
{
    SceneRef r;
    r.nodes = sc->nodes;
    r.geom = sc->geom;
    r.tris = sc->tris;
    r.app = sc->app;
    r.gid = sc->gid;
    r.tpl_nodes = sc->tpl_nodes;
    r.tpl_tris = sc->tpl_tris;
    r.raw = sc->raw;
    r.nodes4 = sc->nodes4;
    r.n_nodes4 = (uint32_t)sc->n_nodes4;
    r.app_stride = sc->app_stride;
    r.sh_degree = sc->sh_degree;
    r.has_tree = sc->n_valid > 0;
    r.n_nodes = (uint32_t)sc->n_nodes;
    r.n_leaves = (uint32_t)sc->n_leaves;
    r.n_geom = (uint32_t)sc->n_valid;
    return r;
}

int grtx_check_params(const grtx_params *p) { return check_params(p); }

namespace {

int setup(grtx_scene *sc, const grtx_camera *cam, const grtx_params *p, TraceArgs &a)
{
    if (!sc) return grtx_fail(GRTX_ERR_INVALID_ARG, "scene is NULL");
    int st = check_params(p);
    if (st) return st;
    if (p->alpha_min != sc->alpha_min)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_min differs from the one the scene was built with");
    st = fill_camera(a, cam);
    if (st) return st;
    a.sc = grtx_scene_ref(sc);
    a.traversal = p->traversal;
    a.T_min = p->T_min;
    a.alpha_max = p->alpha_max;
    a.bg0 = p->bg[0];
    a.bg1 = p->bg[1];
    a.bg2 = p->bg[2];
    a.ckpt_cap = p->ckpt_capacity > 0 ? p->ckpt_capacity
                 : (p->traversal == GRTX_TRAVERSAL_SINGLE ? GRTX_DEFAULT_SINGLE_CAPACITY : GRTX_DEFAULT_CKPT_CAPACITY);
    a.evict_cap = p->evict_capacity > 0 ? p->evict_capacity : GRTX_DEFAULT_EVICT_CAPACITY;
    a.packet_stack = p->packet_stack > 0 ? std::min(p->packet_stack, kPacketStack) : kPacketStack;
    return GRTX_OK;
}

int run(grtx_scene *sc, TraceArgs &a, int k, bool instr, int pass, unsigned *queue, cudaStream_t s, bool wide = false)
{
    int form = kernel_form(sc->form, wide, sc->bvh_quant != 0);
    bool single = a.traversal == GRTX_TRAVERSAL_SINGLE && pass == PASS_FWD;
    int bps = 0;
    int occ = single ? trace_single_occupancy(form, instr, &bps) : occupancy_k(k, form, instr, pass, &bps);
    if (occ != GRTX_OK || bps <= 0) return grtx_fail(GRTX_ERR_CUDA, "occupancy query failed");
    int blocks = sm_count() * bps;
    int n_slots = blocks * 128;
    bool ckpt = a.traversal == GRTX_TRAVERSAL_CHECKPOINT;
    // checkpoint: two ping-pong checkpoint lists and the eviction list; single: the hit list
    size_t C = ckpt ? a.ckpt_cap : 1, E = ckpt ? a.evict_cap : 1;
    size_t per_slot = single ? (size_t)a.ckpt_cap : 2 * C + E;
    uint2 *base = nullptr;
    int st = ensure_workspace(sc, n_slots, per_slot, s, &base);
    if (st) return st;
    a.ck0 = base;
    a.ck1 = single ? base : base + (size_t)n_slots * C;
    a.ev = single ? base : base + (size_t)n_slots * 2 * C;
    a.n_slots = n_slots;
    a.queue = queue;
    if (!set_list_offsets(a, per_slot))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "checkpoint/eviction capacities too large for the resident ray slots");
    a.discard = single ? 0 : lists_discardable(a);
    GRTX_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned), s));
    int launched = single ? trace_single_launch(a, form, instr, blocks, s)
                          : launch_k(k, a, form, instr, pass, blocks, s);
    if (launched != GRTX_OK) {
        cudaError_t e = cudaGetLastError();
        return grtx_cuda_fail(e == cudaSuccess ? cudaErrorLaunchFailure : e, "trace launch");
    }
    return GRTX_OK;
}

// Add the per-leaf staged gradients into the caller's arrays (one thread per leaf, so plain
// additions; the caller zeroed or holds earlier sums).
__global__ void k_scatter_grads(const float4 *__restrict__ stage, const uint32_t *__restrict__ gid, int64_t n,
                                float *g_means, float *g_log_scales, float *g_quats, float *g_logits)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const size_t i = gid[s];
    const float4 a = stage[3 * s], b = stage[3 * s + 1], c = stage[3 * s + 2];
    if (g_means) {
        g_means[3 * i] += a.x;
        g_means[3 * i + 1] += a.y;
        g_means[3 * i + 2] += a.z;
    }
    if (g_logits) g_logits[i] += a.w;
    if (g_log_scales) {
        g_log_scales[3 * i] += b.x;
        g_log_scales[3 * i + 1] += b.y;
        g_log_scales[3 * i + 2] += b.z;
    }
    if (g_quats) {
        g_quats[4 * i] += c.x;
        g_quats[4 * i + 1] += c.y;
        g_quats[4 * i + 2] += c.z;
        g_quats[4 * i + 3] += c.w;
    }
}

__global__ void k_gen_rays(CamRef a, float *o, float *d, float *tn, float *tf)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)a.width * a.height) return;
    unsigned item = item_of_pixel(a, p);
    int64_t pix;
    float3 ro, rd;
    float a0, a1;
    if (!make_ray(a, item, pix, ro, rd, a0, a1)) return;
    o[3 * pix] = ro.x; o[3 * pix + 1] = ro.y; o[3 * pix + 2] = ro.z;
    d[3 * pix] = rd.x; d[3 * pix + 1] = rd.y; d[3 * pix + 2] = rd.z;
    if (tn) tn[pix] = a0;
    if (tf) tf[pix] = a1;
}

}  // namespace

extern "C" GRTX_API int grtx_generate_rays(const grtx_camera *cam, float *d_origins, float *d_dirs, float *d_tnear,
                                           float *d_tfar, void *stream)
{
    TraceArgs a = {};
    int st = fill_camera(a, cam);
    if (st) return st;
    if (!d_origins || !d_dirs) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL output");
    int64_t n = (int64_t)cam->width * cam->height;
    k_gen_rays<<<grtx_div_up(n, 256), 256, 0, S(stream)>>>(a.cam, d_origins, d_dirs, d_tnear, d_tfar);
    GRTX_CHECK_LAUNCH("grtx_generate_rays");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_trace_forward(grtx_scene *sc, const grtx_camera *cam, const grtx_params *p,
                                           const grtx_trace_outputs *out, void *stream)
{
    TraceArgs a = {};
    int st = setup(sc, cam, p, a);
    if (st) return st;
    if (!out || !out->rgbT) return grtx_fail(GRTX_ERR_INVALID_ARG, "rgbT output is NULL");
    if (((uintptr_t)out->rgbT & 15) != 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "rgbT must be 16-byte aligned");
    if (out->blended_ids && out->ids_cap <= 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "ids_cap must be positive");
    if ((out->visits != nullptr) != (out->visits_n != nullptr))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "visits and visits_n go together");
    if (out->visits && (out->visits_cap <= 0 || out->visits_stride <= 0 || out->visits_rows <= 0))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "visits_cap, visits_stride and visits_rows must be positive");
    a.rgbT = (float4 *)out->rgbT;
    a.n_blended = out->n_blended;
    a.ids = out->blended_ids;
    a.ids_cap = out->ids_cap;
    a.stats = out->stats;
    a.visits = out->visits;
    a.visits_n = out->visits_n;
    a.visits_cap = out->visits_cap;
    a.visits_stride = out->visits_stride;
    a.visits_rows = out->visits_rows;
    cudaStream_t s = S(stream);
    bool instr = out->n_blended || out->blended_ids || out->stats || out->visits;
    int pass = PASS_FWD;
    if (out->saved) {
        const grtx_saved *sv = out->saved;
        if (!sv->leaves || !sv->n || sv->cap <= 0)
            return grtx_fail(GRTX_ERR_INVALID_ARG, "saved lists need leaves, n and a positive cap");
        if (sc->form != GRTX_FORM_SPHERE) return grtx_fail(GRTX_ERR_INVALID_ARG, "saved lists need the sphere form");
        if (instr || a.traversal == GRTX_TRAVERSAL_SINGLE)
            return grtx_fail(GRTX_ERR_INVALID_ARG,
                             "saved lists take checkpoint or restart traversal and no other optional output");
        a.save_leaves = sv->leaves;
        a.save_n = sv->n;
        a.save_cap = sv->cap;
        pass = PASS_SAVE;
    }
    const bool wide = p->bvh_width == 4;
    if (wide) {
        if (sc->bvh_width != 4 && sc->n_valid > 0)
            return grtx_fail(GRTX_ERR_INVALID_ARG, "bvh_width 4: the scene was built without 4-wide nodes");
        if (a.traversal == GRTX_TRAVERSAL_SINGLE || pass != PASS_FWD)
            return grtx_fail(GRTX_ERR_INVALID_ARG, "4-wide nodes take checkpoint or restart traversal, no saved lists");
    }
    if (out->visits) GRTX_CUDA(cudaMemsetAsync(out->visits_n, 0, (size_t)out->visits_rows * 4, s));
    if (out->blended_ids)
        GRTX_CUDA(cudaMemsetAsync(out->blended_ids, 0xff, (size_t)cam->width * cam->height * out->ids_cap * 4, s));
    return run(sc, a, p->k, instr, pass, sc->d_counter, s, wide);
}

namespace {

int segments_launch_k(int k, const TraceArgs &a, const ServeSeg *segs, const unsigned *begins, int n, int blocks, cudaStream_t s)
{
    switch (k) {
    case 1: return serve_launch<1>(a, segs, begins, n, blocks, s, ServeLive{});
    case 2: return serve_launch<2>(a, segs, begins, n, blocks, s, ServeLive{});
    case 4: return serve_launch<4>(a, segs, begins, n, blocks, s, ServeLive{});
    case 8: return serve_launch<8>(a, segs, begins, n, blocks, s, ServeLive{});
    case 16: return serve_launch<16>(a, segs, begins, n, blocks, s, ServeLive{});
    default: return serve_launch<32>(a, segs, begins, n, blocks, s, ServeLive{});
    }
}

int segments_occupancy_k(int k, int *bps)
{
    switch (k) {
    case 1: return serve_occupancy<1>(bps);
    case 2: return serve_occupancy<2>(bps);
    case 4: return serve_occupancy<4>(bps);
    case 8: return serve_occupancy<8>(bps);
    case 16: return serve_occupancy<16>(bps);
    default: return serve_occupancy<32>(bps);
    }
}

}  // namespace

extern "C" GRTX_API int grtx_trace_forward_batch(grtx_scene *sc, const grtx_camera *cams, int n_cams,
                                                 const grtx_params *p, float *const *rgbT, void *stream)
{
    if (!cams || !rgbT) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    if (n_cams < 1 || n_cams > GRTX_MAX_BATCH) return grtx_fail(GRTX_ERR_INVALID_ARG, "n_cams must be in [1, 64]");
    TraceArgs a = {};
    int st = setup(sc, &cams[0], p, a);
    if (st) return st;
    if (sc->form != GRTX_FORM_SPHERE) return grtx_fail(GRTX_ERR_INVALID_ARG, "batched traces need the sphere form");
    if (a.traversal == GRTX_TRAVERSAL_SINGLE)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "batched traces take checkpoint or restart traversal");
    ServeSeg v[GRTX_MAX_BATCH], h[GRTX_MAX_BATCH];
    unsigned items[GRTX_MAX_BATCH], begins[GRTX_MAX_BATCH];
    uint64_t all = 0;
    for (int i = 0; i < n_cams; ++i) {
        if (!rgbT[i] || ((uintptr_t)rgbT[i] & 15))
            return grtx_fail(GRTX_ERR_INVALID_ARG, "every rgbT output must be non-NULL and 16-byte aligned");
        items[i] = 0;
        st = grtx_fill_camera(v[i].cam, items[i], &cams[i]);
        if (st) return st;
        all += items[i];
        if (all >= (1ull << 31)) return grtx_fail(GRTX_ERR_INVALID_ARG, "too many rays");
        v[i].sc = grtx_scene_ref(sc);
        v[i].out = (float4 *)rgbT[i];
        v[i].item_begin = 0;
        v[i].pad = 0;
    }
    // The queue hands out the smallest views first: a small view cannot fill the GPU alone and
    // often holds the longest rays (bounce rays), so queued last its warps would run on after
    // the large views finish; queued first they run beside them (identical outputs). The
    // table stays sorted by step_begin for the kernel's search.
    int order[GRTX_MAX_BATCH];
    for (int i = 0; i < n_cams; ++i) order[i] = i;
    std::stable_sort(order, order + n_cams, [&](int x, int y) { return items[x] < items[y]; });
    unsigned total = 0;
    for (int j = 0; j < n_cams; ++j) {
        h[j] = v[order[j]];
        h[j].step_begin = total;
        begins[j] = total;
        h[j].count = items[order[j]];
        total += items[order[j]];
    }
    int bps = 0;
    if (segments_occupancy_k(p->k, &bps) != GRTX_OK || bps <= 0) return grtx_fail(GRTX_ERR_CUDA, "occupancy query failed");
    int blocks = sm_count() * bps;
    int n_slots = blocks * 128;
    bool ckpt = a.traversal == GRTX_TRAVERSAL_CHECKPOINT;
    size_t C = ckpt ? a.ckpt_cap : 1, E = ckpt ? a.evict_cap : 1;
    uint2 *base = nullptr;
    cudaStream_t s = S(stream);
    st = ensure_workspace(sc, n_slots, 2 * C + E, s, &base);
    if (st) return st;
    a.ck0 = base;
    a.ck1 = base + (size_t)n_slots * C;
    a.ev = base + (size_t)n_slots * 2 * C;
    a.n_slots = n_slots;
    a.queue = sc->d_counter + 2;
    a.n_items = total;
    if (!set_list_offsets(a, 2 * C + E))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "checkpoint/eviction capacities too large for the resident ray slots");
    a.discard = lists_discardable(a);
    ServeSeg *d = nullptr;      // the records, then the begins array
    st = grtx_malloc_async((void **)&d, (sizeof(ServeSeg) + sizeof(unsigned)) * n_cams, s);
    if (st) return st;
    unsigned *d_begins = reinterpret_cast<unsigned *>(d + n_cams);
    GRTX_CUDA(cudaMemcpyAsync(d, h, sizeof(ServeSeg) * n_cams, cudaMemcpyHostToDevice, s));
    GRTX_CUDA(cudaMemcpyAsync(d_begins, begins, sizeof(unsigned) * n_cams, cudaMemcpyHostToDevice, s));
    GRTX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), s));
    int launched = segments_launch_k(p->k, a, d, d_begins, n_cams, blocks, s);
    cudaFreeAsync(d, s);
    if (launched != GRTX_OK) {
        cudaError_t e = cudaGetLastError();
        return grtx_cuda_fail(e == cudaSuccess ? cudaErrorLaunchFailure : e, "batched trace launch");
    }
    return GRTX_OK;
}

namespace {

int backward(grtx_scene *sc, const grtx_gaussians *g, const grtx_camera *cam, const grtx_params *p,
             const float *d_rgbT, const float *d_dL_drgbT, const grtx_saved *saved, const grtx_grads *grads,
             cudaStream_t s)
{
    TraceArgs a = {};
    int st = setup(sc, cam, p, a);
    if (st) return st;
    if (sc->form == GRTX_FORM_PROXY20) return grtx_fail(GRTX_ERR_INVALID_ARG, "backward needs a sphere or icosphere scene");
    if (!g || g->n != sc->n || g->sh_degree != sc->sh_degree)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "gaussians do not match the scene");
    if (sc->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "a parameter array is NULL");
    if (!d_rgbT || !d_dL_drgbT || !grads) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)d_rgbT & 15) || ((uintptr_t)d_dL_drgbT & 15))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "image buffers must be 16-byte aligned");
    // the backward replays k-buffer rounds; a single-round forward gives the same blend lists
    if (a.traversal == GRTX_TRAVERSAL_SINGLE) {
        a.traversal = GRTX_TRAVERSAL_RESTART;
        a.ckpt_cap = GRTX_DEFAULT_CKPT_CAPACITY;
    }
    a.fwd_rgbT = (const float4 *)d_rgbT;
    a.dL_drgbT = (const float4 *)d_dL_drgbT;
    a.means = g->means;
    a.log_scales = g->log_scales;
    a.quats = g->quats;
    a.logits = g->opacity_logits;
    a.g_means = grads->means;
    a.g_log_scales = grads->log_scales;
    a.g_quats = grads->quats;
    a.g_logits = grads->opacity_logits;
    a.g_sh = grads->sh;
    a.n_sh = sc->n_coef * 3;
    a.vec_sh = a.n_sh == 48 && ((uintptr_t)grads->sh & 15) == 0;
    if (saved) {
        if (!saved->leaves || !saved->n || saved->cap <= 0)
            return grtx_fail(GRTX_ERR_INVALID_ARG, "saved lists need leaves, n and a positive cap");
        if (sc->form != GRTX_FORM_SPHERE) return grtx_fail(GRTX_ERR_INVALID_ARG, "saved lists need the sphere form");
        a.save_leaves = saved->leaves;
        a.save_n = saved->n;
        a.save_cap = saved->cap;
    }
    // gradients of means, logits, log-scales and quaternions are staged per leaf (vector
    // atomics in the kernel), then added into the caller's arrays
    const bool staged = sc->n_valid > 0 && (grads->means || grads->log_scales || grads->quats || grads->opacity_logits);
    if (staged) {
        st = grtx_malloc_async((void **)&a.g_stage, (size_t)sc->n_valid * 48, s);
        if (st) return st;
        GRTX_CUDA(cudaMemsetAsync(a.g_stage, 0, (size_t)sc->n_valid * 48, s));
    }
    st = run(sc, a, p->k, false, PASS_BWD, sc->d_counter + 1, s);
    if (staged) {
        if (st == GRTX_OK)
            k_scatter_grads<<<grtx_div_up(sc->n_valid, 256), 256, 0, s>>>(a.g_stage, sc->gid, sc->n_valid, grads->means,
                                                                         grads->log_scales, grads->quats,
                                                                         grads->opacity_logits);
        cudaFreeAsync(a.g_stage, s);
        if (st == GRTX_OK) GRTX_CHECK_LAUNCH("gradient scatter");
    }
    return st;
}

}  // namespace

extern "C" GRTX_API int grtx_trace_backward(grtx_scene *sc, const grtx_gaussians *g, const grtx_camera *cam,
                                            const grtx_params *p, const float *d_rgbT, const float *d_dL_drgbT,
                                            const grtx_grads *grads, void *stream)
{
    return backward(sc, g, cam, p, d_rgbT, d_dL_drgbT, nullptr, grads, S(stream));
}

extern "C" GRTX_API int grtx_trace_backward_saved(grtx_scene *sc, const grtx_gaussians *g, const grtx_camera *cam,
                                                  const grtx_params *p, const float *d_rgbT,
                                                  const float *d_dL_drgbT, const grtx_saved *saved,
                                                  const grtx_grads *grads, void *stream)
{
    if (!saved) return grtx_fail(GRTX_ERR_INVALID_ARG, "saved is NULL");
    return backward(sc, g, cam, p, d_rgbT, d_dL_drgbT, saved, grads, S(stream));
}
