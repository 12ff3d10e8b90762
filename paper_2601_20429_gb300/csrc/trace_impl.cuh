// Trace kernels: one thread per ray, persistent warps pulling 8x4-pixel tiles from a queue.
// Per ray: rounds of {pre-fill the k-buffer from the eviction list; traverse from the root
// (first round / restart) or from the checkpointed nodes (later rounds); blend the k-buffer
// in depth order with early termination} (Sec. III-A; Sec. IV-B, Listing 1).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "grtx_internal.cuh"

// Scene arrays a trace reads (leaf order; see grtx_scene).
struct SceneRef {
    const float4 *nodes;
    const float4 *geom;
    const float4 *tris;
    const float *app;
    const uint32_t *gid;
    const float4 *tpl_nodes, *tpl_tris;   // icosphere forms: shared template BVH and triangles
    const float4 *raw;                    // [n_valid][3] raw parameters in leaf order (backward)
    const float4 *nodes4;                 // 4-wide nodes (8 float4 each), or NULL
    int app_stride, sh_degree, has_tree;
    uint32_t n_nodes, n_leaves, n_geom;   // internal nodes, leaf records, Gaussian records
    uint32_t n_nodes4;
};

// Leaf kinds of the trace kernels: one analytic unit sphere per Gaussian; one world-space
// proxy triangle per leaf (monolithic); one Gaussian instance whose leaf test traverses the
// shared icosphere template in unit-sphere space before the exact test.
// 3 and 4: sphere leaves under 4-wide nodes, with float or quantised child boxes
enum : int { FORM_SPHERE = 0, FORM_PROXY = 1, FORM_ICO = 2, FORM_SPHERE4 = 3, FORM_SPHERE4Q = 4 };

// A camera (rays generated in-kernel) or an explicit ray list.
struct CamRef {
    int cam_type, width, height, tiles_x;
    float3 pos, right, up, fwd;
    float tan_half, aspect, fish_f;
    float t_near, t_far;
    const float *ray_o, *ray_d, *ray_tn, *ray_tf;
};

struct TraceArgs {
    SceneRef sc;
    CamRef cam;
    unsigned n_items;            // queue items: 32 per warp tile (camera) or rays rounded up
    // parameters
    int traversal;               // GRTX_TRAVERSAL_*
    float T_min, alpha_max;
    float bg0, bg1, bg2;
    int ckpt_cap, evict_cap;
    int packet_stack;            // warp-stack entries a packet may use (1..kPacketStack)
    // per-slot workspace, interleaved [entry][slot]; the kernels address every list entry as
    // ck0[offset] with a 32-bit offset (ck1 = ck0 + ck1_off, ev = ck0 + ev_off; the host checks
    // that the whole workspace has fewer than 2^31 entries)
    uint2 *ck0, *ck1, *ev;
    uint32_t ck1_off, ev_off;
    int n_slots;
    int discard;                 // drop dead list lines from L2 after each tile (lists 256-byte aligned)
    unsigned *queue;
    // outputs
    float4 *rgbT;
    int32_t *n_blended;
    uint32_t *ids;
    int ids_cap;
    uint32_t *visits, *visits_n;   // visit log of sampled rays (see grtx_trace_outputs)
    int visits_cap, visits_stride, visits_rows;
    uint32_t *save_leaves;         // blend lists saved by a forward for its backward (grtx_saved)
    int32_t *save_n;
    int save_cap;
    grtx_stats *stats;
    // backward
    const float4 *fwd_rgbT, *dL_drgbT;
    const float *means, *log_scales, *quats, *logits;
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
    float4 *g_stage;             // [n_valid][3] per-leaf gradients of (mu, logit), log-scales, q
    int n_sh;
    int vec_sh;                  // gradients of SH (48 floats) may use float4 atomics
};

// One request of a serving step: its scene, camera, output, and which of its queue items
// this step covers (items [item_begin, item_begin + count) of the request map to step items
// [step_begin, step_begin + count)). Counts are multiples of 32. The kernel finds a tile's
// segment by a search over a separate array `begins` of the segments' step_begin values
// (ascending; entries past the last segment hold 0xffffffff, so that a launch's n_segs may be
// its table's capacity while the host appends segments).
// Records are 256-byte aligned so that a record the host appends while a launch runs shares
// no cache line with one the launch has already read.
struct __align__(256) ServeSeg {
    SceneRef sc;
    CamRef cam;
    float4 *out;
    unsigned item_begin, step_begin, count, pad;
};

// Controls of a serving launch (all NULL / 0 for a plain batched launch):
//   seg_done, seg_flag, seq: per-segment completion. The warp that finishes a segment's last
//     tile writes seq to seg_flag[segment] (pinned host memory mapped into the device).
//   avail: {items, closed}. The host appends segments while the launch runs: it writes their
//     records and begins entries, then raises the item count, and last, once it appends no
//     more, sets closed = 1. NULL: the launch's n_items is final. A warp claims its next tile
//     whether or not it is published yet and waits for it (sleeping between checks) until it
//     is published, the launch is closed, or linger_ns pass without any publication.
//   lost: [0] a count, then the first item of each tile a warp claimed and gave up on after
//     linger_ns; the host traces those again if it published them after all. lost_cap: the
//     launch's warps, since a warp stops after giving up.
//   exited: a count of warps that gave up, mirrored into exited_host (mapped host memory) so
//     that the host stops appending to a launch that has begun to wind down.
//   claimed_host: mapped host memory; every 16th claim, and every claim a warp has to wait
//     for, writes its end there, so that the host sees how much published work is left and
//     publishes more only when it runs low (the host chooses what runs next, instead of a long
//     queue fixing it).
static_assert(sizeof(ServeSeg) == 256, "a segment record fills one 256-byte slot");

struct ServeLive {
    unsigned *seg_done;
    unsigned *seg_flag;
    unsigned seq;
    const unsigned *avail;
    unsigned *lost;
    unsigned lost_cap;
    unsigned *exited;
    unsigned *exited_host;
    unsigned linger_ns;
    unsigned *claimed_host;
};

struct Counters {
    unsigned nodes, leaves, blended, rounds, ckpt, evictions, fallbacks, overflow;
    unsigned oob;      // fetch indices found outside their arrays (instrumented path only)
    uint32_t *vlog;    // the current ray's row of the visit log, or NULL (instrumented path only)
    unsigned vn, vcap;
};

// One node or leaf-record fetch of the current ray into its visit-log row (if it has one).
__device__ __forceinline__ void log_visit(Counters &c, uint32_t ref)
{
    if (c.vlog) {
        if (c.vn < c.vcap) c.vlog[c.vn] = ref;
        ++c.vn;
    }
}

// Self-check of the instrumented kernels (the ones that fill grtx_stats): before a node or
// leaf record is fetched its index is compared with the size of its array, and so is the
// Gaussian index a proxy triangle names. An index outside is counted (grtx_stats.bounds_errors)
// and not fetched; the traversal treats it as a miss. Every parity render runs these kernels,
// so every parity case is also a check that the traversal never leaves the scene's arrays.
__device__ __forceinline__ bool ref_ok(const SceneRef &sc, uint32_t ref, Counters &c, bool count = true)
{
    bool ok = (ref & GRTX_LEAF) ? (ref & ~GRTX_LEAF) < sc.n_leaves : ref < sc.n_nodes;
    if (!ok && count) ++c.oob;
    return ok;
}

__device__ __forceinline__ bool ref4_ok(const SceneRef &sc, uint32_t ref, Counters &c, bool count = true)
{
    bool ok = (ref & GRTX_LEAF) ? (ref & ~GRTX_LEAF) < sc.n_leaves : ref < sc.n_nodes4;
    if (!ok && count) ++c.oob;
    return ok;
}

__device__ __forceinline__ bool gauss_ok(const SceneRef &sc, uint32_t gi, Counters &c)
{
    if (gi < sc.n_geom) return true;
    ++c.oob;
    return false;
}

#define GRTX_INF __int_as_float(0x7f800000)

// Start / finish the visit log of one ray (valid: the lane holds a ray with output index pix).
__device__ __forceinline__ void visits_begin(const TraceArgs &a, Counters &c, bool valid, int64_t pix)
{
    c.vlog = nullptr;
    c.vn = 0;
    if (a.visits && valid && pix % a.visits_stride == 0 && pix / a.visits_stride < a.visits_rows) {
        c.vlog = a.visits + (size_t)(pix / a.visits_stride) * a.visits_cap;
        c.vcap = (unsigned)a.visits_cap;
    }
}
__device__ __forceinline__ void visits_end(const TraceArgs &a, Counters &c, int64_t pix)
{
    if (c.vlog) a.visits_n[pix / a.visits_stride] = c.vn;
    c.vlog = nullptr;
}

// ------------------------------------------------------------------------------------------
// Rays
// ------------------------------------------------------------------------------------------
// Queue items: a warp's 32 items are an 8x4 pixel tile (tiles_x > 0: cameras, and ray lists
// laid out as an image of at least four rows, so that a warp's rays are neighbours), or 32
// consecutive rays of a list (tiles_x = 0). Output index pix = y * width + x either way.
__device__ __forceinline__ unsigned item_of_pixel(const CamRef &a, int64_t p)
{
    if (!a.tiles_x) return (unsigned)p;
    int x = (int)(p % a.width), y = (int)(p / a.width);
    return (unsigned)(((y / 4) * a.tiles_x + (x / 8)) * 32 + (y % 4) * 8 + (x % 8));
}

__device__ __forceinline__ bool make_ray(const CamRef &a, unsigned item, int64_t &pix, float3 &o, float3 &d,
                                         float &tn, float &tf)
{
    int px = 0, py = 0;
    if (a.tiles_x) {
        unsigned tile = item >> 5, l = item & 31u;
        px = (int)(tile % (unsigned)a.tiles_x) * 8 + (int)(l & 7u);
        py = (int)(tile / (unsigned)a.tiles_x) * 4 + (int)(l >> 3);
        if (px >= a.width || py >= a.height) return false;
        pix = (int64_t)py * a.width + px;
    } else {
        if ((int64_t)item >= (int64_t)a.width * a.height) return false;
        pix = item;
    }
    if (a.cam_type == GRTX_CAMERA_RAYS) {
        o = make_float3(a.ray_o[3 * pix], a.ray_o[3 * pix + 1], a.ray_o[3 * pix + 2]);
        d = make_float3(a.ray_d[3 * pix], a.ray_d[3 * pix + 1], a.ray_d[3 * pix + 2]);
        tn = a.ray_tn ? a.ray_tn[pix] : a.t_near;
        tf = a.ray_tf ? a.ray_tf[pix] : a.t_far;
        return true;
    }
    float dx, dy, dz;
    if (a.cam_type == GRTX_CAMERA_PINHOLE) {
        float u = (2.0f * (px + 0.5f) / a.width - 1.0f) * a.tan_half * a.aspect;
        float v = (1.0f - 2.0f * (py + 0.5f) / a.height) * a.tan_half;
        dx = a.fwd.x + u * a.right.x + v * a.up.x;
        dy = a.fwd.y + u * a.right.y + v * a.up.y;
        dz = a.fwd.z + u * a.right.z + v * a.up.z;
    } else {
        float ex = px + 0.5f - 0.5f * a.width, ey = 0.5f * a.height - (py + 0.5f);
        float r = sqrtf(ex * ex + ey * ey);
        float th = r / a.fish_f;
        float cp = r > 0.f ? ex / r : 1.f, sp = r > 0.f ? ey / r : 0.f;
        float st, ct;
        sincosf(th, &st, &ct);
        dx = st * cp * a.right.x + st * sp * a.up.x + ct * a.fwd.x;
        dy = st * cp * a.right.y + st * sp * a.up.y + ct * a.fwd.y;
        dz = st * cp * a.right.z + st * sp * a.up.z + ct * a.fwd.z;
    }
    float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    o = a.pos;
    d = make_float3(dx * inv, dy * inv, dz * inv);
    tn = a.t_near;
    tf = a.t_far;
    return true;
}

__device__ __forceinline__ float safe_rcp(float x)
{
    return fabsf(x) > 1e-30f ? 1.0f / x : copysignf(1e30f, x);
}

// ------------------------------------------------------------------------------------------
// k-buffer (Sec. III-A): the k nearest keys (t, leaf index) found so far, ascending. It lives in
// shared memory as a structure of arrays over the block's 128 threads (entry j of thread x at
// [j * 128 + x], so a warp touching one entry hits 32 distinct banks), which keeps its 2k
// words out of the register file; t_max, the farthest kept depth once full, stays in a register.
// ------------------------------------------------------------------------------------------
constexpr int kBlock = 128;

template <int K>
struct KBuf {
    float *t;
    uint32_t *id;
    int n;
    float tmax;
    __device__ __forceinline__ void clear()
    {
        n = 0;
        tmax = GRTX_INF;
    }
    __device__ __forceinline__ float T(int j) const { return t[j * kBlock]; }
    __device__ __forceinline__ uint32_t I(int j) const { return id[j * kBlock]; }
    __device__ __forceinline__ bool contains(float ct, uint32_t ci) const
    {
        for (int j = 0; j < n; ++j)
            if (t[j * kBlock] == ct && id[j * kBlock] == ci) return true;
        return false;
    }
    // Insert (ct, ci) in key order. When the buffer was already full the larger of {new key,
    // farthest kept key} is rejected: it is returned in (ct, ci) and the result is true.
    __device__ __forceinline__ bool insert(float &ct, uint32_t &ci)
    {
        int pos;
        bool rejected = false;
        float nt = ct;
        uint32_t ni = ci;
        if (n == K) {
            float lt = t[(K - 1) * kBlock];
            uint32_t li = id[(K - 1) * kBlock];
            if (!(nt < lt || (nt == lt && ni < li))) return true;
            ct = lt;
            ci = li;
            rejected = true;
            pos = K - 1;
        } else {
            pos = n++;
        }
        while (pos > 0) {
            float pt = t[(pos - 1) * kBlock];
            uint32_t pi = id[(pos - 1) * kBlock];
            if (!(nt < pt || (nt == pt && ni < pi))) break;
            t[pos * kBlock] = pt;
            id[pos * kBlock] = pi;
            --pos;
        }
        t[pos * kBlock] = nt;
        id[pos * kBlock] = ni;
        if (n == K) tmax = t[(K - 1) * kBlock];
        return rejected;
    }
};

__device__ __forceinline__ bool key_after(float t, uint32_t i, float Lt, uint32_t Li)
{
    return t > Lt || (t == Lt && i > Li);
}

// Closest approach of the ray to the centre of a Gaussian in its unit-sphere space (Sec. IV-A):
// with the record rows (A_j | mu_j), o_l = A (o - mu), d_l = A d, t = -(o_l.d_l)/(d_l.d_l) and
// D2 = |o_l + t d_l|^2. t is the max-response depth of Sec. III-A Eq. t-max-resp, and D2 <= 1
// iff alpha >= alpha_min. Stage 1 runs for every leaf and only filters: in FP32 its absolute
// error in D2 grows like |o_l| (the ray origin measured in Gaussian widths), so the threshold
// is widened to 1 + 1e-5 + 4e-6 |o_l|, tested in squared form (no square root). Its t only
// seeds stage 2, whose Newton step lands on the minimiser from any nearby start, so the
// quotient is the fast approximate one.
__device__ __forceinline__ bool sphere_candidate(float4 r0, float4 r1, float4 r2, float3 o, float3 d, float &t)
{
    float vx = o.x - r0.w, vy = o.y - r1.w, vz = o.z - r2.w;
    float olx = fmaf(r0.x, vx, fmaf(r0.y, vy, r0.z * vz));
    float oly = fmaf(r1.x, vx, fmaf(r1.y, vy, r1.z * vz));
    float olz = fmaf(r2.x, vx, fmaf(r2.y, vy, r2.z * vz));
    float dlx = fmaf(r0.x, d.x, fmaf(r0.y, d.y, r0.z * d.z));
    float dly = fmaf(r1.x, d.x, fmaf(r1.y, d.y, r1.z * d.z));
    float dlz = fmaf(r2.x, d.x, fmaf(r2.y, d.y, r2.z * d.z));
    float aa = fmaf(dlx, dlx, fmaf(dly, dly, dlz * dlz));
    float bb = fmaf(olx, dlx, fmaf(oly, dly, olz * dlz));
    t = __fdividef(-bb, aa);
    float px = fmaf(t, dlx, olx), py = fmaf(t, dly, oly), pz = fmaf(t, dlz, olz);
    float D2 = fmaf(px, px, fmaf(py, py, pz * pz));
    float oo = fmaf(olx, olx, fmaf(oly, oly, olz * olz));
    float ex = D2 - (1.0f + 1e-5f);
    return ex <= 0.0f || ex * ex <= 1.6e-11f * oo;    // ex <= 4e-6 sqrt(oo)
}

// Error-free a + b = s + e (Knuth's two-sum).
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    float s = __fadd_rn(a, b);
    float bv = __fsub_rn(s, a);
    float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return s;
}

// Stage 2 for candidates: the world offset w = o + t d - mu is formed as an unevaluated sum of
// two floats (two-sum for o - mu, an FMA for the rounding error of t d), mapped to unit-sphere
// space, and t is moved to the exact minimiser along the line by one Newton step. D2 is then
// accurate to a few ulp of 1 whatever the distance from the ray origin. w receives the world
// offset of the closest point from the mean.
__device__ __forceinline__ void sphere_refine(float4 r0, float4 r1, float4 r2, float3 o, float3 d, float &t, float &D2,
                                              float w[3])
{
    const float oc[3] = {o.x, o.y, o.z}, dc[3] = {d.x, d.y, d.z}, mu[3] = {r0.w, r1.w, r2.w};
    float wh[3], wl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float vl, e1;
        float vh = two_sum(oc[c], -mu[c], vl);
        float ph = __fmul_rn(t, dc[c]);
        float pl = fmaf(t, dc[c], -ph);
        wh[c] = two_sum(vh, ph, e1);
        wl[c] = e1 + vl + pl;
    }
    const float4 R[3] = {r0, r1, r2};
    float p[3], dl[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float lo = fmaf(R[j].x, wl[0], fmaf(R[j].y, wl[1], R[j].z * wl[2]));
        p[j] = fmaf(R[j].x, wh[0], fmaf(R[j].y, wh[1], fmaf(R[j].z, wh[2], lo)));
        dl[j] = fmaf(R[j].x, d.x, fmaf(R[j].y, d.y, R[j].z * d.z));
    }
    // the step only corrects t, so the fast quotient's few-ulp relative error in it stays far
    // below one ulp of t
    float delta = __fdividef(fmaf(p[0], dl[0], fmaf(p[1], dl[1], p[2] * dl[2])),
                             fmaf(dl[0], dl[0], fmaf(dl[1], dl[1], dl[2] * dl[2])));
    t -= delta;
#pragma unroll
    for (int j = 0; j < 3; ++j) p[j] = fmaf(-delta, dl[j], p[j]);
    D2 = fmaf(p[0], p[0], fmaf(p[1], p[1], p[2] * p[2]));
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = fmaf(-delta, dc[c], wh[c] + wl[c]);
}

// Full test of one Gaussian record: returns true for a hit candidate and then (t, D2, w).
__device__ __forceinline__ bool sphere_test(const float4 *__restrict__ g, float3 o, float3 d, float &t, float &D2,
                                            float w[3])
{
    float4 r0 = __ldg(g), r1 = __ldg(g + 1), r2 = __ldg(g + 2);
    if (!sphere_candidate(r0, r1, r2, o, d, t)) return false;
    sphere_refine(r0, r1, r2, o, d, t, D2, w);
    return true;
}

// Real spherical harmonics up to degree 3 (no Condon-Shortley phase), index l*l + l + m,
// times the coefficients: c = max(0, sum_k Y_k(dir) f_k + 0.5); raw receives the sum + 0.5.
// The record holds the coefficients as (k, channel) pairs padded to a multiple of 4 floats
// and is read with float4 loads.
__device__ __forceinline__ void sh_color(const float *__restrict__ f, int deg, int stride, float3 n, float c[3],
                                         float raw[3], float Y[16])
{
    float x = n.x, y = n.y, z = n.z;
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = 0.f;
    Y[0] = 0.28209479177387814f;
    if (deg >= 1) {
        Y[1] = 0.4886025119029199f * y;
        Y[2] = 0.4886025119029199f * z;
        Y[3] = 0.4886025119029199f * x;
    }
    if (deg >= 2) {
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = 1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (3.f * z * z - 1.f);
        Y[7] = 1.0925484305920792f * x * z;
        Y[8] = 0.5462742152960396f * (x * x - y * y);
    }
    if (deg >= 3) {
        Y[9] = 0.5900435899266435f * y * (3.f * x * x - y * y);
        Y[10] = 2.890611442640554f * x * y * z;
        Y[11] = 0.4570457994644658f * y * (5.f * z * z - 1.f);
        Y[12] = 0.3731763325901154f * z * (5.f * z * z - 3.f);
        Y[13] = 0.4570457994644658f * x * (5.f * z * z - 1.f);
        Y[14] = 1.445305721320277f * z * (x * x - y * y);
        Y[15] = 0.5900435899266435f * x * (x * x - 3.f * y * y);
    }
    float acc[3] = {0.5f, 0.5f, 0.5f};
    const int n_vec = stride >> 2;
    const float4 *f4 = reinterpret_cast<const float4 *>(f);
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        if (j < n_vec) {
            float4 q = __ldg(f4 + j);
            const float qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = 4 * j + e;                // flat index = 3 k + channel
                if (i < 48) acc[i % 3] = fmaf(Y[i / 3], qq[e], acc[i % 3]);
            }
        }
    }
    raw[0] = acc[0]; raw[1] = acc[1]; raw[2] = acc[2];
    c[0] = fmaxf(acc[0], 0.f); c[1] = fmaxf(acc[1], 0.f); c[2] = fmaxf(acc[2], 0.f);
}

// Slab test of one child box against the ray over [tn, tf]: entry / exit distances, each
// plane distance as one FMA, l * inv - o * inv. Its rounding error is an ulp of the origin's
// plane distance, far inside the margin between a box's entry and the depth of any Gaussian hit
// in it, except for grazing hits at alpha_min; an axis-parallel ray (inv = 1e30) lying exactly
// in a face plane may lose that box, which it could only touch tangentially.
__device__ __forceinline__ void slab(float lx, float ly, float lz, float hx, float hy, float hz, float3 o, float3 inv,
                                     float tn, float tf, float &t0, float &t1)
{
    const float px = -o.x * inv.x, py = -o.y * inv.y, pz = -o.z * inv.z;
    float ax = fmaf(lx, inv.x, px), bx = fmaf(hx, inv.x, px);
    float ay = fmaf(ly, inv.y, py), by = fmaf(hy, inv.y, py);
    float az = fmaf(lz, inv.z, pz), bz = fmaf(hz, inv.z, pz);
    t0 = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), tn));
    t1 = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), tf));
}

// Ray / triangle (Moller-Trumbore) with a small barycentric tolerance so that shared edges
// of the proxy never leak; returns the hit distance or +inf.
__device__ __forceinline__ float tri_hit(float4 v0, float4 v1, float4 v2, float3 o, float3 d)
{
    float e1x = v1.x - v0.x, e1y = v1.y - v0.y, e1z = v1.z - v0.z;
    float e2x = v2.x - v0.x, e2y = v2.y - v0.y, e2z = v2.z - v0.z;
    float px = d.y * e2z - d.z * e2y, py = d.z * e2x - d.x * e2z, pz = d.x * e2y - d.y * e2x;
    float det = e1x * px + e1y * py + e1z * pz;
    if (fabsf(det) < 1e-30f) return GRTX_INF;
    float id = 1.0f / det;
    float sx = o.x - v0.x, sy = o.y - v0.y, sz = o.z - v0.z;
    float u = (sx * px + sy * py + sz * pz) * id;
    const float eps = 1e-5f;
    if (u < -eps || u > 1.f + eps) return GRTX_INF;
    float qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    float v = (d.x * qx + d.y * qy + d.z * qz) * id;
    if (v < -eps || u + v > 1.f + eps) return GRTX_INF;
    return (e2x * qx + e2y * qy + e2z * qz) * id;
}

// Leaf test of the instanced-icosphere forms (Sec. IV-A, second option): the ray in Gaussian
// gi's unit-sphere space (o_l = A (o - mu), d_l = A d, so t is the world t) traverses the
// shared template BVH; true at the first template triangle hit beyond t_near. The local ray
// is scaled by 1 / (1 + 1e-5 + 4e-6 |o_l|), which inflates the template against the FP32
// error of o_l without changing t, so that no exact hit is lost.
template <bool INSTR>
__device__ __forceinline__ bool template_touch(const SceneRef &sc, uint32_t gi, float3 o, float3 d, float tn,
                                               Counters &cnt)
{
    const float4 *g = sc.geom + 4 * (size_t)gi;
    float4 r0 = __ldg(g), r1 = __ldg(g + 1), r2 = __ldg(g + 2);
    float rx = o.x - r0.w, ry = o.y - r1.w, rz = o.z - r2.w;
    float3 ol = make_float3(r0.x * rx + r0.y * ry + r0.z * rz, r1.x * rx + r1.y * ry + r1.z * rz,
                            r2.x * rx + r2.y * ry + r2.z * rz);
    float sc_l = 1.0f / (1.0f + 1e-5f + 4e-6f * sqrtf(ol.x * ol.x + ol.y * ol.y + ol.z * ol.z));
    ol = make_float3(ol.x * sc_l, ol.y * sc_l, ol.z * sc_l);
    float3 dl = make_float3((r0.x * d.x + r0.y * d.y + r0.z * d.z) * sc_l, (r1.x * d.x + r1.y * d.y + r1.z * d.z) * sc_l,
                            (r2.x * d.x + r2.y * d.y + r2.z * d.z) * sc_l);
    float3 inv = make_float3(safe_rcp(dl.x), safe_rcp(dl.y), safe_rcp(dl.z));
    uint32_t stack[16];
    int sp = 0;
    uint32_t ref = 0u;
    for (;;) {
        if (ref & GRTX_LEAF) {
            if (INSTR) cnt.leaves++;
            const float4 *tr = sc.tpl_tris + 3 * (size_t)(ref & ~GRTX_LEAF);
            if (tri_hit(__ldg(tr), __ldg(tr + 1), __ldg(tr + 2), ol, dl) > tn) return true;
        } else {
            if (INSTR) cnt.nodes++;
            const float4 *nd = sc.tpl_nodes + 4 * (size_t)ref;
            float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            float e0, x0, e1, x1;
            slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ol, inv, tn, GRTX_INF, e0, x0);
            slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ol, inv, tn, GRTX_INF, e1, x1);
            bool h0 = e0 <= x0, h1 = e1 <= x1;
            uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
            if (h0 && h1) {
                bool near0 = e0 <= e1;
                ref = near0 ? c0 : c1;
                if (sp < 16) stack[sp++] = near0 ? c1 : c0;
                continue;
            }
            if (h0 || h1) {
                ref = h0 ? c0 : c1;
                continue;
            }
        }
        if (sp == 0) return false;
        ref = stack[--sp];
    }
}

// ------------------------------------------------------------------------------------------
// 4-wide nodes (FORM_SPHERE4; see grtx_params.bvh_width). A node holds its four children's
// boxes as per-axis rows; empty children have empty boxes (lo = +inf, hi = -inf) and ref
// GRTX_NONE. The rounds are those of the binary traversal: a child whose entry exceeds t_max
// is checkpointed, the others are visited, nearest first.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float pick4(const float v[4], int i)
{
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}
__device__ __forceinline__ uint32_t pick4(const uint32_t v[4], int i)
{
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}

// Float4 words of one 4-wide node: 8 with float child boxes, 4 with quantised ones.
template <bool Q>
__device__ __forceinline__ const float4 *node4(const SceneRef &sc, uint32_t ref)
{
    return sc.nodes4 + (Q ? 4 : 8) * (size_t)ref;
}

// Decoded quantised box coordinate: the node's corner plus q steps (one FMA, exactly as the
// build checked it). eb: the step's biased exponent.
__device__ __forceinline__ float dq(uint32_t q, uint32_t eb, float o)
{
    return fmaf(__uint2float_rn(q), __uint_as_float(eb << 23), o);
}

// Entry and exit of the ray in each child box of a 4-wide node (e > x: missed).
template <bool Q>
__device__ __forceinline__ void slab4(const float4 *__restrict__ nd, float3 o, float3 inv, float tn, float tf, float e[4],
                                      float x[4], uint32_t c[4])
{
    if (Q) {
        const float4 h = __ldg(nd);
        const uint4 qa = __ldg(reinterpret_cast<const uint4 *>(nd + 1));
        const uint4 qb = __ldg(reinterpret_cast<const uint4 *>(nd + 2));
        const uint4 qc = __ldg(reinterpret_cast<const uint4 *>(nd + 3));
        const uint32_t eb = __float_as_uint(h.w);
        const uint32_t ex = eb & 0xffu, ey = (eb >> 8) & 0xffu, ez = (eb >> 16) & 0xffu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int sh = 8 * j;
            slab(dq((qa.x >> sh) & 0xffu, ex, h.x), dq((qa.y >> sh) & 0xffu, ey, h.y), dq((qa.z >> sh) & 0xffu, ez, h.z),
                 dq((qa.w >> sh) & 0xffu, ex, h.x), dq((qb.x >> sh) & 0xffu, ey, h.y), dq((qb.y >> sh) & 0xffu, ez, h.z),
                 o, inv, tn, tf, e[j], x[j]);
        }
        c[0] = qb.z;
        c[1] = qb.w;
        c[2] = qc.x;
        c[3] = qc.y;
        return;
    }
    const float4 lx = __ldg(nd), ly = __ldg(nd + 1), lz = __ldg(nd + 2);
    const float4 hx = __ldg(nd + 3), hy = __ldg(nd + 4), hz = __ldg(nd + 5);
    const float4 rf = __ldg(nd + 6);
    slab(lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, o, inv, tn, tf, e[0], x[0]);
    slab(lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, o, inv, tn, tf, e[1], x[1]);
    slab(lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, o, inv, tn, tf, e[2], x[2]);
    slab(lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, o, inv, tn, tf, e[3], x[3]);
    c[0] = __float_as_uint(rf.x);
    c[1] = __float_as_uint(rf.y);
    c[2] = __float_as_uint(rf.z);
    c[3] = __float_as_uint(rf.w);
}

// Order (key, ord) pairs ascending by key: a 5-comparator network over 4 entries.
__device__ __forceinline__ void sort4(float k[4], int ord[4])
{
#define GRTX_CSWAP(i, j)                                                              \
    if (k[j] < k[i]) {                                                                \
        float tk = k[i]; k[i] = k[j]; k[j] = tk;                                      \
        int to = ord[i]; ord[i] = ord[j]; ord[j] = to;                                \
    }
    GRTX_CSWAP(0, 1) GRTX_CSWAP(2, 3) GRTX_CSWAP(0, 2) GRTX_CSWAP(1, 3) GRTX_CSWAP(1, 2)
#undef GRTX_CSWAP
}

// The sphere-leaf test of one leaf slot inside a round (shared by the 4-wide traversals):
// a hit with key in (L, t_max] enters the k-buffer; a hit the full buffer rejects goes to the
// eviction list when checkpointing. Returns false when the eviction list would overflow.
template <int K, bool INSTR>
__device__ __forceinline__ bool leaf4(const TraceArgs &a, const SceneRef &sc, uint32_t ref, float3 o, float3 d, float tn,
                                      float tf, float Lt, uint32_t Li, bool ckpt, uint32_t ev, int &n_ev, KBuf<K> &kb,
                                      float &tmax, Counters &cnt)
{
    const uint32_t gi = ref & ~GRTX_LEAF;
    if (INSTR) {
        cnt.leaves++;
        log_visit(cnt, ref);
    }
    float t, D2, w[3];
    if (sphere_test(sc.geom + 4 * (size_t)gi, o, d, t, D2, w) && D2 <= 1.0f && t > tn && t <= tf &&
        key_after(t, gi, Lt, Li)) {
        float ct = t;
        uint32_t ci = gi;
        if (kb.insert(ct, ci) && ckpt) {
            if (n_ev >= a.evict_cap) return false;
            a.ck0[ev + (uint32_t)n_ev * (uint32_t)a.n_slots] = make_uint2(__float_as_uint(ct), ci);
            ++n_ev;
            if (INSTR) cnt.evictions++;
        }
        tmax = kb.tmax;
    }
    return true;
}

// Entry distance of the ray into child `slot` of 4-wide node `parent`.
template <bool Q>
__device__ __forceinline__ float child_entry4(const SceneRef &sc, uint32_t parent, uint32_t slot, float3 o, float3 inv,
                                              float tn, float tf)
{
    float te, x;
    if (Q) {
        const float4 *nd = node4<true>(sc, parent);
        const float4 h = __ldg(nd);
        const uint4 qa = __ldg(reinterpret_cast<const uint4 *>(nd + 1));
        const uint4 qb = __ldg(reinterpret_cast<const uint4 *>(nd + 2));
        const uint32_t eb = __float_as_uint(h.w), sh = 8 * slot;
        const uint32_t ex = eb & 0xffu, ey = (eb >> 8) & 0xffu, ez = (eb >> 16) & 0xffu;
        slab(dq((qa.x >> sh) & 0xffu, ex, h.x), dq((qa.y >> sh) & 0xffu, ey, h.y), dq((qa.z >> sh) & 0xffu, ez, h.z),
             dq((qa.w >> sh) & 0xffu, ex, h.x), dq((qb.x >> sh) & 0xffu, ey, h.y), dq((qb.y >> sh) & 0xffu, ez, h.z), o,
             inv, tn, tf, te, x);
    } else {
        const float *pn = reinterpret_cast<const float *>(node4<false>(sc, parent));
        slab(__ldg(pn + slot), __ldg(pn + 4 + slot), __ldg(pn + 8 + slot), __ldg(pn + 12 + slot), __ldg(pn + 16 + slot),
             __ldg(pn + 20 + slot), o, inv, tn, tf, te, x);
    }
    return te;
}

// One round of one ray over 4-wide nodes (the per-ray rounds; see trace_round).
template <int K, bool INSTR, bool Q>
__device__ __forceinline__ bool trace_round4(const TraceArgs &a, const SceneRef &sc, float3 o, float3 d, float3 inv,
                                             float tn, float tf, float Lt, uint32_t Li, bool ckpt, bool from_root,
                                             uint32_t src, int n_src, uint32_t dst, int &n_dst, uint32_t ev,
                                             int &n_ev, KBuf<K> &kb, Counters &cnt)
{
    const uint32_t S = (uint32_t)a.n_slots;
    uint2 *__restrict__ const L = a.ck0;
    uint32_t stack[GRTX_STACK4];               // node refs; a popped entry is visited (see trace_round)
    int sp = 0, si = 0;
    float tmax = kb.tmax;
    uint32_t ref;
    float te;
    n_dst = 0;
    if (from_root) {
        n_src = 0;
        ref = 0u;
        te = tn;
    } else {
        if (n_src == 0) return true;
        uint2 v = L[src];
        ref = v.x;
        te = __uint_as_float(v.y);
        si = 1;
    }
    for (;;) {
        if (te > tmax) {
            if (ckpt) {
                if (n_dst >= a.ckpt_cap) return false;
                L[dst + (uint32_t)n_dst * S] = make_uint2(ref, __float_as_uint(te));
                ++n_dst;
                if (INSTR) cnt.ckpt++;
            }
        } else if (INSTR && !ref4_ok(sc, ref, cnt)) {
        } else if (ref & GRTX_LEAF) {
            if (!leaf4<K, INSTR>(a, sc, ref, o, d, tn, tf, Lt, Li, ckpt, ev, n_ev, kb, tmax, cnt)) return false;
        } else {
            if (INSTR) {
                cnt.nodes++;
                log_visit(cnt, ref);
            }
            float e[4], x[4];
            uint32_t c[4];
            slab4<Q>(node4<Q>(sc, ref), o, inv, tn, tf, e, x, c);
            int ord[4] = {0, 1, 2, 3};
            int nh = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool h = e[j] <= x[j] && !(x[j] < Lt) && c[j] != GRTX_NONE;
                nh += h;
                if (!h) e[j] = GRTX_INF;           // misses sort last
            }
            if (nh > 0) {
                sort4(e, ord);
#pragma unroll
                for (int j = 3; j >= 1; --j) {    // farthest first onto the stack, so the nearest pops first
                    if (j < nh) {
                        const uint32_t cj = pick4(c, ord[j]);
                        if (e[j] > tmax) {
                            if (ckpt) {
                                if (n_dst >= a.ckpt_cap) return false;
                                L[dst + (uint32_t)n_dst * S] = make_uint2(cj, __float_as_uint(e[j]));
                                ++n_dst;
                                if (INSTR) cnt.ckpt++;
                            }
                        } else if (sp < GRTX_STACK4) {
                            stack[sp++] = cj;
                        } else if (INSTR) {
                            cnt.overflow++;
                        }
                    }
                }
                ref = pick4(c, ord[0]);
                te = e[0];
                continue;
            }
        }
        if (sp > 0) {
            ref = stack[--sp];
            te = -GRTX_INF;
        } else if (si < n_src) {
            uint2 v = L[src + (uint32_t)si * S];
            ++si;
            ref = v.x;
            te = __uint_as_float(v.y);
        } else {
            break;
        }
    }
    return true;
}

// A round of a warp's rays from the root as one packet over 4-wide nodes (see packet_round).
// At a node every lane tests the four children; the warp continues into the child its lowest
// active lane enters first and keeps the others, with the lanes that want them, on the warp's
// stack (entries: child, parent << 2 | child slot, lane mask); a popped child's entry
// distance is recomputed per lane from its box in the parent.
template <int K, bool INSTR, bool Q>
__device__ __forceinline__ bool packet_round4(const TraceArgs &a, const SceneRef &sc, bool valid, uint4 *pst, float3 o,
                                              float3 d, float3 inv, float tn, float tf, float Lt, uint32_t Li,
                                              bool ckpt, uint32_t dst, int &n_dst, uint32_t ev, int &n_ev, KBuf<K> &kb,
                                              Counters &cnt, bool &lane_ok)
{
    const unsigned full = 0xffffffffu;
    const uint32_t S = (uint32_t)a.n_slots;
    uint2 *__restrict__ const L = a.ck0;
    const int lane = threadIdx.x & 31;
    float tmax = kb.tmax;
    n_dst = 0;
    n_ev = 0;
    lane_ok = true;
    if (!sc.has_tree) return true;
    int sp = 0;
    uint32_t ref = 0u, parent = GRTX_NONE, slot = 0u;
    unsigned m = __ballot_sync(full, valid);
    float te = tn;
    bool have_te = true;
    for (;;) {
        const bool in = (m >> lane) & 1u;
        if (!have_te && in) te = child_entry4<Q>(sc, parent, slot, o, inv, tn, tf);   // a popped child
        const bool go = in && lane_ok && !(te > tmax);
        if (in && lane_ok && te > tmax && ckpt) {
            if (n_dst >= a.ckpt_cap) {
                lane_ok = false;
            } else {
                L[dst + (uint32_t)n_dst * S] = make_uint2(ref, __float_as_uint(te));
                ++n_dst;
                if (INSTR) cnt.ckpt++;
            }
        }
        m = __ballot_sync(full, go);
        bool pop = true;
        if (m && (!INSTR || ref4_ok(sc, ref, cnt, go))) {   // ref is the warp's: all lanes agree
            if (ref & GRTX_LEAF) {
                if (go && !leaf4<K, INSTR>(a, sc, ref, o, d, tn, tf, Lt, Li, ckpt, ev, n_ev, kb, tmax, cnt))
                    lane_ok = false;
            } else {
                float e[4], x[4];
                uint32_t c[4];
                slab4<Q>(node4<Q>(sc, ref), o, inv, tn, tf, e, x, c);
                bool h[4];
                unsigned mh[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    h[j] = go && e[j] <= x[j] && !(x[j] < Lt) && c[j] != GRTX_NONE;
                    mh[j] = __ballot_sync(full, h[j]);
                }
                if (INSTR && go) {
                    cnt.nodes++;
                    log_visit(cnt, ref);
                }
                // order the wanted children by the lowest active lane's entry distances (children
                // it misses after those it enters, in child order; children nobody wants last)
                const int leader = __ffs(m) - 1;
                float k2[4];
                int rk[4], ord[4] = {0, 1, 2, 3};
                int nc = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float kl = __shfl_sync(full, h[j] ? e[j] : GRTX_INF, leader);
                    rk[j] = mh[j] == 0u ? 2 : (kl < GRTX_INF ? 0 : 1);
                    k2[j] = kl;
                    nc += mh[j] != 0u;
                }
                if (nc > 0) {
#define GRTX_CSWAP4(i, j)                                                                                 \
    if (rk[j] < rk[i] || (rk[j] == rk[i] && rk[i] == 0 && k2[j] < k2[i])) {                            \
        int tr = rk[i]; rk[i] = rk[j]; rk[j] = tr;                                                        \
        float tk = k2[i]; k2[i] = k2[j]; k2[j] = tk;                                                      \
        int to = ord[i]; ord[i] = ord[j]; ord[j] = to;                                                    \
    }
                    GRTX_CSWAP4(0, 1) GRTX_CSWAP4(2, 3) GRTX_CSWAP4(0, 2) GRTX_CSWAP4(1, 3) GRTX_CSWAP4(1, 2)
#undef GRTX_CSWAP4
                    if (sp + nc - 1 > a.packet_stack) {       // too deep for the warp's stack
                        lane_ok = false;
                        return false;
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int j = 3; j >= 1; --j) {        // farthest first
                            if (j < nc) {
                                const int oj = ord[j];
                                pst[sp + (nc - 1 - j)] = make_uint4(pick4(c, oj), (ref << 2) | (uint32_t)oj,
                                                                    oj == 0 ? mh[0] : (oj == 1 ? mh[1] : (oj == 2 ? mh[2] : mh[3])), 0u);
                            }
                        }
                    }
                    sp += nc - 1;
                    __syncwarp(full);
                    const int f = ord[0];
                    parent = ref;
                    slot = (uint32_t)f;
                    m = f == 0 ? mh[0] : (f == 1 ? mh[1] : (f == 2 ? mh[2] : mh[3]));
                    te = pick4(e, f);
                    ref = pick4(c, f);
                    have_te = true;
                    pop = false;
                }
            }
        }
        if (pop) {
            if (sp == 0) break;
            --sp;
            const uint4 v = pst[sp];
            ref = v.x;
            parent = v.y >> 2;
            slot = v.y & 3u;
            m = v.z;
            have_te = false;
        }
    }
    return true;
}

// ------------------------------------------------------------------------------------------
// One traversal round over keys in (L, t_max] (Sec. III-A). With ckpt, it starts from the
// checkpoint source list (or the root in the first round), writes nodes failing the t_max
// test to the destination list and rejected hits to the eviction list (Sec. IV-B);
// otherwise it starts at the root and culls. Returns false when a capacity is exceeded.
// ------------------------------------------------------------------------------------------
template <int K, int FORM, bool INSTR>
__device__ __forceinline__ bool trace_round(const TraceArgs &a, const SceneRef &sc, float3 o, float3 d, float3 inv,
                                            float inv_len, float tn, float tf,
                                            float Lt, uint32_t Li, bool ckpt, bool from_root,
                                            uint32_t src, int n_src, uint32_t dst, int &n_dst, uint32_t ev,
                                            int &n_ev, KBuf<K> &kb, Counters &cnt)
{
    if constexpr (FORM == FORM_SPHERE4 || FORM == FORM_SPHERE4Q)
        return trace_round4<K, INSTR, FORM == FORM_SPHERE4Q>(a, sc, o, d, inv, tn, tf, Lt, Li, ckpt, from_root, src,
                                                             n_src, dst, n_dst, ev, n_ev, kb, cnt);
    const uint32_t S = (uint32_t)a.n_slots;
    uint2 *__restrict__ const L = a.ck0;      // lists: src, dst and ev are entry offsets into L
    // far children deferred within this round: node refs only (4 bytes each); a popped entry
    // is visited without re-testing its entry depth, since its children meet the t_max test
    uint32_t stack[GRTX_STACK];
    int sp = 0, si = 0;
    float tmax = kb.tmax;
    uint32_t ref;
    float te;
    n_dst = 0;
    if (from_root) {
        n_src = 0;                    // a restart never resumes checkpointed subtrees
        ref = 0u;
        te = tn;
    } else {
        if (n_src == 0) return true;
        uint2 v = L[src];
        ref = v.x;
        te = __uint_as_float(v.y);
        si = 1;
    }
    for (;;) {
        if (te > tmax) {                              // fails the t_max test
            if (ckpt) {
                if (n_dst >= a.ckpt_cap) return false;
                L[dst + (uint32_t)n_dst * S] = make_uint2(ref, __float_as_uint(te));
                ++n_dst;
                if (INSTR) cnt.ckpt++;
            }
        } else if (INSTR && !ref_ok(sc, ref, cnt)) {  // not fetched (self-check)
        } else if (ref & GRTX_LEAF) {
            uint32_t idx = ref & ~GRTX_LEAF;
            if (INSTR) {
                cnt.leaves++;
                log_visit(cnt, ref);
            }
            uint32_t gi;
            bool touch = true;
            if (FORM == FORM_PROXY) {
                const float4 *tr = sc.tris + 3 * (size_t)idx;
                float4 v0 = __ldg(tr), v1 = __ldg(tr + 1), v2 = __ldg(tr + 2);
                gi = __float_as_uint(v0.w);
                touch = (!INSTR || gauss_ok(sc, gi, cnt)) && tri_hit(v0, v1, v2, o, d) > tn;
            } else {
                gi = idx;
                if (FORM == FORM_ICO) touch = template_touch<INSTR>(sc, gi, o, d, tn, cnt);
            }
            float t, D2, w[3];
            if (touch && sphere_test(sc.geom + 4 * (size_t)gi, o, d, t, D2, w)) {
                if (D2 <= 1.0f && t > tn && t <= tf && key_after(t, gi, Lt, Li)) {
                    if (FORM != FORM_PROXY || !kb.contains(t, gi)) {
                        float ct = t;
                        uint32_t ci = gi;
                        if (kb.insert(ct, ci) && ckpt) {       // any-hit: rejected -> eviction list
                            if (n_ev >= a.evict_cap) return false;
                            L[ev + (uint32_t)n_ev * S] = make_uint2(__float_as_uint(ct), ci);
                            ++n_ev;
                            if (INSTR) cnt.evictions++;
                        }
                        tmax = kb.tmax;                        // farthest kept key
                    }
                }
            }
        } else {
            if (INSTR) {
                cnt.nodes++;
                log_visit(cnt, ref);
            }
            const float4 *nd = sc.nodes + 4 * (size_t)ref;
            float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
            float e0, x0, e1, x1;
            slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, o, inv, tn, tf, e0, x0);
            slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, o, inv, tn, tf, e1, x1);
            bool h0 = e0 <= x0 && !(x0 < Lt);
            bool h1 = e1 <= x1 && !(x1 < Lt) && c1 != GRTX_NONE;
            bool near0 = e0 <= e1;
            if (FORM == FORM_PROXY) {
                // a proxy face can lie up to one proxy diameter beyond the Gaussian's key, so
                // the t_max test of a proxy subtree is taken at entry - (its largest diameter)
                e0 = fmaf(-n3.z, inv_len, e0);
                e1 = fmaf(-n3.w, inv_len, e1);
            }
            if (h0 && h1) {
                uint32_t far_ref = near0 ? c1 : c0;
                float far_t = near0 ? e1 : e0;
                ref = near0 ? c0 : c1;
                te = near0 ? e0 : e1;
                if (far_t > tmax) {
                    if (ckpt) {
                        if (n_dst >= a.ckpt_cap) return false;
                        L[dst + (uint32_t)n_dst * S] = make_uint2(far_ref, __float_as_uint(far_t));
                        ++n_dst;
                        if (INSTR) cnt.ckpt++;
                    }
                } else if (sp < GRTX_STACK) {
                    stack[sp++] = far_ref;
                } else if (INSTR) {
                    cnt.overflow++;
                }
                continue;
            }
            if (h0 || h1) {
                ref = h0 ? c0 : c1;
                te = h0 ? e0 : e1;
                continue;
            }
        }
        if (sp > 0) {
            ref = stack[--sp];
            te = -GRTX_INF;
        } else if (si < n_src) {
            uint2 v = L[src + (uint32_t)si * S];
            ++si;
            ref = v.x;
            te = __uint_as_float(v.y);
        } else {
            break;
        }
    }
    return true;
}

// ------------------------------------------------------------------------------------------
// A round of a warp's rays from the root as one packet (round 1, and every round when
// restarting). Every ray of a warp starts its first round at the root (Sec. III-A), and the
// rays of an 8x4 pixel tile need nearly the same nodes, so the warp
// walks one node sequence -- the union of what its rays need -- loading each node once for all
// lanes instead of once per lane, with no divergence between node and leaf steps. Each lane
// keeps its own entry test against its t_max, its k-buffer, checkpoint and eviction lists,
// exactly as in trace_round, so every ray's round ends with the same k-buffer (the traversal
// order, hence the checkpoint lists, may differ). The warp's stack (kPacketStack entries of
// (node, parent << 1 | child slot, lane mask), in shared memory) holds far children with the
// lanes that want them; a popped node's entry distance is recomputed per lane from its box in
// the parent. Every lane of the warp must call this together (full-mask ballots); lanes
// without a ray pass valid = false. lane_ok is false for a lane whose lists overflowed, and for
// every lane if the warp's stack would overflow (returns false then): such a lane redoes the
// round from the root on its own, as after any capacity overflow in trace_ray.
// ------------------------------------------------------------------------------------------
constexpr int kPacketStack = GRTX_PACKET_STACK;

template <int K, int FORM, bool INSTR>
__device__ __forceinline__ bool packet_round(const TraceArgs &a, const SceneRef &sc, bool valid, uint4 *pst, float3 o,
                                             float3 d, float3 inv, float inv_len, float tn, float tf, float Lt,
                                             uint32_t Li, bool ckpt, uint32_t dst, int &n_dst,
                                             uint32_t ev, int &n_ev, KBuf<K> &kb, Counters &cnt,
                                             bool &lane_ok)
{
    if constexpr (FORM == FORM_SPHERE4 || FORM == FORM_SPHERE4Q)
        return packet_round4<K, INSTR, FORM == FORM_SPHERE4Q>(a, sc, valid, pst, o, d, inv, tn, tf, Lt, Li, ckpt, dst,
                                                              n_dst, ev, n_ev, kb, cnt, lane_ok);
    const unsigned full = 0xffffffffu;
    const uint32_t S = (uint32_t)a.n_slots;
    uint2 *__restrict__ const L = a.ck0;      // lists: dst and ev are entry offsets into L
    const int lane = threadIdx.x & 31;
    float tmax = kb.tmax;
    n_dst = 0;
    n_ev = 0;
    lane_ok = true;
    if (!sc.has_tree) return true;                      // nothing to traverse (uniform)
    int sp = 0;
    uint32_t ref = 0u, parent = GRTX_NONE, slot = 0u;
    unsigned m = __ballot_sync(full, valid);
    float te = tn;
    bool have_te = true;
    for (;;) {
        bool in = (m >> lane) & 1u;
        if (!have_te && in) {                           // a popped node: entry from the parent's box
            const float4 *pn = sc.nodes + 4 * (size_t)parent;
            float x;
            if (slot == 0u) {
                float4 n0 = __ldg(pn), n1 = __ldg(pn + 1);
                slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, o, inv, tn, tf, te, x);
            } else {
                float4 n1 = __ldg(pn + 1), n2 = __ldg(pn + 2);
                slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, o, inv, tn, tf, te, x);
            }
            if (FORM == FORM_PROXY) te = fmaf(-(slot == 0u ? __ldg(pn + 3).z : __ldg(pn + 3).w), inv_len, te);
        }
        bool go = in && lane_ok && !(te > tmax);
        if (in && lane_ok && te > tmax && ckpt) {       // fails the t_max test: checkpoint it
            if (n_dst >= a.ckpt_cap) {
                lane_ok = false;
            } else {
                L[dst + (uint32_t)n_dst * S] = make_uint2(ref, __float_as_uint(te));
                ++n_dst;
                if (INSTR) cnt.ckpt++;
            }
        }
        m = __ballot_sync(full, go);
        bool pop = true;
        if (m && (!INSTR || ref_ok(sc, ref, cnt, go))) {   // ref is the warp's: all lanes agree
            if (ref & GRTX_LEAF) {
                if (go) {
                    uint32_t idx = ref & ~GRTX_LEAF;
                    if (INSTR) {
                        cnt.leaves++;
                        log_visit(cnt, ref);
                    }
                    uint32_t gi;
                    bool touch = true;
                    if (FORM == FORM_PROXY) {
                        const float4 *tr = sc.tris + 3 * (size_t)idx;
                        float4 v0 = __ldg(tr), v1 = __ldg(tr + 1), v2 = __ldg(tr + 2);
                        gi = __float_as_uint(v0.w);
                        touch = (!INSTR || gauss_ok(sc, gi, cnt)) && tri_hit(v0, v1, v2, o, d) > tn;
                    } else {
                        gi = idx;
                        if (FORM == FORM_ICO) touch = template_touch<INSTR>(sc, gi, o, d, tn, cnt);
                    }
                    float t, D2, w[3];
                    if (touch && sphere_test(sc.geom + 4 * (size_t)gi, o, d, t, D2, w) && D2 <= 1.0f && t > tn &&
                        t <= tf && key_after(t, gi, Lt, Li) && (FORM != FORM_PROXY || !kb.contains(t, gi))) {
                        float ct = t;
                        uint32_t ci = gi;
                        if (kb.insert(ct, ci) && ckpt) {
                            if (n_ev >= a.evict_cap) {
                                lane_ok = false;
                            } else {
                                L[ev + (uint32_t)n_ev * S] = make_uint2(__float_as_uint(ct), ci);
                                ++n_ev;
                                if (INSTR) cnt.evictions++;
                            }
                        }
                        tmax = kb.tmax;
                    }
                }
            } else {
                const float4 *nd = sc.nodes + 4 * (size_t)ref;
                float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
                uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
                bool h0 = false, h1 = false, near0 = true;
                float e0 = 0.f, e1 = 0.f;
                if (go) {
                    if (INSTR) {
                        cnt.nodes++;
                        log_visit(cnt, ref);
                    }
                    float x0, x1;
                    slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, o, inv, tn, tf, e0, x0);
                    slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, o, inv, tn, tf, e1, x1);
                    h0 = e0 <= x0 && !(x0 < Lt);
                    h1 = e1 <= x1 && !(x1 < Lt) && c1 != GRTX_NONE;
                    near0 = e0 <= e1;
                    if (FORM == FORM_PROXY) {             // t_max tests at entry - slack (see trace_round)
                        e0 = fmaf(-n3.z, inv_len, e0);
                        e1 = fmaf(-n3.w, inv_len, e1);
                    }
                }
                unsigned m0 = __ballot_sync(full, h0), m1 = __ballot_sync(full, h1);
                if (m0 && m1) {
                    unsigned both = m0 & m1, vote = __ballot_sync(full, h0 && h1 && near0);
                    bool n0first = both ? (2 * __popc(vote) >= __popc(both)) : (__popc(m0) >= __popc(m1));
                    if (sp >= a.packet_stack) {               // too deep for the warp's stack
                        lane_ok = false;
                        return false;
                    }
                    if (lane == 0)
                        pst[sp] = make_uint4(n0first ? c1 : c0, (ref << 1) | (n0first ? 1u : 0u), n0first ? m1 : m0, 0u);
                    ++sp;
                    __syncwarp(full);
                    parent = ref;
                    slot = n0first ? 0u : 1u;
                    m = n0first ? m0 : m1;
                    te = n0first ? e0 : e1;
                    ref = n0first ? c0 : c1;
                    have_te = true;
                    pop = false;
                } else if (m0 || m1) {
                    parent = ref;
                    slot = m0 ? 0u : 1u;
                    m = m0 ? m0 : m1;
                    te = m0 ? e0 : e1;
                    ref = m0 ? c0 : c1;
                    have_te = true;
                    pop = false;
                }
            }
        }
        if (pop) {
            if (sp == 0) break;
            --sp;
            uint4 v = pst[sp];
            ref = v.x;
            parent = v.y >> 1;
            slot = v.y & 1u;
            m = v.z;
            have_te = false;
        }
    }
    return true;
}

// ------------------------------------------------------------------------------------------
// Blending (Sec. II-B Eq. volume-render) and its derivative.
// ------------------------------------------------------------------------------------------
struct BlendState {
    float C[3];
    float T;
    // backward
    float G[4];        // dL/d(r, g, b, T_out)
    float Cf[3];       // forward colour without background
    float Tf;          // forward transmittance at termination
    float dLdT;        // dL/dT_out + bg . dL/dC
};

__device__ __forceinline__ float atomic_add_f(float *p, float v)
{
    return atomicAdd(p, v);
}

template <bool BWD>
__device__ __forceinline__ void blend_one(const TraceArgs &a, const SceneRef &sc, BlendState &st, uint32_t idx,
                                          float3 o, float3 d)
{
    const float nrm = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);     // colour along the unit direction
    const float3 dn = make_float3(d.x * nrm, d.y * nrm, d.z * nrm);
    const float4 *g = sc.geom + 4 * (size_t)idx;
    float t, D2, e[3];
    {
        float4 r0 = __ldg(g), r1 = __ldg(g + 1), r2 = __ldg(g + 2);
        sphere_candidate(r0, r1, r2, o, d, t);
        sphere_refine(r0, r1, r2, o, d, t, D2, e);
    }
    float4 r3 = __ldg(g + 3);
    float al_raw = r3.x * exp2f(r3.y * D2);
    bool clamped = !(al_raw < a.alpha_max);
    float al = clamped ? a.alpha_max : al_raw;
    float c[3], raw[3], Y[16];
    sh_color(sc.app + (size_t)idx * sc.app_stride, sc.sh_degree, sc.app_stride, dn, c, raw, Y);
    float w = st.T * al;
    if (!BWD) {
        st.C[0] = fmaf(w, c[0], st.C[0]);
        st.C[1] = fmaf(w, c[1], st.C[1]);
        st.C[2] = fmaf(w, c[2], st.C[2]);
        st.T *= (1.0f - al);
        return;
    }
    uint32_t gi = sc.gid[idx];
    // colour: dC/dc = T alpha; c = max(0, raw)
    if (a.g_sh) {
        const float dc[3] = {raw[0] > 0.f ? st.G[0] * w : 0.f, raw[1] > 0.f ? st.G[1] * w : 0.f,
                             raw[2] > 0.f ? st.G[2] * w : 0.f};
        float *gs = a.g_sh + (size_t)gi * a.n_sh;
        if (a.vec_sh) {
            // degree 3: the 48 coefficient gradients as 12 vector atomics (sm_90+ float4 add)
            if (dc[0] != 0.f || dc[1] != 0.f || dc[2] != 0.f) {
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    float v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) v[e] = Y[(4 * j + e) / 3] * dc[(4 * j + e) % 3];
                    atomicAdd(reinterpret_cast<float4 *>(gs) + j, make_float4(v[0], v[1], v[2], v[3]));
                }
            }
        } else {
            int nk = (sc.sh_degree + 1) * (sc.sh_degree + 1);
            for (int ch = 0; ch < 3; ++ch) {
                if (dc[ch] == 0.f) continue;
                for (int k = 0; k < nk; ++k) atomic_add_f(gs + 3 * k + ch, dc[ch] * Y[k]);
            }
        }
    }
    st.C[0] = fmaf(w, c[0], st.C[0]);
    st.C[1] = fmaf(w, c[1], st.C[1]);
    st.C[2] = fmaf(w, c[2], st.C[2]);
    float inv1m = __fdividef(1.0f, 1.0f - al);           // 1 - al >= 1 - alpha_max > 0
    float dLda = -st.dLdT * st.Tf * inv1m;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dLda += st.G[ch] * (st.T * c[ch] - (st.Cf[ch] - st.C[ch]) * inv1m);
    st.T *= (1.0f - al);
    if (clamped || dLda == 0.f) return;
    if (!a.g_stage) return;
    // alpha = o exp(-d2/2), d2 = |S^-1 R^T (x* - mu)|^2 at x* = o + t d (t fixed: envelope).
    // The raw parameters come packed in leaf order, (mu, logit), (log-scales, 0), q.
    const float4 *rw = sc.raw + 3 * (size_t)idx;
    const float4 r_ml = __ldg(rw), r_ls = __ldg(rw + 1), r_q = __ldg(rw + 2);
    float op = __fdividef(1.0f, 1.0f + expf(-r_ml.w));
    const float g_logit = dLda * al_raw * (1.0f - op);
    float dLdd2 = -0.5f * dLda * al_raw;
    // inverse scales 1/s_j = exp(-log s_j)
    float is[3] = {expf(-r_ls.x), expf(-r_ls.y), expf(-r_ls.z)};
    float qw = r_q.x, qx = r_q.y, qy = r_q.z, qz = r_q.w;
    float iq = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    float w_ = qw * iq, x = qx * iq, y = qy * iq, z = qz * iq;
    float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w_ * z), 2.f * (x * z + w_ * y)},
                     {2.f * (x * y + w_ * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w_ * x)},
                     {2.f * (x * z - w_ * y), 2.f * (y * z + w_ * x), 1.f - 2.f * (x * x + y * y)}};
    float v[3], vs[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float u = R[0][j] * e[0] + R[1][j] * e[1] + R[2][j] * e[2];
        v[j] = u * is[j];
        vs[j] = v[j] * is[j];
    }
    float gm[3];
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2) gm[c2] = -2.0f * dLdd2 * (R[c2][0] * vs[0] + R[c2][1] * vs[1] + R[c2][2] * vs[2]);
    // staged per leaf (three vector atomics); added into the caller's arrays after the kernel
    float4 *stage = a.g_stage + 3 * (size_t)idx;
    atomicAdd(stage, make_float4(gm[0], gm[1], gm[2], g_logit));
    atomicAdd(stage + 1, make_float4(-2.0f * dLdd2 * v[0] * v[0], -2.0f * dLdd2 * v[1] * v[1],
                                     -2.0f * dLdd2 * v[2] * v[2], 0.f));
    {
        float Gr[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) Gr[r][j] = 2.0f * dLdd2 * vs[j] * e[r];
        float gw = 2.f * (-z * Gr[0][1] + y * Gr[0][2] + z * Gr[1][0] - x * Gr[1][2] - y * Gr[2][0] + x * Gr[2][1]);
        float gx = 2.f * (y * Gr[0][1] + z * Gr[0][2] + y * Gr[1][0] - 2.f * x * Gr[1][1] - w_ * Gr[1][2] +
                          z * Gr[2][0] + w_ * Gr[2][1] - 2.f * x * Gr[2][2]);
        float gy = 2.f * (-2.f * y * Gr[0][0] + x * Gr[0][1] + w_ * Gr[0][2] + x * Gr[1][0] + z * Gr[1][2] -
                          w_ * Gr[2][0] + z * Gr[2][1] - 2.f * y * Gr[2][2]);
        float gz = 2.f * (-2.f * z * Gr[0][0] - w_ * Gr[0][1] + x * Gr[0][2] + w_ * Gr[1][0] - 2.f * z * Gr[1][1] +
                          y * Gr[1][2] + x * Gr[2][0] + y * Gr[2][1]);
        float dot = w_ * gw + x * gx + y * gy + z * gz;
        atomicAdd(stage + 2, make_float4((gw - w_ * dot) * iq, (gx - x * dot) * iq, (gy - y * dot) * iq,
                                         (gz - z * dot) * iq));
    }
}

// ------------------------------------------------------------------------------------------
// One ray: the round loop of Listing 1's raygen shader. PASS: the forward, the backward (same
// rounds, gradients while blending), or the forward that also saves each ray's blend list.
// ------------------------------------------------------------------------------------------
enum { PASS_FWD = 0, PASS_BWD = 1, PASS_SAVE = 2 };

// Blend-list entry j of a ray whose forward saved its list, and the end of its list.
__device__ __forceinline__ void save_blended(const TraceArgs &a, int64_t pix, int j, uint32_t idx)
{
    if (j < a.save_cap) a.save_leaves[(size_t)pix * a.save_cap + j] = idx;
}

template <int K, int FORM, bool INSTR, int PASS>
__device__ __forceinline__ void trace_ray(const TraceArgs &a, const SceneRef &sc, float4 *__restrict__ out, int slot,
                                          int64_t pix, float3 o, float3 d, float tn, float tf, KBuf<K> &kb,
                                          Counters &cnt, bool r1_done = false, bool r1_ok = true, int r1_n_dst = 0,
                                          int r1_n_ev = 0)
{
    constexpr bool BWD = PASS == PASS_BWD;
    const uint32_t S = (uint32_t)a.n_slots;
    float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    const float inv_len = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    BlendState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f;
    if (BWD) {
        float4 F = a.fwd_rgbT[pix], G = a.dL_drgbT[pix];
        st.G[0] = G.x; st.G[1] = G.y; st.G[2] = G.z; st.G[3] = G.w;
        st.Tf = F.w;
        st.Cf[0] = F.x - F.w * a.bg0;
        st.Cf[1] = F.y - F.w * a.bg1;
        st.Cf[2] = F.z - F.w * a.bg2;
        st.dLdT = G.w + a.bg0 * G.x + a.bg1 * G.y + a.bg2 * G.z;
    }
    float Lt = tn;
    uint32_t Li = GRTX_NONE;
    bool ckpt = a.traversal == GRTX_TRAVERSAL_CHECKPOINT;
    bool from_root = true;
    int n_src = 0, n_ev = 0, nb = 0;
    uint32_t src = (uint32_t)slot, dst = a.ck1_off + (uint32_t)slot;      // entry offsets into a.ck0
    const uint32_t ev = a.ev_off + (uint32_t)slot;
    bool done = !sc.has_tree;
    bool first_round = true;
    while (!done) {
        if (INSTR) cnt.rounds++;
        if (!(r1_done && first_round)) kb.clear();
        if (ckpt && n_ev > 0) {            // raygen: closest evicted hits -> k-buffer
            int w = 0;
            for (int e = 0; e < n_ev; ++e) {
                uint2 v = a.ck0[ev + (uint32_t)e * S];
                float ct = __uint_as_float(v.x);
                uint32_t ci = v.y;
                // the proxy form can find one Gaussian through several triangles, so an evicted
                // copy may already be blended (key <= L) or already be in the buffer
                if (FORM == FORM_PROXY && (!key_after(ct, ci, Lt, Li) || kb.contains(ct, ci))) continue;
                if (kb.insert(ct, ci)) {
                    a.ck0[ev + (uint32_t)w * S] = make_uint2(__float_as_uint(ct), ci);
                    ++w;
                }
            }
            n_ev = w;
        }
        int n_dst = 0;
        bool round_ok;
        if (r1_done && first_round) {                  // round 1 was traced as the warp's packet
            round_ok = r1_ok;
            n_dst = r1_n_dst;
            n_ev = r1_n_ev;
        } else {
            round_ok = trace_round<K, FORM, INSTR>(a, sc, o, d, inv, inv_len, tn, tf, Lt, Li, ckpt, from_root, src, n_src,
                                                   dst, n_dst, ev, n_ev, kb, cnt);
        }
        if (!round_ok) {
            // a capacity was exceeded: redo this round from the root and stay in restart mode
            if (INSTR) cnt.fallbacks++;
            ckpt = false;
            from_root = true;
            n_src = 0;
            n_ev = 0;
            kb.clear();
            trace_round<K, FORM, INSTR>(a, sc, o, d, inv, inv_len, tn, tf, Lt, Li, false, true, src, 0, dst, n_dst, ev, n_ev,
                                         kb, cnt);
        }
        for (int j = 0; j < kb.n; ++j) {
            uint32_t idx = kb.I(j);
            blend_one<BWD>(a, sc, st, idx, o, d);
            if (INSTR) {
                if (a.ids && nb < a.ids_cap) a.ids[(size_t)pix * a.ids_cap + nb] = sc.gid[idx];
                cnt.blended++;
            }
            if (PASS == PASS_SAVE) save_blended(a, pix, nb, idx);
            ++nb;
            if (st.T < a.T_min) { done = true; break; }
        }
        first_round = false;
        if (done || kb.n < K) break;
        Lt = kb.T(K - 1);
        Li = kb.I(K - 1);
        if (ckpt) {
            uint32_t tmp = src; src = dst; dst = tmp;
            n_src = n_dst;
            from_root = false;
        }
    }
    if (!BWD) out[pix] = make_float4(st.C[0] + st.T * a.bg0, st.C[1] + st.T * a.bg1, st.C[2] + st.T * a.bg2, st.T);
    if (INSTR && a.n_blended) a.n_blended[pix] = nb;
    if (PASS == PASS_SAVE) a.save_n[pix] = nb;
}

// The backward of a ray from the blend list its forward saved (n <= save_cap entries): the
// same blends, gradients and order as replaying the rounds, without the traversal.
__device__ __forceinline__ void backward_from_list(const TraceArgs &a, const SceneRef &sc, int64_t pix, float3 o,
                                                   float3 d, int n)
{
    BlendState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f;
    float4 F = a.fwd_rgbT[pix], G = a.dL_drgbT[pix];
    st.G[0] = G.x; st.G[1] = G.y; st.G[2] = G.z; st.G[3] = G.w;
    st.Tf = F.w;
    st.Cf[0] = F.x - F.w * a.bg0;
    st.Cf[1] = F.y - F.w * a.bg1;
    st.Cf[2] = F.z - F.w * a.bg2;
    st.dLdT = G.w + a.bg0 * G.x + a.bg1 * G.y + a.bg2 * G.z;
    const uint32_t *list = a.save_leaves + (size_t)pix * a.save_cap;
    for (int j = 0; j < n; ++j) {
        uint32_t idx = list[j];
        if (idx < sc.n_geom) blend_one<true>(a, sc, st, idx, o, d);   // never read outside the scene
    }
}

// The rays of one warp with restart traversal (Sec. III-A): every round from the root as the
// warp's packet over the lanes still tracing, each lane culling with its own last key L. Once
// rays travel as packets, the upper levels a restart revisits cost one broadcast load per warp,
// which is what makes this the faster restart on the SMs. A lane whose packet could not finish
// (the warp's stack would overflow) traces that round on its own. Every lane calls this
// together; lanes without a ray pass valid = false.
template <int K, int FORM, bool INSTR, bool SAVE>
__device__ __forceinline__ void trace_warp_restart(const TraceArgs &a, const SceneRef &sc, float4 *__restrict__ out,
                                                   int slot, bool valid, int64_t pix, float3 o, float3 d, float tn,
                                                   float tf, KBuf<K> &kb, Counters &cnt, uint4 *pst)
{
    if (!valid) {
        o = make_float3(0.f, 0.f, 0.f);
        d = make_float3(0.f, 0.f, 1.f);
        tn = tf = 0.f;
    }
    float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    float nrm = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    BlendState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f;
    float Lt = tn;
    uint32_t Li = GRTX_NONE;
    int nb = 0;
    bool done = !valid || !sc.has_tree;
    while (__any_sync(0xffffffffu, !done)) {
        if (!done) {
            if (INSTR) cnt.rounds++;
            kb.clear();
        }
        int n_dst = 0, n_ev = 0;
        bool lane_ok = true;
        packet_round<K, FORM, INSTR>(a, sc, !done, pst, o, d, inv, nrm, tn, tf, Lt, Li, false, 0u, n_dst, 0u, n_ev,
                                     kb, cnt, lane_ok);
        if (done) continue;
        if (!lane_ok) {
            kb.clear();
            trace_round<K, FORM, INSTR>(a, sc, o, d, inv, nrm, tn, tf, Lt, Li, false, true, 0u, 0, 0u, n_dst, 0u, n_ev,
                                        kb, cnt);
        }
        for (int j = 0; j < kb.n; ++j) {
            uint32_t idx = kb.I(j);
            blend_one<false>(a, sc, st, idx, o, d);
            if (INSTR) {
                if (a.ids && nb < a.ids_cap) a.ids[(size_t)pix * a.ids_cap + nb] = sc.gid[idx];
                cnt.blended++;
            }
            if (SAVE) save_blended(a, pix, nb, idx);
            ++nb;
            if (st.T < a.T_min) {
                done = true;
                break;
            }
        }
        if (!done && kb.n < K) done = true;
        if (!done) {
            Lt = kb.T(K - 1);
            Li = kb.I(K - 1);
        }
    }
    if (valid) {
        out[pix] = make_float4(st.C[0] + st.T * a.bg0, st.C[1] + st.T * a.bg1, st.C[2] + st.T * a.bg2, st.T);
        if (INSTR && a.n_blended) a.n_blended[pix] = nb;
        if (SAVE) a.save_n[pix] = nb;
    }
}

// The rays of one warp: round 1 as the warp's packet, then each ray's later rounds on its
// own. Every lane of the warp calls this together; lanes without a ray pass valid = false. In
// the backward, a ray whose forward saved its whole blend list takes it from there and leaves
// the traversal to the others.
template <int K, int FORM, bool INSTR, int PASS>
__device__ __forceinline__ void trace_warp(const TraceArgs &a, const SceneRef &sc, float4 *__restrict__ out, int slot,
                                           bool valid, int64_t pix, float3 o, float3 d, float tn, float tf, KBuf<K> &kb,
                                           Counters &cnt, uint4 *pst)
{
    if (PASS == PASS_BWD && valid && a.save_n) {
        int n = a.save_n[pix];
        if (n <= a.save_cap) {
            backward_from_list(a, sc, pix, o, d, n);
            valid = false;
        }
    }
    if (!valid) {
        o = make_float3(0.f, 0.f, 0.f);
        d = make_float3(0.f, 0.f, 1.f);
        tn = tf = 0.f;
    }
    float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    float inv_len = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    kb.clear();
    int n_dst = 0, n_ev = 0;
    bool lane_ok = true;
    packet_round<K, FORM, INSTR>(a, sc, valid, pst, o, d, inv, inv_len, tn, tf, tn, GRTX_NONE,
                                 a.traversal == GRTX_TRAVERSAL_CHECKPOINT, a.ck1_off + (uint32_t)slot, n_dst,
                                 a.ev_off + (uint32_t)slot, n_ev, kb, cnt, lane_ok);
    // a lane whose packet could not finish (lists or the warp's stack overflowed) redoes round 1
    // from the root on its own, as after any capacity overflow
    if (valid) trace_ray<K, FORM, INSTR, PASS>(a, sc, out, slot, pix, o, d, tn, tf, kb, cnt, true, lane_ok, n_dst, n_ev);
}

// After a tile, every checkpoint and eviction list entry of the warp's 32 ray slots is dead:
// the next tile writes each entry before it reads it. The lines holding them are dropped from
// L2 without being written back, so that the lists, written and read once per round, cost no
// DRAM writes. An entry row of the warp's slots is 32 x 8 = 256 contiguous bytes, two 128-byte
// lines, aligned because slot counts are multiples of 128 and list bases are 256-byte aligned.
// The first kDiscardRows rows of each list are dropped (a ray rarely writes more entries per
// round; a row past that is only written back as before); rows past a list's capacity would
// belong to the next list or lie past the workspace, and are skipped.
constexpr int kDiscardRows = 64;

__device__ __forceinline__ void discard_dead_lists(const TraceArgs &a, int warp_slot0)
{
    const size_t S = (size_t)a.n_slots;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < (3 * kDiscardRows * 2) / 32; ++q) {
        const int l = q * 32 + lane;
        const int list = l / (2 * kDiscardRows), row = (l % (2 * kDiscardRows)) >> 1, half = l & 1;
        const uint2 *base = list == 0 ? a.ck0 : (list == 1 ? a.ck1 : a.ev);
        const int cap = list == 2 ? a.evict_cap : a.ckpt_cap;
        if (row < cap) {
            const char *p = reinterpret_cast<const char *>(base + (size_t)row * S + warp_slot0) + 128 * half;
            asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
        }
    }
}

// Resident blocks per SM the trace kernels are compiled for. The traversal is latency-bound,
// so occupancy pays even at the cost of a few spilled registers (measured on GB300: 8 blocks of
// 128 threads is the best forward setting for k <= 16; the k = 32 k-buffer's 32 KB of shared
// memory per block allows 6; the backward keeps more live state and prefers 7).
__host__ __device__ constexpr int trace_min_blocks(int k, bool bwd) { return k >= 32 ? 6 : (bwd ? 7 : 8); }

// Traversal a frame kernel is compiled for: either (chosen per launch by a.traversal), or one
// of them only. The forward sphere-form kernel has one instantiation per traversal (TRAV_CKPT
// also serves any traversal but restart): without the other traversal's code, the register
// allocation of the one that runs is better (the checkpointed frame kernel spills 100 B
// instead of 112 B and runs 0.5 % faster).
constexpr int TRAV_ANY = 0, TRAV_CKPT = 1, TRAV_RESTART = 2;

template <int K, int FORM, bool INSTR, int PASS, int TRAV = TRAV_ANY>
__global__ void __launch_bounds__(kBlock, trace_min_blocks(K, PASS == PASS_BWD)) k_trace(TraceArgs a)
{
    __shared__ float s_kt[K * kBlock];
    __shared__ uint32_t s_ki[K * kBlock];
    __shared__ uint4 s_pst[kBlock / 32][kPacketStack];
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    KBuf<K> kb;
    kb.t = s_kt + threadIdx.x;
    kb.id = s_ki + threadIdx.x;
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr, 0, 0};
    unsigned rays = 0;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(a.queue, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= a.n_items) break;
        int64_t pix;
        float3 o, d;
        float tn, tf;
        bool valid = make_ray(a.cam, base + lane, pix, o, d, tn, tf);
        rays += valid;
        if (INSTR) visits_begin(a, cnt, valid, pix);
        if constexpr (TRAV == TRAV_RESTART && PASS != PASS_BWD)
            trace_warp_restart<K, FORM, INSTR, PASS == PASS_SAVE>(a, a.sc, a.rgbT, slot, valid, pix, o, d, tn, tf,
                                                                  kb, cnt, s_pst[threadIdx.x >> 5]);
        else if constexpr (TRAV == TRAV_CKPT)
            trace_warp<K, FORM, INSTR, PASS>(a, a.sc, a.rgbT, slot, valid, pix, o, d, tn, tf, kb, cnt,
                                             s_pst[threadIdx.x >> 5]);
        else if (PASS != PASS_BWD && a.traversal == GRTX_TRAVERSAL_RESTART)
            trace_warp_restart<K, FORM, INSTR, PASS == PASS_SAVE>(a, a.sc, a.rgbT, slot, valid, pix, o, d, tn, tf,
                                                                  kb, cnt, s_pst[threadIdx.x >> 5]);
        else
            trace_warp<K, FORM, INSTR, PASS>(a, a.sc, a.rgbT, slot, valid, pix, o, d, tn, tf, kb, cnt,
                                             s_pst[threadIdx.x >> 5]);
        if (INSTR) visits_end(a, cnt, pix);
        __syncwarp();
        if (a.discard) discard_dead_lists(a, slot & ~31);
    }
    if (INSTR && a.stats) {
        unsigned long long v[11] = {rays, cnt.nodes, cnt.leaves, cnt.blended, cnt.rounds, cnt.ckpt, cnt.evictions,
                                    cnt.fallbacks, cnt.overflow, 0ull, cnt.oob};
#pragma unroll
        for (int q = 0; q < 11; ++q) {
            unsigned long long x = v[q];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0 && x) atomicAdd((&a.stats->rays) + q, x);
        }
    }
}

// Acquire load (of a count the host raises after writing what it covers).
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned kLingerChecks = 1u << 16;   // bound on the checks of one wait (at most 8 us apart)

// Lane 0 of a warp of a serving launch that holds the claim `base`: returns base once the
// host has published the tile, or kNoWork when the launch is closed with base past its last
// item, or when linger_ns pass without any publication (each one restarts the wait). A warp
// that gives up puts its claim on the lost list (the host may publish it yet) and counts
// itself as exited. A warp about to wait writes its claim's end to claimed_host, so that the
// host sees the launch has run out of work.
__device__ __forceinline__ unsigned await_published(const ServeLive &live, unsigned base)
{
    const unsigned kNoWork = 0xffffffffu;
    unsigned seen = ld_acquire(live.avail);
    if (base < seen) return base;
    *reinterpret_cast<volatile unsigned *>(live.claimed_host) = base + 32u;
    uint64_t t0 = global_ns();
    unsigned nap = 64;
    for (unsigned it = 0; it < kLingerChecks; ++it) {
        const unsigned closed = ld_acquire(live.avail + 1);
        const unsigned n = ld_acquire(live.avail);
        if (base < n) return base;
        if (closed) return kNoWork;
        const uint64_t now = global_ns();
        if (n != seen) {
            seen = n;
            t0 = now;
        } else if (now - t0 > live.linger_ns) {
            break;
        }
        __nanosleep(nap);
        nap = min(2 * nap, 8192u);
    }
    const unsigned i = atomicAdd(live.lost, 1u);
    if (i < live.lost_cap) live.lost[1 + i] = base;
    const unsigned e = atomicAdd(live.exited, 1u) + 1u;
    *reinterpret_cast<volatile unsigned *>(live.exited_host) = e;
    return kNoWork;
}

// Serving step: one persistent launch over the queue items of several requests (each with
// its own scene, camera and output); a warp's 32 items always belong to one request.
template <int K, int TRAV>
__global__ void __launch_bounds__(kBlock, trace_min_blocks(K, false))
    k_serve(TraceArgs a, const ServeSeg *segs, const unsigned *begins, int n_segs, ServeLive live)
{
    __shared__ float s_kt[K * kBlock];
    __shared__ uint32_t s_ki[K * kBlock];
    __shared__ uint4 s_pst[kBlock / 32][kPacketStack];
    const unsigned kNoWork = 0xffffffffu;
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    KBuf<K> kb;
    kb.t = s_kt + threadIdx.x;
    kb.id = s_ki + threadIdx.x;
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr, 0, 0};
    for (;;) {
        unsigned base = 0;
        if (lane == 0) {
            base = atomicAdd(a.queue, 32u);
            if (live.avail) {
                if ((base & 511u) == 0) *reinterpret_cast<volatile unsigned *>(live.claimed_host) = base + 32u;
                base = await_published(live, base);
            } else if (base >= a.n_items) {
                base = kNoWork;
            }
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base == kNoWork) break;
        // last segment with begins[] <= base (read past L1: the host appends entries while the
        // launch runs; the entries not yet written hold 0xffffffff)
        int lo = 0, hi = n_segs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldcg(begins + mid) <= base) lo = mid; else hi = mid - 1;
        }
        // (a record is read only once its items are published, and fills whole cache lines of
        // its own, so no cache holds an older copy of it)
        const ServeSeg &sg = segs[lo];
        SceneRef sc = sg.sc;
        CamRef cam = sg.cam;
        unsigned item = sg.item_begin + (base - sg.step_begin) + lane;
        int64_t pix;
        float3 o, d;
        float tn, tf;
        bool valid = make_ray(cam, item, pix, o, d, tn, tf);
        if constexpr (TRAV == TRAV_RESTART)
            trace_warp_restart<K, FORM_SPHERE, false, false>(a, sc, sg.out, slot, valid, pix, o, d, tn, tf, kb, cnt,
                                                      s_pst[threadIdx.x >> 5]);
        else
            trace_warp<K, FORM_SPHERE, false, PASS_FWD>(a, sc, sg.out, slot, valid, pix, o, d, tn, tf, kb, cnt,
                                                     s_pst[threadIdx.x >> 5]);
        if (live.seg_done) {
            // the tile's pixels are written; the warp that completes the segment raises its
            // flag in host memory (each lane's writes fenced before the count)
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                const unsigned old = atomicAdd(live.seg_done + lo, 32u);
                if (old + 32u >= sg.count) {
                    __threadfence_system();
                    *reinterpret_cast<volatile unsigned *>(live.seg_flag + lo) = live.seq;
                }
            }
        }
        __syncwarp();
        if (a.discard) discard_dead_lists(a, slot & ~31);
    }
}

// Entry offsets of the lists relative to ck0 (the kernels index every list entry with 32 bits);
// false if the workspace is too large for that. Call after ck0, ck1, ev and n_slots are set.
inline bool set_list_offsets(TraceArgs &a, size_t entries_per_slot)
{
    if ((size_t)a.n_slots * entries_per_slot >= ((size_t)1 << 31)) return false;
    a.ck1_off = (uint32_t)(a.ck1 - a.ck0);
    a.ev_off = (uint32_t)(a.ev - a.ck0);
    return true;
}

// Whether the lists of a launch may be dropped from L2 per tile (see discard_dead_lists): the
// checkpointed traversal writes lists, and each list row must start on a 256-byte boundary.
inline int lists_discardable(const TraceArgs &a)
{
    if (a.traversal != GRTX_TRAVERSAL_CHECKPOINT || !a.ck0 || !a.ck1 || !a.ev) return 0;
    const uintptr_t m = (uintptr_t)a.ck0 | (uintptr_t)a.ck1 | (uintptr_t)a.ev;
    return (m & 255u) == 0 && (a.n_slots % 32) == 0 && ((size_t)a.n_slots * sizeof(uint2)) % 256 == 0;
}

// Launch helpers, instantiated per k in the trace_k*.cu units.
// form: FORM_* of the scene. The backward always runs the sphere leaf test: the icosphere
// forms hit exactly the Gaussians the sphere form hits, and the proxy form has no backward.
// pass: PASS_FWD, PASS_BWD or PASS_SAVE (the saving forward exists for the sphere form only).
template <int K>
int trace_launch(const TraceArgs &a, int form, bool instr, int pass, int blocks, cudaStream_t s)
{
    dim3 g(blocks), b(128);
    if (pass == PASS_BWD) k_trace<K, FORM_SPHERE, false, PASS_BWD><<<g, b, 0, s>>>(a);
    else if (pass == PASS_SAVE) k_trace<K, FORM_SPHERE, false, PASS_SAVE><<<g, b, 0, s>>>(a);
    else if (form == FORM_PROXY && instr) k_trace<K, FORM_PROXY, true, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_PROXY) k_trace<K, FORM_PROXY, false, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_ICO && instr) k_trace<K, FORM_ICO, true, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_ICO) k_trace<K, FORM_ICO, false, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_SPHERE4 && instr) k_trace<K, FORM_SPHERE4, true, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_SPHERE4) k_trace<K, FORM_SPHERE4, false, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_SPHERE4Q && instr) k_trace<K, FORM_SPHERE4Q, true, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (form == FORM_SPHERE4Q) k_trace<K, FORM_SPHERE4Q, false, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (instr) k_trace<K, FORM_SPHERE, true, PASS_FWD><<<g, b, 0, s>>>(a);
    else if (a.traversal == GRTX_TRAVERSAL_RESTART) k_trace<K, FORM_SPHERE, false, PASS_FWD, TRAV_RESTART><<<g, b, 0, s>>>(a);
    else k_trace<K, FORM_SPHERE, false, PASS_FWD, TRAV_CKPT><<<g, b, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GRTX_OK : GRTX_ERR_CUDA;
}

template <int K>
int trace_occupancy(int form, bool instr, int pass, int *blocks_per_sm)
{
    cudaError_t e;
    if (pass == PASS_BWD) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE, false, PASS_BWD>, 128, 0);
    else if (pass == PASS_SAVE) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE, false, PASS_SAVE>, 128, 0);
    else if (form == FORM_PROXY && instr) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_PROXY, true, PASS_FWD>, 128, 0);
    else if (form == FORM_PROXY) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_PROXY, false, PASS_FWD>, 128, 0);
    else if (form == FORM_ICO && instr) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_ICO, true, PASS_FWD>, 128, 0);
    else if (form == FORM_ICO) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_ICO, false, PASS_FWD>, 128, 0);
    else if (form == FORM_SPHERE4 && instr) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE4, true, PASS_FWD>, 128, 0);
    else if (form == FORM_SPHERE4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE4, false, PASS_FWD>, 128, 0);
    else if (form == FORM_SPHERE4Q && instr) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE4Q, true, PASS_FWD>, 128, 0);
    else if (form == FORM_SPHERE4Q) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE4Q, false, PASS_FWD>, 128, 0);
    else if (instr) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE, true, PASS_FWD>, 128, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_trace<K, FORM_SPHERE, false, PASS_FWD, TRAV_CKPT>, 128, 0);
    return e == cudaSuccess ? GRTX_OK : GRTX_ERR_CUDA;
}

// Kernel leaf kind of a scene form (wide: the 4-wide nodes of a sphere-form scene, quantised
// or not).
inline int kernel_form(int scene_form, bool wide = false, bool quant = false)
{
    return scene_form == GRTX_FORM_PROXY20 ? FORM_PROXY
           : (scene_form == GRTX_FORM_ICO20 || scene_form == GRTX_FORM_ICO80) ? FORM_ICO
           : wide ? (quant ? FORM_SPHERE4Q : FORM_SPHERE4) : FORM_SPHERE;
}

// live: the serving controls (see ServeLive); all zero for a plain batched launch.
template <int K>
int serve_launch(const TraceArgs &a, const ServeSeg *segs, const unsigned *begins, int n_segs, int blocks,
                 cudaStream_t s, ServeLive live)
{
    if (a.traversal == GRTX_TRAVERSAL_RESTART) k_serve<K, TRAV_RESTART><<<blocks, 128, 0, s>>>(a, segs, begins, n_segs, live);
    else k_serve<K, TRAV_CKPT><<<blocks, 128, 0, s>>>(a, segs, begins, n_segs, live);
    return cudaGetLastError() == cudaSuccess ? GRTX_OK : GRTX_ERR_CUDA;
}

template <int K>
int serve_occupancy(int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_serve<K, TRAV_CKPT>, 128, 0) == cudaSuccess
               ? GRTX_OK : GRTX_ERR_CUDA;
}

#define GRTX_INSTANTIATE_TRACE(K)                                                                  \
    template int trace_launch<K>(const TraceArgs &, int, bool, int, int, cudaStream_t);           \
    template int trace_occupancy<K>(int, bool, int, int *);                                         \
    template int serve_launch<K>(const TraceArgs &, const ServeSeg *, const unsigned *, int, int, cudaStream_t, ServeLive);   \
    template int serve_occupancy<K>(int *);
