// Secondary rays off planar rectangular mirrors and through glass balls (Sec. VI "GRTX-HW on
// Secondary Rays": a rectangular mirror and a spherical glass object placed in the scene,
// primary and secondary rays traced separately). Primary rays stop at the nearest object;
// each primary that hits one spawns one reflected or refracted ray; the secondary image is
// composited behind the primary's Gaussians.
#include <cuda_runtime.h>

#include "trace_impl.cuh"

int grtx_fill_camera(CamRef &a, unsigned &n_items_out, const grtx_camera *cam);

namespace {

__global__ void k_mirror_rays(CamRef cam, grtx_mirror m, float *__restrict__ po, float *__restrict__ pd,
                              float *__restrict__ ptn, float *__restrict__ ptf, float *__restrict__ so,
                              float *__restrict__ sd, float *__restrict__ stn, float *__restrict__ stf,
                              int32_t *__restrict__ spix, int32_t *__restrict__ n_sec)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = (int64_t)cam.width * cam.height;
    bool hit = false;
    float3 o = make_float3(0.f, 0.f, 0.f), d = o, q = o, r = o;
    int64_t pix = -1;
    if (p < n) {
        unsigned item = item_of_pixel(cam, p);
        float tn, tf;
        if (make_ray(cam, item, pix, o, d, tn, tf)) {
            const float3 c = make_float3(m.center[0], m.center[1], m.center[2]);
            const float3 nn = make_float3(m.normal[0], m.normal[1], m.normal[2]);
            float den = d.x * nn.x + d.y * nn.y + d.z * nn.z;
            if (fabsf(den) > 1e-20f) {
                float t = ((c.x - o.x) * nn.x + (c.y - o.y) * nn.y + (c.z - o.z) * nn.z) / den;
                if (t > tn && t < tf) {
                    q = make_float3(fmaf(t, d.x, o.x), fmaf(t, d.y, o.y), fmaf(t, d.z, o.z));
                    float du = (q.x - c.x) * m.axis_u[0] + (q.y - c.y) * m.axis_u[1] + (q.z - c.z) * m.axis_u[2];
                    float dv = (q.x - c.x) * m.axis_v[0] + (q.y - c.y) * m.axis_v[1] + (q.z - c.z) * m.axis_v[2];
                    if (fabsf(du) <= m.half_u && fabsf(dv) <= m.half_v) {
                        hit = true;
                        tf = t;
                        float k2 = 2.0f * den;
                        r = make_float3(d.x - k2 * nn.x, d.y - k2 * nn.y, d.z - k2 * nn.z);
                    }
                }
            }
            po[3 * pix] = o.x; po[3 * pix + 1] = o.y; po[3 * pix + 2] = o.z;
            pd[3 * pix] = d.x; pd[3 * pix + 1] = d.y; pd[3 * pix + 2] = d.z;
            ptn[pix] = tn;
            ptf[pix] = tf;
        }
    }
    // warp-aggregated compaction keeps each warp's secondary rays together and in pixel order
    unsigned mask = __ballot_sync(0xffffffffu, hit);
    int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(n_sec, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) {
        int j = base + __popc(mask & ((1u << lane) - 1u));
        so[3 * j] = q.x; so[3 * j + 1] = q.y; so[3 * j + 2] = q.z;
        sd[3 * j] = r.x; sd[3 * j + 1] = r.y; sd[3 * j + 2] = r.z;
        stn[j] = m.t_near_secondary;
        stf[j] = INFINITY;
        spix[j] = (int32_t)pix;
    }
}

struct BounceObjects {
    grtx_mirror m[GRTX_MAX_BOUNCE_OBJECTS];
    grtx_glass g[GRTX_MAX_BOUNCE_OBJECTS];
    int nm, ng;
};

__device__ __forceinline__ float3 f3(const float *v) { return make_float3(v[0], v[1], v[2]); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 axpy(float s, float3 x, float3 y)
{
    return make_float3(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z));
}
__device__ __forceinline__ float3 unit(float3 v)
{
    float r = rsqrtf(dot3(v, v));
    return make_float3(v.x * r, v.y * r, v.z * r);
}

// Snell refraction of unit I at unit normal N facing against I, eta = n_from / n_to.
__device__ __forceinline__ float3 refract(float3 I, float3 N, float eta)
{
    float ci = -dot3(N, I);
    float k = 1.0f - eta * eta * (1.0f - ci * ci);
    float ct = k > 0.0f ? sqrtf(k) : 0.0f;
    return axpy(eta * ci - ct, N, make_float3(eta * I.x, eta * I.y, eta * I.z));
}

__global__ void k_secondary_rays(CamRef cam, BounceObjects ob, float *__restrict__ po, float *__restrict__ pd,
                                 float *__restrict__ ptn, float *__restrict__ ptf, float *__restrict__ so,
                                 float *__restrict__ sd, float *__restrict__ stn, float *__restrict__ stf,
                                 int32_t *__restrict__ spix, int32_t *__restrict__ n_sec)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = (int64_t)cam.width * cam.height;
    bool hit = false;
    float3 q = make_float3(0.f, 0.f, 0.f), r = q;
    float s_tn = 0.f;
    int64_t pix = -1;
    if (p < n) {
        unsigned item = item_of_pixel(cam, p);
        float3 o, d;
        float tn, tf;
        if (make_ray(cam, item, pix, o, d, tn, tf)) {
            float t_best = tf;
            int kind = 0, which = 0;
            for (int i = 0; i < ob.nm; ++i) {
                const grtx_mirror &m = ob.m[i];
                float3 c = f3(m.center), nn = f3(m.normal);
                float den = dot3(d, nn);
                if (fabsf(den) <= 1e-20f) continue;
                float t = dot3(make_float3(c.x - o.x, c.y - o.y, c.z - o.z), nn) / den;
                if (!(t > tn && t < t_best)) continue;
                float3 h = axpy(t, d, make_float3(o.x - c.x, o.y - c.y, o.z - c.z));
                if (fabsf(dot3(h, f3(m.axis_u))) > m.half_u || fabsf(dot3(h, f3(m.axis_v))) > m.half_v) continue;
                t_best = t;
                kind = 1;
                which = i;
            }
            for (int i = 0; i < ob.ng; ++i) {
                const grtx_glass &g = ob.g[i];
                float3 oc = make_float3(o.x - g.center[0], o.y - g.center[1], o.z - g.center[2]);
                float b = dot3(oc, d), cc = dot3(oc, oc) - g.radius * g.radius;
                if (!(cc > 0.0f)) continue;                 // starts inside (or on) the ball
                float disc = b * b - dot3(d, d) * cc;
                if (!(disc > 0.0f)) continue;
                float den = sqrtf(disc) - b;                // = a * (far root) > 0 when ahead
                if (!(den > 0.0f)) continue;
                float t = cc / den;                         // near root without cancellation
                if (!(t > tn && t < t_best)) continue;
                t_best = t;
                kind = 2;
                which = i;
            }
            if (kind == 1) {
                const grtx_mirror &m = ob.m[which];
                float3 nn = f3(m.normal);
                float k2 = 2.0f * dot3(d, nn);
                q = axpy(t_best, d, o);
                r = make_float3(d.x - k2 * nn.x, d.y - k2 * nn.y, d.z - k2 * nn.z);
                s_tn = m.t_near_secondary;
            } else if (kind == 2) {
                const grtx_glass &g = ob.g[which];
                float3 c = f3(g.center);
                float3 rel1 = axpy(t_best, d, make_float3(o.x - c.x, o.y - c.y, o.z - c.z));
                float3 v = unit(refract(unit(d), unit(rel1), 1.0f / g.ior));
                float t2 = -2.0f * dot3(v, rel1);
                float3 rel2 = axpy(t2, v, rel1);
                float3 n2 = unit(rel2);
                r = unit(refract(v, make_float3(-n2.x, -n2.y, -n2.z), g.ior));
                q = make_float3(c.x + rel2.x, c.y + rel2.y, c.z + rel2.z);
                s_tn = g.t_near_secondary;
            }
            hit = kind != 0;
            if (hit) tf = t_best;
            po[3 * pix] = o.x; po[3 * pix + 1] = o.y; po[3 * pix + 2] = o.z;
            pd[3 * pix] = d.x; pd[3 * pix + 1] = d.y; pd[3 * pix + 2] = d.z;
            ptn[pix] = tn;
            ptf[pix] = tf;
        }
    }
    unsigned mask = __ballot_sync(0xffffffffu, hit);
    int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(n_sec, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (hit) {
        int j = base + __popc(mask & ((1u << lane) - 1u));
        so[3 * j] = q.x; so[3 * j + 1] = q.y; so[3 * j + 2] = q.z;
        sd[3 * j] = r.x; sd[3 * j + 1] = r.y; sd[3 * j + 2] = r.z;
        stn[j] = s_tn;
        stf[j] = INFINITY;
        spix[j] = (int32_t)pix;
    }
}

__global__ void k_composite_bounce(float4 *__restrict__ rgbT, const float4 *__restrict__ sec, const int32_t *__restrict__ spix,
                                   const int32_t *__restrict__ n_sec, float bg0, float bg1, float bg2)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *n_sec) return;
    int p = spix[j];
    float4 a = rgbT[p], b = sec[j];
    // the primary's background term T bg is replaced by T times the reflected radiance
    rgbT[p] = make_float4(a.x + a.w * (b.x - bg0), a.y + a.w * (b.y - bg1), a.z + a.w * (b.z - bg2), a.w * b.w);
}

}  // namespace

extern "C" GRTX_API int grtx_mirror_rays(const grtx_camera *cam, const grtx_mirror *m, float *d_prim_origins,
                                         float *d_prim_dirs, float *d_prim_tnear, float *d_prim_tfar,
                                         float *d_sec_origins, float *d_sec_dirs, float *d_sec_tnear,
                                         float *d_sec_tfar, int32_t *d_sec_pixel, int32_t *d_n_sec, void *stream)
{
    CamRef c = {};
    unsigned items = 0;
    int st = grtx_fill_camera(c, items, cam);
    if (st) return st;
    if (!m || !(m->half_u >= 0.f) || !(m->half_v >= 0.f) || !(m->t_near_secondary >= 0.f))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "bad mirror");
    if (!d_prim_origins || !d_prim_dirs || !d_prim_tnear || !d_prim_tfar || !d_sec_origins || !d_sec_dirs ||
        !d_sec_tnear || !d_sec_tfar || !d_sec_pixel || !d_n_sec)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL output");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t n = (int64_t)cam->width * cam->height;
    GRTX_CUDA(cudaMemsetAsync(d_n_sec, 0, sizeof(int32_t), s));
    k_mirror_rays<<<grtx_div_up(n, 256), 256, 0, s>>>(c, *m, d_prim_origins, d_prim_dirs, d_prim_tnear, d_prim_tfar,
                                                      d_sec_origins, d_sec_dirs, d_sec_tnear, d_sec_tfar, d_sec_pixel,
                                                      d_n_sec);
    GRTX_CHECK_LAUNCH("grtx_mirror_rays");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_secondary_rays(const grtx_camera *cam, const grtx_mirror *mirrors, int n_mirrors,
                                            const grtx_glass *glass, int n_glass, float *d_prim_origins,
                                            float *d_prim_dirs, float *d_prim_tnear, float *d_prim_tfar,
                                            float *d_sec_origins, float *d_sec_dirs, float *d_sec_tnear,
                                            float *d_sec_tfar, int32_t *d_sec_pixel, int32_t *d_n_sec, void *stream)
{
    CamRef c = {};
    unsigned items = 0;
    int st = grtx_fill_camera(c, items, cam);
    if (st) return st;
    if (n_mirrors < 0 || n_mirrors > GRTX_MAX_BOUNCE_OBJECTS || n_glass < 0 || n_glass > GRTX_MAX_BOUNCE_OBJECTS)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "object counts must be in [0, GRTX_MAX_BOUNCE_OBJECTS]");
    if ((n_mirrors > 0 && !mirrors) || (n_glass > 0 && !glass)) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL object list");
    BounceObjects ob = {};
    ob.nm = n_mirrors;
    ob.ng = n_glass;
    for (int i = 0; i < n_mirrors; ++i) {
        const grtx_mirror &m = mirrors[i];
        if (!(m.half_u >= 0.f) || !(m.half_v >= 0.f) || !(m.t_near_secondary >= 0.f))
            return grtx_fail(GRTX_ERR_INVALID_ARG, "bad mirror");
        ob.m[i] = m;
    }
    for (int i = 0; i < n_glass; ++i) {
        const grtx_glass &g = glass[i];
        if (!(g.radius > 0.f) || !(g.ior > 0.f) || !(g.t_near_secondary >= 0.f))
            return grtx_fail(GRTX_ERR_INVALID_ARG, "bad glass ball");
        ob.g[i] = g;
    }
    if (!d_prim_origins || !d_prim_dirs || !d_prim_tnear || !d_prim_tfar || !d_sec_origins || !d_sec_dirs ||
        !d_sec_tnear || !d_sec_tfar || !d_sec_pixel || !d_n_sec)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL output");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t n = (int64_t)cam->width * cam->height;
    GRTX_CUDA(cudaMemsetAsync(d_n_sec, 0, sizeof(int32_t), s));
    k_secondary_rays<<<grtx_div_up(n, 256), 256, 0, s>>>(c, ob, d_prim_origins, d_prim_dirs, d_prim_tnear,
                                                         d_prim_tfar, d_sec_origins, d_sec_dirs, d_sec_tnear,
                                                         d_sec_tfar, d_sec_pixel, d_n_sec);
    GRTX_CHECK_LAUNCH("grtx_secondary_rays");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_composite_bounce(float *d_rgbT, const float *d_sec_rgbT, const int32_t *d_sec_pixel,
                                              const int32_t *d_n_sec, int64_t max_sec, const float bg[3], void *stream)
{
    if (!d_rgbT || !d_sec_rgbT || !d_sec_pixel || !d_n_sec || !bg || max_sec < 0)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "bad composite arguments");
    if (((uintptr_t)d_rgbT & 15) || ((uintptr_t)d_sec_rgbT & 15))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "image buffers must be 16-byte aligned");
    if (max_sec == 0) return GRTX_OK;
    k_composite_bounce<<<grtx_div_up(max_sec, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        (float4 *)d_rgbT, (const float4 *)d_sec_rgbT, d_sec_pixel, d_n_sec, bg[0], bg[1], bg[2]);
    GRTX_CHECK_LAUNCH("grtx_composite_bounce");
    return GRTX_OK;
}
