// Multi-level instancing (Sec. VI "Support for Dynamic and Multi-Object Scenes"): a world of
// placed objects. Each object is a built sphere-form scene (its own instance BVH over unit
// spheres); a scene-level BVH (TLAS) over the objects' world boxes sits on top. The trace is
// the k-buffer round loop of the single-scene kernel over this two-level structure: at a TLAS
// leaf the ray is mapped into the object's frame and descends its BVH, and traversal entries
// (stack and checkpoint lists) carry the instance of object-level nodes, as the paper's
// checkpoint entry carries a TLAS-leaf address for BLAS nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "host_bvh.h"
#include "trace_impl.cuh"

int grtx_fill_camera(CamRef &a, unsigned &n_items_out, const grtx_camera *cam);
SceneRef grtx_scene_ref(const grtx_scene *sc);
int grtx_check_params(const grtx_params *p);

namespace {

constexpr int kWorldStack = 32 + GRTX_STACK;   // TLAS depth (<= 32) + object depth (< GRTX_STACK)
constexpr int kMaxTlasDepth = 32;

struct InstRec {
    float4 w2o[3];            // rows (L^-1 | -L^-1 c): x_object = w2o (x_world, 1)
    SceneRef sc;
    uint32_t leaf_base;       // world leaf index of the object's leaf 0
    uint32_t id_base;         // world Gaussian id of the object's Gaussian 0
    uint32_t pad0, pad1;
};

struct WorldArgs {
    TraceArgs a;              // camera, parameters, outputs, eviction list, queue
    const float4 *tl_nodes;   // scene-level BVH, leaf ref = row of inst
    const InstRec *inst;      // non-empty instances
    const uint32_t *leaf_base;// inst[i].leaf_base, ascending
    int n_inst, n_tl_nodes;
    uint4 *wck0, *wck1;       // checkpoint lists of (ref, t bits, instance, 0), [entry][slot]
};

// The self-check of the instrumented kernels (see ref_ok) at either level of the world.
__device__ __forceinline__ bool world_ref_ok(const WorldArgs &W, uint32_t inst, uint32_t ref, Counters &c,
                                             bool count = true)
{
    if (inst != GRTX_NONE) return ref_ok(W.inst[inst].sc, ref, c, count);
    bool ok = (ref & GRTX_LEAF) ? (ref & ~GRTX_LEAF) < (uint32_t)W.n_inst : ref < (uint32_t)W.n_tl_nodes;
    if (!ok && count) ++c.oob;
    return ok;
}

__device__ __forceinline__ void to_object(const InstRec &I, float3 o, float3 d, float3 &oo, float3 &od)
{
    float4 r0 = I.w2o[0], r1 = I.w2o[1], r2 = I.w2o[2];
    oo = make_float3(fmaf(r0.x, o.x, fmaf(r0.y, o.y, fmaf(r0.z, o.z, r0.w))),
                     fmaf(r1.x, o.x, fmaf(r1.y, o.y, fmaf(r1.z, o.z, r1.w))),
                     fmaf(r2.x, o.x, fmaf(r2.y, o.y, fmaf(r2.z, o.z, r2.w))));
    od = make_float3(fmaf(r0.x, d.x, fmaf(r0.y, d.y, r0.z * d.z)), fmaf(r1.x, d.x, fmaf(r1.y, d.y, r1.z * d.z)),
                     fmaf(r2.x, d.x, fmaf(r2.y, d.y, r2.z * d.z)));
}

// Row of the instance holding world leaf index key (the last i with leaf_base[i] <= key).
__device__ __forceinline__ int find_instance(const WorldArgs &W, uint32_t key)
{
    int lo = 0, hi = W.n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(W.leaf_base + mid) <= key) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One round over keys in (L, t_max] through the two-level structure (see trace_round).
template <int K, bool INSTR>
__device__ __forceinline__ bool world_round(const WorldArgs &W, float3 o, float3 d, float3 inv, float tn, float tf,
                                            float Lt, uint32_t Li, bool ckpt, bool from_root,
                                            const uint4 *__restrict__ src, int n_src, uint4 *__restrict__ dst,
                                            int &n_dst, uint2 *__restrict__ ev, int &n_ev, KBuf<K> &kb,
                                            Counters &cnt)
{
    const size_t S = (size_t)W.a.n_slots;
    // far children still to visit: node ref and instance (a popped node is entered without the
    // t_max test of its entry, -inf: its children are tested, which is exact and halves the
    // stack's local-memory traffic against keeping the entry distance)
    uint2 stack[kWorldStack];
    int sp = 0, si = 0;
    float tmax = kb.tmax;
    uint32_t ref, inst;
    float te;
    n_dst = 0;
    if (from_root) {
        n_src = 0;
        ref = 0u;
        inst = GRTX_NONE;
        te = tn;
    } else {
        if (n_src == 0) return true;
        uint4 v = src[0];
        ref = v.x;
        te = __uint_as_float(v.y);
        inst = v.z;
        si = 1;
    }
    uint32_t cur = GRTX_NONE;
    float3 ob = o, db = d, ib = inv;
    const float4 *nodes = W.tl_nodes, *geom = nullptr;
    uint32_t base = 0;
    for (;;) {
        if (inst != cur) {                            // entering another level: map the ray
            cur = inst;
            if (inst == GRTX_NONE) {
                ob = o;
                db = d;
                ib = inv;
                nodes = W.tl_nodes;
            } else {
                const InstRec &I = W.inst[inst];
                to_object(I, o, d, ob, db);
                ib = make_float3(safe_rcp(db.x), safe_rcp(db.y), safe_rcp(db.z));
                nodes = I.sc.nodes;
                geom = I.sc.geom;
                base = I.leaf_base;
            }
        }
        if (te > tmax) {                              // fails the t_max test
            if (ckpt) {
                if (n_dst >= W.a.ckpt_cap) return false;
                dst[(size_t)n_dst * S] = make_uint4(ref, __float_as_uint(te), inst, 0u);
                ++n_dst;
                if (INSTR) cnt.ckpt++;
            }
        } else if (INSTR && !world_ref_ok(W, inst, ref, cnt)) {   // not fetched (self-check)
        } else if (ref & GRTX_LEAF) {
            if (inst == GRTX_NONE) {                  // TLAS leaf: descend into the object's root
                inst = ref & ~GRTX_LEAF;
                ref = 0u;
                continue;
            }
            uint32_t gi = ref & ~GRTX_LEAF;
            if (INSTR) cnt.leaves++;
            float t, D2, w[3];
            if (sphere_test(geom + 4 * (size_t)gi, ob, db, t, D2, w)) {
                uint32_t key = base + gi;
                if (D2 <= 1.0f && t > tn && t <= tf && key_after(t, key, Lt, Li)) {
                    float ct = t;
                    uint32_t ci = key;
                    if (kb.insert(ct, ci) && ckpt) {
                        if (n_ev >= W.a.evict_cap) return false;
                        ev[(size_t)n_ev * S] = make_uint2(__float_as_uint(ct), ci);
                        ++n_ev;
                        if (INSTR) cnt.evictions++;
                    }
                    tmax = kb.tmax;
                }
            }
        } else {
            if (INSTR) cnt.nodes++;
            const float4 *nd = nodes + 4 * (size_t)ref;
            float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
            float e0, x0, e1, x1;
            slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ob, ib, tn, tf, e0, x0);
            slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ob, ib, tn, tf, e1, x1);
            bool h0 = e0 <= x0 && !(x0 < Lt);
            bool h1 = e1 <= x1 && !(x1 < Lt) && c1 != GRTX_NONE;
            bool near0 = e0 <= e1;
            if (h0 && h1) {
                uint32_t far_ref = near0 ? c1 : c0;
                float far_t = near0 ? e1 : e0;
                ref = near0 ? c0 : c1;
                te = near0 ? e0 : e1;
                if (far_t > tmax) {
                    if (ckpt) {
                        if (n_dst >= W.a.ckpt_cap) return false;
                        dst[(size_t)n_dst * S] = make_uint4(far_ref, __float_as_uint(far_t), inst, 0u);
                        ++n_dst;
                        if (INSTR) cnt.ckpt++;
                    }
                } else if (sp < kWorldStack) {
                    stack[sp++] = make_uint2(far_ref, inst);
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
            --sp;
            ref = stack[sp].x;
            te = -GRTX_INF;
            inst = stack[sp].y;
        } else if (si < n_src) {
            uint4 v = src[(size_t)si * S];
            ++si;
            ref = v.x;
            te = __uint_as_float(v.y);
            inst = v.z;
        } else {
            break;
        }
    }
    return true;
}

// Round 1 of a warp's rays through the world as one packet (see packet_round): the warp walks
// one sequence of TLAS and object nodes, each lane with its own ray in the current object's
// frame, entry tests, k-buffer and lists. Stack entries carry the instance of object-level
// nodes. Every lane of the warp calls this together; lanes without a ray pass valid = false.
template <int K, bool INSTR>
__device__ __forceinline__ void world_packet_round(const WorldArgs &W, bool valid, uint4 *pst, float3 o, float3 d,
                                                   float3 inv, float tn, float tf, bool ckpt, uint4 *__restrict__ dst,
                                                   int &n_dst, uint2 *__restrict__ ev, int &n_ev, KBuf<K> &kb,
                                                   Counters &cnt, bool &lane_ok)
{
    const unsigned full = 0xffffffffu;
    const size_t S = (size_t)W.a.n_slots;
    const int lane = threadIdx.x & 31;
    const float Lt = tn;
    const uint32_t Li = GRTX_NONE;
    float tmax = kb.tmax;
    n_dst = 0;
    n_ev = 0;
    lane_ok = true;
    if (W.n_inst == 0) return;
    int sp = 0;
    uint32_t ref = 0u, parent = GRTX_NONE, slot = 0u, inst = GRTX_NONE, cur = GRTX_NONE;
    unsigned m = __ballot_sync(full, valid);
    float te = tn;
    bool have_te = true;
    float3 ob = o, db = d, ib = inv;
    const float4 *nodes = W.tl_nodes, *geom = nullptr;
    uint32_t base = 0;
    for (;;) {
        if (inst != cur) {                                  // another level: map each lane's ray
            cur = inst;
            if (inst == GRTX_NONE) {
                ob = o;
                db = d;
                ib = inv;
                nodes = W.tl_nodes;
            } else {
                const InstRec &I = W.inst[inst];
                to_object(I, o, d, ob, db);
                ib = make_float3(safe_rcp(db.x), safe_rcp(db.y), safe_rcp(db.z));
                nodes = I.sc.nodes;
                geom = I.sc.geom;
                base = I.leaf_base;
            }
        }
        bool in = (m >> lane) & 1u;
        if (!have_te && in) {                               // a popped node: entry from the parent's box
            const float4 *pn = nodes + 4 * (size_t)parent;
            float x;
            if (slot == 0u) {
                float4 n0 = __ldg(pn), n1 = __ldg(pn + 1);
                slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ob, ib, tn, tf, te, x);
            } else {
                float4 n1 = __ldg(pn + 1), n2 = __ldg(pn + 2);
                slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ob, ib, tn, tf, te, x);
            }
        }
        bool go = in && lane_ok && !(te > tmax);
        if (in && lane_ok && te > tmax && ckpt) {
            if (n_dst >= W.a.ckpt_cap) {
                lane_ok = false;
            } else {
                dst[(size_t)n_dst * S] = make_uint4(ref, __float_as_uint(te), inst, 0u);
                ++n_dst;
                if (INSTR) cnt.ckpt++;
            }
        }
        m = __ballot_sync(full, go);
        bool pop = true;
        if (m && (!INSTR || world_ref_ok(W, inst, ref, cnt, go))) {   // ref is the warp's
            if (ref & GRTX_LEAF) {
                if (inst == GRTX_NONE) {                    // TLAS leaf: descend into the object's root
                    inst = ref & ~GRTX_LEAF;
                    ref = 0u;
                    have_te = true;
                    continue;
                }
                if (go) {
                    uint32_t gi = ref & ~GRTX_LEAF;
                    if (INSTR) cnt.leaves++;
                    float t, D2, w[3];
                    uint32_t key = base + gi;
                    if (sphere_test(geom + 4 * (size_t)gi, ob, db, t, D2, w) && D2 <= 1.0f && t > tn && t <= tf &&
                        key_after(t, key, Lt, Li)) {
                        float ct = t;
                        uint32_t ci = key;
                        if (kb.insert(ct, ci) && ckpt) {
                            if (n_ev >= W.a.evict_cap) {
                                lane_ok = false;
                            } else {
                                ev[(size_t)n_ev * S] = make_uint2(__float_as_uint(ct), ci);
                                ++n_ev;
                                if (INSTR) cnt.evictions++;
                            }
                        }
                        tmax = kb.tmax;
                    }
                }
            } else {
                const float4 *nd = nodes + 4 * (size_t)ref;
                float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
                uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
                bool h0 = false, h1 = false, near0 = true;
                float e0 = 0.f, e1 = 0.f;
                if (go) {
                    if (INSTR) cnt.nodes++;
                    float x0, x1;
                    slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, ob, ib, tn, tf, e0, x0);
                    slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, ob, ib, tn, tf, e1, x1);
                    h0 = e0 <= x0 && !(x0 < Lt);
                    h1 = e1 <= x1 && !(x1 < Lt) && c1 != GRTX_NONE;
                    near0 = e0 <= e1;
                }
                unsigned m0 = __ballot_sync(full, h0), m1 = __ballot_sync(full, h1);
                if (m0 && m1) {
                    unsigned both = m0 & m1, vote = __ballot_sync(full, h0 && h1 && near0);
                    bool n0first = both ? (2 * __popc(vote) >= __popc(both)) : (__popc(m0) >= __popc(m1));
                    if (sp >= W.a.packet_stack) {             // too deep for the warp's stack
                        lane_ok = false;
                        return;
                    }
                    if (lane == 0)
                        pst[sp] = make_uint4(n0first ? c1 : c0, (ref << 1) | (n0first ? 1u : 0u), n0first ? m1 : m0, inst);
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
            inst = v.w;
            have_te = false;
        }
    }
}

// One ray through the world: the round loop of trace_ray with world_round and blending in
// the frame of each Gaussian's object.
template <int K, bool INSTR>
__device__ __forceinline__ void world_ray(const WorldArgs &W, int slot, int64_t pix, float3 o, float3 d, float tn,
                                          float tf, KBuf<K> &kb, Counters &cnt, bool r1_ok, int r1_n_dst, int r1_n_ev)
{
    const TraceArgs &a = W.a;
    const size_t S = (size_t)a.n_slots;
    float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    BlendState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f;
    float Lt = tn;
    uint32_t Li = GRTX_NONE;
    bool ckpt = a.traversal == GRTX_TRAVERSAL_CHECKPOINT;
    bool from_root = true;
    int n_src = 0, n_ev = 0, nb = 0;
    uint4 *src = W.wck0 + slot, *dst = W.wck1 + slot;
    uint2 *ev = a.ev + slot;
    bool done = W.n_inst == 0;
    bool first_round = true;
    while (!done) {
        if (INSTR) cnt.rounds++;
        if (!first_round) kb.clear();
        if (ckpt && n_ev > 0) {
            int w = 0;
            for (int e = 0; e < n_ev; ++e) {
                uint2 v = ev[(size_t)e * S];
                float ct = __uint_as_float(v.x);
                uint32_t ci = v.y;
                if (kb.insert(ct, ci)) {
                    ev[(size_t)w * S] = make_uint2(__float_as_uint(ct), ci);
                    ++w;
                }
            }
            n_ev = w;
        }
        int n_dst = 0;
        bool round_ok;
        if (first_round) {                             // round 1 was traced as the warp's packet
            round_ok = r1_ok;
            n_dst = r1_n_dst;
            n_ev = r1_n_ev;
        } else {
            round_ok = world_round<K, INSTR>(W, o, d, inv, tn, tf, Lt, Li, ckpt, from_root, src, n_src, dst, n_dst, ev,
                                             n_ev, kb, cnt);
        }
        if (!round_ok) {
            if (INSTR) cnt.fallbacks++;
            ckpt = false;
            from_root = true;
            n_src = 0;
            n_ev = 0;
            kb.clear();
            world_round<K, INSTR>(W, o, d, inv, tn, tf, Lt, Li, false, true, src, 0, dst, n_dst, ev, n_ev, kb, cnt);
        }
        for (int j = 0; j < kb.n; ++j) {
            uint32_t key = kb.I(j);
            const InstRec &I = W.inst[find_instance(W, key)];
            uint32_t gi = key - I.leaf_base;
            float3 oo, od;
            to_object(I, o, d, oo, od);
            blend_one<false>(a, I.sc, st, gi, oo, od);      // colour along the object-frame direction
            if (INSTR) {
                if (a.ids && nb < a.ids_cap) a.ids[(size_t)pix * a.ids_cap + nb] = I.id_base + I.sc.gid[gi];
                cnt.blended++;
            }
            ++nb;
            if (st.T < a.T_min) {
                done = true;
                break;
            }
        }
        first_round = false;
        if (done || kb.n < K) break;
        Lt = kb.T(K - 1);
        Li = kb.I(K - 1);
        if (ckpt) {
            uint4 *tmp = src;
            src = dst;
            dst = tmp;
            n_src = n_dst;
            from_root = false;
        }
    }
    a.rgbT[pix] = make_float4(st.C[0] + st.T * a.bg0, st.C[1] + st.T * a.bg1, st.C[2] + st.T * a.bg2, st.T);
    if (INSTR && a.n_blended) a.n_blended[pix] = nb;
}

template <int K, bool INSTR>
__global__ void __launch_bounds__(kBlock, trace_min_blocks(K, false)) k_trace_world(WorldArgs W)
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
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(W.a.queue, 32u);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= W.a.n_items) break;
        int64_t pix;
        float3 o, d;
        float tn, tf;
        bool valid = make_ray(W.a.cam, b + lane, pix, o, d, tn, tf);
        if (!valid) {
            o = make_float3(0.f, 0.f, 0.f);
            d = make_float3(0.f, 0.f, 1.f);
            tn = tf = 0.f;
        }
        // round 1 of the warp's rays as one packet (every lane takes part), later rounds per ray
        float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
        kb.clear();
        int n_dst = 0, n_ev = 0;
        bool lane_ok = true;
        world_packet_round<K, INSTR>(W, valid, s_pst[threadIdx.x >> 5], o, d, inv, tn, tf,
                                     W.a.traversal == GRTX_TRAVERSAL_CHECKPOINT, W.wck1 + slot, n_dst, W.a.ev + slot,
                                     n_ev, kb, cnt, lane_ok);
        if (valid) {
            ++rays;
            world_ray<K, INSTR>(W, slot, pix, o, d, tn, tf, kb, cnt, lane_ok, n_dst, n_ev);
        }
        __syncwarp();
    }
    if (INSTR && W.a.stats) {
        unsigned long long v[11] = {rays, cnt.nodes, cnt.leaves, cnt.blended, cnt.rounds, cnt.ckpt, cnt.evictions,
                                    cnt.fallbacks, cnt.overflow, 0ull, cnt.oob};
#pragma unroll
        for (int q = 0; q < 11; ++q) {
            unsigned long long x = v[q];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0 && x) atomicAdd((&W.a.stats->rays) + q, x);
        }
    }
}

template <int K>
int world_launch(const WorldArgs &W, bool instr, int blocks, cudaStream_t s)
{
    if (instr) k_trace_world<K, true><<<blocks, kBlock, 0, s>>>(W);
    else k_trace_world<K, false><<<blocks, kBlock, 0, s>>>(W);
    return cudaGetLastError() == cudaSuccess ? GRTX_OK : GRTX_ERR_CUDA;
}

template <int K>
int world_occupancy(bool instr, int *bps)
{
    cudaError_t e = instr ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_trace_world<K, true>, kBlock, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_trace_world<K, false>, kBlock, 0);
    return e == cudaSuccess ? GRTX_OK : GRTX_ERR_CUDA;
}

}  // namespace

struct grtx_world {
    float alpha_min = 0.f;
    int n_inst = 0;            // non-empty instances (rows of the table and TLAS leaves)
    int n_tl_nodes = 0;
    int tl_depth = 0;
    float4 *tl_nodes = nullptr;
    InstRec *inst = nullptr;
    uint32_t *leaf_base = nullptr;
    cudaStream_t stream = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    unsigned *counter = nullptr;
};

namespace {

void world_free_tables(grtx_world *w)
{
    if (w->stream) cudaStreamSynchronize(w->stream);
    cudaFree(w->tl_nodes);
    cudaFree(w->inst);
    cudaFree(w->leaf_base);
    w->tl_nodes = nullptr;
    w->inst = nullptr;
    w->leaf_base = nullptr;
    w->n_inst = 0;
    w->n_tl_nodes = 0;
}

int world_set(grtx_world *w, const grtx_instance *inst, int n, cudaStream_t s)
{
    if (!inst || n < 1) return grtx_fail(GRTX_ERR_INVALID_ARG, "need at least one instance");
    std::vector<InstRec> rows;
    std::vector<host_bvh::Box> boxes;
    std::vector<uint32_t> bases;
    uint64_t leaves = 0, ids = 0;
    float alpha_min = 0.f;
    for (int i = 0; i < n; ++i) {
        const grtx_scene *sc = inst[i].scene;
        if (!sc) return grtx_fail(GRTX_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": scene is NULL");
        if (sc->form != GRTX_FORM_SPHERE)
            return grtx_fail(GRTX_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": worlds take sphere-form scenes");
        if (i == 0) alpha_min = sc->alpha_min;
        else if (sc->alpha_min != alpha_min) return grtx_fail(GRTX_ERR_INVALID_ARG, "scenes differ in alpha_min");
        const float *m = inst[i].object_to_world;
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(m[k])) return grtx_fail(GRTX_ERR_INVALID_ARG, "non-finite object_to_world");
        double L[9] = {m[0], m[1], m[2], m[4], m[5], m[6], m[8], m[9], m[10]}, c[3] = {m[3], m[7], m[11]};
        double c00 = L[4] * L[8] - L[5] * L[7], c01 = L[5] * L[6] - L[3] * L[8], c02 = L[3] * L[7] - L[4] * L[6];
        double det = L[0] * c00 + L[1] * c01 + L[2] * c02;
        double scale = 0;
        for (double x : L) scale = std::max(scale, std::fabs(x));
        if (!(std::fabs(det) > 1e-12 * scale * scale * scale))
            return grtx_fail(GRTX_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": object_to_world is not invertible");
        double Li[9] = {c00 / det, (L[2] * L[7] - L[1] * L[8]) / det, (L[1] * L[5] - L[2] * L[4]) / det,
                        c01 / det, (L[0] * L[8] - L[2] * L[6]) / det, (L[2] * L[3] - L[0] * L[5]) / det,
                        c02 / det, (L[1] * L[6] - L[0] * L[7]) / det, (L[0] * L[4] - L[1] * L[3]) / det};
        uint64_t id_base = ids;
        ids += (uint64_t)sc->n;
        if (sc->n_valid == 0) continue;                 // nothing to hit: not in the TLAS
        InstRec r = {};
        for (int a = 0; a < 3; ++a) {
            double off = -(Li[3 * a] * c[0] + Li[3 * a + 1] * c[1] + Li[3 * a + 2] * c[2]);
            r.w2o[a] = make_float4((float)Li[3 * a], (float)Li[3 * a + 1], (float)Li[3 * a + 2], (float)off);
        }
        r.sc = grtx_scene_ref(sc);
        r.leaf_base = (uint32_t)leaves;
        r.id_base = (uint32_t)id_base;
        leaves += (uint64_t)sc->n_leaves;
        // world box: the object's bounds through the map, widened against FP32 rounding
        host_bvh::Box b = host_bvh::empty_box();
        for (int corner = 0; corner < 8; ++corner) {
            double x[3] = {sc->bounds[(corner & 1) ? 3 : 0], sc->bounds[(corner & 2) ? 4 : 1],
                           sc->bounds[(corner & 4) ? 5 : 2]};
            for (int a = 0; a < 3; ++a) {
                double y = L[3 * a] * x[0] + L[3 * a + 1] * x[1] + L[3 * a + 2] * x[2] + c[a];
                b[a] = std::min(b[a], (float)y);
                b[3 + a] = std::max(b[3 + a], (float)y);
            }
        }
        for (int a = 0; a < 3; ++a) {
            float pad = 1e-5f * (b[3 + a] - b[a]) + 1e-6f * std::max(std::fabs(b[a]), std::fabs(b[3 + a])) + 1e-30f;
            b[a] -= pad;
            b[3 + a] += pad;
        }
        rows.push_back(r);
        boxes.push_back(b);
        bases.push_back(r.leaf_base);
    }
    if (leaves >= 0xFFFFFFFFull || ids > 0xFFFFFFFFull)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "more than 2^32 - 2 leaves or Gaussians in the world");
    int depth = 0;
    std::vector<host_bvh::Node> nodes;
    if (!rows.empty()) {
        nodes = host_bvh::build(boxes, &depth);
        if (depth > kMaxTlasDepth) return grtx_fail(GRTX_ERR_INVALID_ARG, "scene-level BVH deeper than 32");
    }
    world_free_tables(w);               // waits for earlier traces of this world
    w->alpha_min = alpha_min;
    w->stream = s;
    w->tl_depth = depth;
    if (rows.empty()) return GRTX_OK;
    // the world stays empty (n_inst = 0) unless every table reaches the device
    cudaError_t e = cudaMalloc(&w->tl_nodes, nodes.size() * sizeof(host_bvh::Node));
    if (e == cudaSuccess) e = cudaMalloc(&w->inst, rows.size() * sizeof(InstRec));
    if (e == cudaSuccess) e = cudaMalloc(&w->leaf_base, bases.size() * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(w->tl_nodes, nodes.data(), nodes.size() * sizeof(host_bvh::Node), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->inst, rows.data(), rows.size() * sizeof(InstRec), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(w->leaf_base, bases.data(), bases.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        world_free_tables(w);
        return grtx_cuda_fail(e, "world table upload");
    }
    w->n_inst = (int)rows.size();
    w->n_tl_nodes = (int)nodes.size();
    return GRTX_OK;
}

int sm_count_here()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

extern "C" GRTX_API int grtx_world_create(const grtx_instance *inst, int n, void *stream, grtx_world **out)
{
    if (!out) return grtx_fail(GRTX_ERR_INVALID_ARG, "out is NULL");
    grtx_world *w = new (std::nothrow) grtx_world();
    if (!w) return grtx_fail(GRTX_ERR_OOM, "host allocation failed");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int st = world_set(w, inst, n, s);
    if (st == GRTX_OK) {
        cudaError_t e = cudaMalloc(&w->counter, sizeof(unsigned));
        if (e != cudaSuccess) st = grtx_cuda_fail(e, "cudaMalloc(world counter)");
    }
    if (st != GRTX_OK) {
        world_free_tables(w);
        cudaFree(w->counter);
        delete w;
        return st;
    }
    *out = w;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_world_update(grtx_world *w, const grtx_instance *inst, int n, void *stream)
{
    if (!w) return grtx_fail(GRTX_ERR_INVALID_ARG, "world is NULL");
    return world_set(w, inst, n, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" GRTX_API int grtx_world_trace_forward(grtx_world *w, const grtx_camera *cam, const grtx_params *p,
                                                 const grtx_trace_outputs *out, void *stream)
{
    if (!w) return grtx_fail(GRTX_ERR_INVALID_ARG, "world is NULL");
    int st = grtx_check_params(p);
    if (st) return st;
    if (p->k != 8 && p->k != 16 && p->k != 32) return grtx_fail(GRTX_ERR_INVALID_ARG, "worlds trace with k = 8, 16 or 32");
    if (p->traversal != GRTX_TRAVERSAL_CHECKPOINT && p->traversal != GRTX_TRAVERSAL_RESTART)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "worlds trace with checkpoint or restart traversal");
    if (p->alpha_min != w->alpha_min) return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_min differs from the scenes'");
    if (!out || !out->rgbT || ((uintptr_t)out->rgbT & 15))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "rgbT must be a 16-byte aligned device pointer");
    if (out->blended_ids && out->ids_cap <= 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "ids_cap must be positive");
    if (out->saved) return grtx_fail(GRTX_ERR_INVALID_ARG, "saved blend lists are not available for worlds");
    if (out->visits || out->visits_n)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "visit logs are not available for worlds (node indices of the levels collide)");
    WorldArgs W = {};
    TraceArgs &a = W.a;
    st = grtx_fill_camera(a.cam, a.n_items, cam);
    if (st) return st;
    a.traversal = p->traversal;
    a.T_min = p->T_min;
    a.alpha_max = p->alpha_max;
    a.bg0 = p->bg[0];
    a.bg1 = p->bg[1];
    a.bg2 = p->bg[2];
    a.ckpt_cap = p->ckpt_capacity > 0 ? p->ckpt_capacity : GRTX_DEFAULT_CKPT_CAPACITY;
    a.evict_cap = p->evict_capacity > 0 ? p->evict_capacity : GRTX_DEFAULT_EVICT_CAPACITY;
    a.packet_stack = p->packet_stack > 0 ? std::min(p->packet_stack, kPacketStack) : kPacketStack;
    a.rgbT = (float4 *)out->rgbT;
    a.n_blended = out->n_blended;
    a.ids = out->blended_ids;
    a.ids_cap = out->ids_cap;
    a.stats = out->stats;
    bool instr = out->n_blended || out->blended_ids || out->stats;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (out->blended_ids)
        GRTX_CUDA(cudaMemsetAsync(out->blended_ids, 0xff, (size_t)cam->width * cam->height * out->ids_cap * 4, s));
    int bps = 0;
    int occ = p->k == 8 ? world_occupancy<8>(instr, &bps)
              : p->k == 16 ? world_occupancy<16>(instr, &bps) : world_occupancy<32>(instr, &bps);
    if (occ != GRTX_OK || bps <= 0) return grtx_fail(GRTX_ERR_CUDA, "occupancy query failed");
    int blocks = sm_count_here() * bps;
    size_t n_slots = (size_t)blocks * kBlock;
    bool ckpt = a.traversal == GRTX_TRAVERSAL_CHECKPOINT;
    size_t C = ckpt ? (size_t)a.ckpt_cap : 1, E = ckpt ? (size_t)a.evict_cap : 1;
    size_t need = n_slots * (2 * C * sizeof(uint4) + E * sizeof(uint2));
    if (need > w->ws_bytes) {
        if (w->ws) {
            GRTX_CUDA(cudaDeviceSynchronize());          // earlier traces on any stream may use it
            GRTX_CUDA(cudaFreeAsync(w->ws, s));
            w->ws = nullptr;
            w->ws_bytes = 0;
        }
        st = grtx_malloc_async(&w->ws, need, s);
        if (st) return st;
        w->ws_bytes = need;
    }
    W.wck0 = (uint4 *)w->ws;
    W.wck1 = W.wck0 + n_slots * C;
    a.ev = (uint2 *)(W.wck1 + n_slots * C);
    a.n_slots = (int)n_slots;
    a.queue = w->counter;
    W.tl_nodes = w->tl_nodes;
    W.inst = w->inst;
    W.leaf_base = w->leaf_base;
    W.n_inst = w->n_inst;
    W.n_tl_nodes = w->n_tl_nodes;
    w->stream = s;
    GRTX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), s));
    int launched = p->k == 8 ? world_launch<8>(W, instr, blocks, s)
                   : p->k == 16 ? world_launch<16>(W, instr, blocks, s) : world_launch<32>(W, instr, blocks, s);
    if (launched != GRTX_OK) {
        cudaError_t e = cudaGetLastError();
        return grtx_cuda_fail(e == cudaSuccess ? cudaErrorLaunchFailure : e, "world trace launch");
    }
    return GRTX_OK;
}

extern "C" GRTX_API void grtx_world_destroy(grtx_world *w)
{
    if (!w) return;
    world_free_tables(w);
    if (w->ws) cudaFreeAsync(w->ws, w->stream);
    if (w->stream) cudaStreamSynchronize(w->stream);
    else cudaDeviceSynchronize();
    cudaFree(w->counter);
    delete w;
}
