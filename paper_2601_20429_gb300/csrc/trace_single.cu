// Single-round traversal: the baseline of Sec. III-C (Observation II) that collects every
// intersected Gaussian in one traversal, then sorts and blends after it, instead of k-buffer
// rounds with early termination between them.
//
// Per ray: one traversal of the whole BVH over (t_near, t_far] (as the warp's packet, like
// round 1 of the k-buffer kernels) appends every hit key (t, leaf index) to the ray slot's list
// in the trace workspace (capacity ckpt_capacity, interleaved [entry][slot] like the
// checkpoint lists). The list is then made a binary
// min-heap and popped in key order while blending front to back, stopping right after the
// Gaussian that takes T below T_min: the sort stops where termination does, so its cost is
// O(n + b log n) for n hits and b blended. A ray with more hits than the capacity is traced
// again with k-buffer rounds restarted from the root (k = 16), which gives the same result.
#include "trace_impl.cuh"

namespace {

constexpr int kFallbackK = 16;

// Orderable 64-bit key of (t, leaf index): float bits mapped so that unsigned order is
// numeric order for either sign, then the index.
__device__ __forceinline__ uint64_t single_key(uint2 v)
{
    uint32_t b = v.x;
    b ^= (b & 0x80000000u) ? 0xffffffffu : 0x80000000u;
    return ((uint64_t)b << 32) | v.y;
}

__device__ __forceinline__ void heap_sift_down(uint2 *__restrict__ h, size_t S, int i, int n)
{
    uint2 v = h[(size_t)i * S];
    uint64_t kv = single_key(v);
    for (;;) {
        int c = 2 * i + 1;
        if (c >= n) break;
        uint2 cv = h[(size_t)c * S];
        uint64_t kc = single_key(cv);
        if (c + 1 < n) {
            uint2 rv = h[(size_t)(c + 1) * S];
            uint64_t kr = single_key(rv);
            if (kr < kc) {
                ++c;
                cv = rv;
                kc = kr;
            }
        }
        if (kv <= kc) break;
        h[(size_t)i * S] = cv;
        i = c;
    }
    h[(size_t)i * S] = v;
}

// Every hit of the warp's rays, collected as one packet: the warp walks the union of the nodes
// its rays need (one broadcast load per node, see packet_round), each lane appending its own
// hits to its list (stride S).
// Every lane calls this together; lanes without a ray pass valid = false. Returns each lane's
// count, or -1 for a lane whose list overflowed or, for every lane, when the warp's stack would.
template <int FORM, bool INSTR>
__device__ __forceinline__ int packet_collect(const TraceArgs &a, const SceneRef &sc, bool valid, uint4 *pst, float3 o,
                                              float3 d, float3 inv, float tn, float tf, uint2 *__restrict__ list,
                                              Counters &cnt, unsigned &collected)
{
    const unsigned full = 0xffffffffu;
    const size_t S = (size_t)a.n_slots;
    const int lane = threadIdx.x & 31;
    int n = 0;
    bool ok = true;
    if (!sc.has_tree) return 0;
    int sp = 0;
    uint32_t ref = 0u;
    unsigned m = __ballot_sync(full, valid);
    for (;;) {
        bool go = ((m >> lane) & 1u) && ok;
        if (__ballot_sync(full, go) && (!INSTR || ref_ok(sc, ref, cnt, go))) {   // ref is the warp's
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
                        t <= tf) {
                        if (n >= a.ckpt_cap) {
                            ok = false;
                        } else {
                            list[(size_t)n * S] = make_uint2(__float_as_uint(t), gi);
                            ++n;
                            if (INSTR) collected++;
                        }
                    }
                }
            } else {
                const float4 *nd = sc.nodes + 4 * (size_t)ref;
                float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
                uint32_t c0 = __float_as_uint(n3.x), c1 = __float_as_uint(n3.y);
                bool h0 = false, h1 = false, near0 = true;
                if (go) {
                    if (INSTR) {
                        cnt.nodes++;
                        log_visit(cnt, ref);
                    }
                    float e0, x0, e1, x1;
                    slab(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, o, inv, tn, tf, e0, x0);
                    slab(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, o, inv, tn, tf, e1, x1);
                    h0 = e0 <= x0;
                    h1 = e1 <= x1 && c1 != GRTX_NONE;
                    near0 = e0 <= e1;
                }
                unsigned m0 = __ballot_sync(full, h0), m1 = __ballot_sync(full, h1);
                if (m0 && m1) {
                    unsigned both = m0 & m1, vote = __ballot_sync(full, h0 && h1 && near0);
                    bool n0first = both ? (2 * __popc(vote) >= __popc(both)) : (__popc(m0) >= __popc(m1));
                    if (sp >= a.packet_stack) return -1;        // too deep for the warp's stack
                    if (lane == 0) pst[sp] = make_uint4(n0first ? c1 : c0, 0u, n0first ? m1 : m0, 0u);
                    ++sp;
                    __syncwarp(full);
                    m = n0first ? m0 : m1;
                    ref = n0first ? c0 : c1;
                    continue;
                }
                if (m0 || m1) {
                    m = m0 ? m0 : m1;
                    ref = m0 ? c0 : c1;
                    continue;
                }
            }
        }
        if (sp == 0) break;
        --sp;
        uint4 v = pst[sp];
        ref = v.x;
        m = v.z;
    }
    return ok ? n : -1;
}

template <int FORM, bool INSTR>
__device__ __forceinline__ void single_ray(const TraceArgs &a, const SceneRef &sc, int slot, bool valid, int64_t pix,
                                           float3 o, float3 d, float tn, float tf, KBuf<kFallbackK> &kb, Counters &cnt,
                                           unsigned &collected, uint4 *pst)
{
    const size_t S = (size_t)a.n_slots;
    if (!valid) {
        o = make_float3(0.f, 0.f, 0.f);
        d = make_float3(0.f, 0.f, 1.f);
        tn = tf = 0.f;
    }
    float3 inv = make_float3(safe_rcp(d.x), safe_rcp(d.y), safe_rcp(d.z));
    uint2 *list = a.ck0 + slot;
    int n = packet_collect<FORM, INSTR>(a, sc, valid, pst, o, d, inv, tn, tf, list, cnt, collected);
    if (!valid) return;
    if (sc.has_tree) {
        if (INSTR) cnt.rounds++;
        if (n < 0) {                  // more hits than the list holds: k-buffer rounds instead
            if (INSTR) cnt.fallbacks++;
            trace_ray<kFallbackK, FORM, INSTR, false>(a, sc, a.rgbT, slot, pix, o, d, tn, tf, kb, cnt);
            return;
        }
    }
    BlendState st;
    st.C[0] = st.C[1] = st.C[2] = 0.f;
    st.T = 1.f;
    for (int i = n / 2 - 1; i >= 0; --i) heap_sift_down(list, S, i, n);
    uint64_t prev = ~0ull;
    int nb = 0;
    while (n > 0) {
        uint2 top = list[0];
        --n;
        if (n > 0) {
            list[0] = list[(size_t)n * S];
            heap_sift_down(list, S, 0, n);
        }
        uint64_t key = single_key(top);
        if (FORM == FORM_PROXY && key == prev) continue;   // one Gaussian found through several triangles
        prev = key;
        uint32_t idx = top.y;
        blend_one<false>(a, sc, st, idx, o, d);
        if (INSTR) {
            if (a.ids && nb < a.ids_cap) a.ids[(size_t)pix * a.ids_cap + nb] = sc.gid[idx];
            cnt.blended++;
        }
        ++nb;
        if (st.T < a.T_min) break;
    }
    a.rgbT[pix] = make_float4(st.C[0] + st.T * a.bg0, st.C[1] + st.T * a.bg1, st.C[2] + st.T * a.bg2, st.T);
    if (INSTR && a.n_blended) a.n_blended[pix] = nb;
}

template <int FORM, bool INSTR>
__global__ void __launch_bounds__(kBlock, 8) k_trace_single(TraceArgs a)
{
    __shared__ float s_kt[kFallbackK * kBlock];
    __shared__ uint32_t s_ki[kFallbackK * kBlock];
    __shared__ uint4 s_pst[kBlock / 32][kPacketStack];
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    KBuf<kFallbackK> kb;
    kb.t = s_kt + threadIdx.x;
    kb.id = s_ki + threadIdx.x;
    Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0, nullptr, 0, 0};
    unsigned rays = 0, collected = 0;
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
        single_ray<FORM, INSTR>(a, a.sc, slot, valid, pix, o, d, tn, tf, kb, cnt, collected, s_pst[threadIdx.x >> 5]);
        if (INSTR) visits_end(a, cnt, pix);
        __syncwarp();
    }
    if (INSTR && a.stats) {
        unsigned long long v[11] = {rays, cnt.nodes, cnt.leaves, cnt.blended, cnt.rounds, cnt.ckpt, cnt.evictions,
                                    cnt.fallbacks, cnt.overflow, collected, cnt.oob};
#pragma unroll
        for (int q = 0; q < 11; ++q) {
            unsigned long long x = v[q];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0 && x) atomicAdd((&a.stats->rays) + q, x);
        }
    }
}

}  // namespace

int trace_single_launch(const TraceArgs &a, int form, bool instr, int blocks, cudaStream_t s)
{
    dim3 g(blocks), b(kBlock);
    if (form == FORM_PROXY && instr) k_trace_single<FORM_PROXY, true><<<g, b, 0, s>>>(a);
    else if (form == FORM_PROXY) k_trace_single<FORM_PROXY, false><<<g, b, 0, s>>>(a);
    else if (form == FORM_ICO && instr) k_trace_single<FORM_ICO, true><<<g, b, 0, s>>>(a);
    else if (form == FORM_ICO) k_trace_single<FORM_ICO, false><<<g, b, 0, s>>>(a);
    else if (instr) k_trace_single<FORM_SPHERE, true><<<g, b, 0, s>>>(a);
    else k_trace_single<FORM_SPHERE, false><<<g, b, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GRTX_OK : GRTX_ERR_CUDA;
}

template <int FORM, bool INSTR>
static int single_occ(int *bps)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_trace_single<FORM, INSTR>, kBlock, 0) == cudaSuccess
               ? GRTX_OK : GRTX_ERR_CUDA;
}

int trace_single_occupancy(int form, bool instr, int *blocks_per_sm)
{
    if (form == FORM_PROXY) return instr ? single_occ<FORM_PROXY, true>(blocks_per_sm) : single_occ<FORM_PROXY, false>(blocks_per_sm);
    if (form == FORM_ICO) return instr ? single_occ<FORM_ICO, true>(blocks_per_sm) : single_occ<FORM_ICO, false>(blocks_per_sm);
    return instr ? single_occ<FORM_SPHERE, true>(blocks_per_sm) : single_occ<FORM_SPHERE, false>(blocks_per_sm);
}
