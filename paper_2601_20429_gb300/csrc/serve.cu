// Serving: several resident scenes and a stream of camera requests. Requests are admitted
// into a bounded set of slots as earlier ones finish (continuous batching), and, under a
// memory budget, only while their outputs fit the server's output arena; each step is one
// persistent launch whose queue concatenates pieces of every admitted request (mixed scenes
// and resolutions), so rays of new and old requests share the device. Up to four steps are
// in flight, each on its own stream: the host prepares and enqueues the next while the
// others run.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "trace_impl.cuh"

#define GRTX_EXTERN_SERVE(K)                                                                                 \
    extern template int serve_launch<K>(const TraceArgs &, const ServeSeg *, int, int, cudaStream_t, unsigned *,  \
                                        unsigned *, unsigned);                                                    \
    extern template int serve_occupancy<K>(int *);
GRTX_EXTERN_SERVE(1)
GRTX_EXTERN_SERVE(2)
GRTX_EXTERN_SERVE(4)
GRTX_EXTERN_SERVE(8)
GRTX_EXTERN_SERVE(16)
GRTX_EXTERN_SERVE(32)

int grtx_fill_camera(CamRef &a, unsigned &n_items_out, const grtx_camera *cam);
SceneRef grtx_scene_ref(const grtx_scene *sc);
int grtx_check_params(const grtx_params *p);

namespace {

constexpr int kMaxPending = 65536;
constexpr int kSteps = 4;         // step slots (streams) in flight
constexpr int kQueueStride = 32;   // the slots' queue counters on separate 128-byte lines

double now_s()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int serve_launch_k(int k, const TraceArgs &a, const ServeSeg *segs, int n, int blocks, cudaStream_t s,
                   unsigned *seg_done, unsigned *seg_flag, unsigned seq)
{
    switch (k) {
    case 1: return serve_launch<1>(a, segs, n, blocks, s, seg_done, seg_flag, seq);
    case 2: return serve_launch<2>(a, segs, n, blocks, s, seg_done, seg_flag, seq);
    case 4: return serve_launch<4>(a, segs, n, blocks, s, seg_done, seg_flag, seq);
    case 8: return serve_launch<8>(a, segs, n, blocks, s, seg_done, seg_flag, seq);
    case 16: return serve_launch<16>(a, segs, n, blocks, s, seg_done, seg_flag, seq);
    default: return serve_launch<32>(a, segs, n, blocks, s, seg_done, seg_flag, seq);
    }
}

int serve_occupancy_k(int k, int *bps)
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

struct SrvReq {
    grtx_request r;
    CamRef cam;
    unsigned n_items = 0;      // queue items of the whole request (32 per warp tile)
    unsigned next = 0;         // first item not yet scheduled
    double t_admit = 0;
    size_t out_bytes = 0;      // > 0: the server allocates the output from its arena at admission
    int pending_segs = 0;      // segments scheduled in steps and not yet complete
};

// First-fit allocator over the output arena (offsets on the host, 256-byte granules).
struct Arena {
    char *base = nullptr;
    size_t bytes = 0, used = 0;
    std::map<size_t, size_t> free_;     // offset -> size, coalesced
    std::map<size_t, size_t> live;      // offset -> size of outputs handed out
    void reset(char *b, size_t n)
    {
        base = b;
        bytes = n;
        used = 0;
        free_.clear();
        live.clear();
        if (n) free_[0] = n;
    }
    static size_t round(size_t n) { return (n + 255) / 256 * 256; }
    char *alloc(size_t n)
    {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > n) free_[off + n] = sz - n;
            live[off] = n;
            used += n;
            return base + off;
        }
        return nullptr;
    }
    bool release(char *p)
    {
        if (!base || p < base || p >= base + bytes) return false;
        auto it = live.find((size_t)(p - base));
        if (it == live.end()) return false;
        size_t off = it->first, n = it->second;
        live.erase(it);
        used -= n;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {      // merge with the next free block
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                              // and with the previous one
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += n;
                return true;
            }
        }
        free_[off] = n;
        return true;
    }
};

// A step slot: each has its own stream, per-slot lists and queue counter, so that the next
// step's blocks take the SMs the previous step's blocks leave while its slowest warps finish.
// Completion is per segment: the warp that finishes a segment's last tile raises the
// segment's flag in pinned host memory, so a request is reported as soon as its own tiles are
// done, not when the whole step ends.
struct SrvStep {
    cudaEvent_t ev = nullptr;
    cudaStream_t s = nullptr;  // slot 0: the server's stream; the others: created by the server
    bool own_stream = false;
    void *ws = nullptr;        // checkpoint and eviction lists of this slot's launches
    ServeSeg *h = nullptr;     // pinned host copy of the segment table
    ServeSeg *d = nullptr;     // device segment table
    unsigned *d_done = nullptr;     // device: items finished per segment
    unsigned *h_flag = nullptr;     // pinned, mapped: the step's sequence number once a segment is done
    unsigned *d_flag = nullptr;     // device address of h_flag
    unsigned seq = 0;               // this launch's sequence number
    std::vector<SrvReq *> seg_req;  // request of each segment
    std::vector<char> seg_seen;     // segment completion already taken into account
    bool busy = false;
};

}  // namespace

struct grtx_server {
    std::vector<grtx_scene *> scenes;
    grtx_params p;
    int64_t max_rays = 0;
    int max_inflight = 0;
    int64_t budget = 0;         // device bytes the server may hold (0: no cap)
    cudaStream_t s = nullptr;
    std::deque<SrvReq *> pending;
    std::deque<SrvReq *> active;
    SrvStep steps[kSteps];
    int n_steps = kSteps;       // step slots in use (fewer under a small budget)
    std::deque<int> inflight;
    std::deque<grtx_completion> backlog;
    TraceArgs a;
    int blocks = 0;
    size_t list_bytes = 0;      // lists of all step slots
    size_t device_bytes = 0;    // everything the server allocated on the device
    unsigned *queue = nullptr;  // one ray-queue counter per step slot
    Arena arena;                // server-owned outputs (budget > 0)
    unsigned seq = 0;           // launches so far (segment flags carry their launch's number)
};

namespace {

void server_free(grtx_server *v)
{
    for (auto &st : v->steps)
        if (st.ev) cudaStreamSynchronize(st.s);     // (unused slots have no event)
    for (auto &st : v->steps) {
        if (st.ev) cudaEventDestroy(st.ev);
        if (st.h) cudaFreeHost(st.h);
        if (st.d) cudaFree(st.d);
        if (st.d_done) cudaFree(st.d_done);
        if (st.h_flag) cudaFreeHost(st.h_flag);
        if (st.ws) cudaFree(st.ws);
        if (st.own_stream) cudaStreamDestroy(st.s);
    }
    if (v->queue) cudaFree(v->queue);
    if (v->arena.base) cudaFree(v->arena.base);
    for (auto *r : v->pending) delete r;
    for (auto *r : v->active) delete r;
    delete v;
}

// Enqueue one step over the admitted requests' unscheduled items: requests are taken in
// admission order up to max_rays, and the step's queue hands out the smaller pieces first, so
// that small requests, reported per segment, finish early in the step.
int schedule_step(grtx_server *v, int si)
{
    SrvStep &st = v->steps[si];
    st.seg_req.clear();
    st.seg_seen.clear();
    int64_t budget = std::max<int64_t>(32, v->max_rays / 32 * 32);
    struct Piece {
        SrvReq *r;
        unsigned begin, count;
    };
    std::vector<Piece> pieces;
    for (SrvReq *r : v->active) {
        if (r->next >= r->n_items) continue;
        if (budget <= 0) break;
        unsigned take = (unsigned)std::min<int64_t>((int64_t)(r->n_items - r->next), budget);
        pieces.push_back({r, r->next, take});
        r->next += take;
        budget -= take;
    }
    std::stable_sort(pieces.begin(), pieces.end(), [](const Piece &x, const Piece &y) { return x.count < y.count; });
    unsigned total = 0;
    int n = 0;
    for (const Piece &pc : pieces) {
        ServeSeg &g = st.h[n];
        g.sc = grtx_scene_ref(v->scenes[pc.r->r.scene_id]);
        g.cam = pc.r->cam;
        g.out = (float4 *)pc.r->r.d_rgbT;
        g.item_begin = pc.begin;
        g.step_begin = total;
        g.count = pc.count;
        g.pad = 0;
        total += pc.count;
        st.seg_req.push_back(pc.r);
        st.seg_seen.push_back(0);
        pc.r->pending_segs++;
        ++n;
    }
    if (n == 0) return GRTX_OK;
    TraceArgs a = v->a;
    const size_t S = (size_t)a.n_slots;
    a.ck0 = (uint2 *)st.ws;
    a.ck1 = a.ck0 + S * a.ckpt_cap;
    a.ev = a.ck0 + S * 2 * a.ckpt_cap;
    a.queue = v->queue + kQueueStride * si;
    a.n_items = total;
    set_list_offsets(a, 2 * (size_t)a.ckpt_cap + (size_t)a.evict_cap);   // size checked at creation
    a.discard = lists_discardable(a);
    GRTX_CUDA(cudaMemcpyAsync(st.d, st.h, sizeof(ServeSeg) * n, cudaMemcpyHostToDevice, st.s));
    GRTX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), st.s));
    GRTX_CUDA(cudaMemsetAsync(st.d_done, 0, sizeof(unsigned) * n, st.s));
    st.seq = ++v->seq;
    if (serve_launch_k(v->p.k, a, st.d, n, v->blocks, st.s, st.d_done, st.d_flag, st.seq) != GRTX_OK) {
        cudaError_t e = cudaGetLastError();
        return grtx_cuda_fail(e == cudaSuccess ? cudaErrorLaunchFailure : e, "serve step launch");
    }
    GRTX_CUDA(cudaEventRecord(st.ev, st.s));
    st.busy = true;
    v->inflight.push_back(si);
    return GRTX_OK;
}

bool has_unscheduled(const grtx_server *v)
{
    for (const SrvReq *r : v->active)
        if (r->next < r->n_items) return true;
    return false;
}

}  // namespace

extern "C" GRTX_API int grtx_server_create(grtx_scene *const *scenes, int n_scenes, const grtx_params *p,
                                           int64_t mem_budget_bytes, int64_t max_rays_per_step, int max_inflight,
                                           void *stream, grtx_server **out)
{
    if (!scenes || n_scenes <= 0 || !out) return grtx_fail(GRTX_ERR_INVALID_ARG, "need scenes and out");
    int st = grtx_check_params(p);
    if (st) return st;
    if (p->traversal == GRTX_TRAVERSAL_SINGLE)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "serving supports checkpoint and restart traversal");
    for (int i = 0; i < n_scenes; ++i) {
        if (!scenes[i]) return grtx_fail(GRTX_ERR_INVALID_ARG, "scene is NULL");
        if (scenes[i]->form != GRTX_FORM_SPHERE) return grtx_fail(GRTX_ERR_INVALID_ARG, "serving needs sphere-form scenes");
        if (scenes[i]->alpha_min != p->alpha_min) return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_min mismatch");
    }
    if (max_rays_per_step < 0 || max_inflight < 0 || max_inflight > 4096 || mem_budget_bytes < 0)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "bad server limits");
    const int64_t max_rays = max_rays_per_step > 0 ? max_rays_per_step : (int64_t)4 << 20;
    const int inflight_cap = max_inflight > 0 ? max_inflight : 64;
    const size_t C = p->ckpt_capacity > 0 ? p->ckpt_capacity : GRTX_DEFAULT_CKPT_CAPACITY;
    const size_t E = p->evict_capacity > 0 ? p->evict_capacity : GRTX_DEFAULT_EVICT_CAPACITY;
    int bps = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (serve_occupancy_k(p->k, &bps) != GRTX_OK || bps <= 0 || sms <= 0)
        return grtx_fail(GRTX_ERR_CUDA, "occupancy query failed");
    // sizes: the lists of n_steps step slots of `blocks` 128-ray blocks each, the segment
    // tables and queue counters, and (under a budget) the output arena
    const size_t per_block = 128 * (2 * C + E) * sizeof(uint2);
    const int blocks_full = sms * bps;
    if ((size_t)blocks_full * 128 * (2 * C + E) >= ((size_t)1 << 31))
        return grtx_fail(GRTX_ERR_INVALID_ARG, "checkpoint/eviction capacities too large for the resident ray slots");
    const size_t tables = kSteps * kQueueStride * sizeof(unsigned) +
                          (size_t)kSteps * (sizeof(ServeSeg) + sizeof(unsigned)) * inflight_cap;
    int n_steps = kSteps, blocks = blocks_full;
    size_t arena = 0;
    if (mem_budget_bytes > 0) {
        const size_t budget = (size_t)mem_budget_bytes;
        const size_t list_cap = budget / 2;
        const size_t full_step = (size_t)blocks_full * per_block;
        n_steps = (int)std::min<size_t>(kSteps, std::max<size_t>(1, list_cap / full_step));
        blocks = (int)std::min<size_t>((size_t)blocks_full, list_cap / ((size_t)n_steps * per_block));
        if (blocks < 1)
            return grtx_fail(GRTX_ERR_INVALID_ARG, "memory budget of " + std::to_string(budget) +
                                                       " bytes is below twice one block of lists (" +
                                                       std::to_string(per_block) + " bytes)");
        size_t lists = (size_t)n_steps * blocks * per_block;
        if (lists + tables > budget) return grtx_fail(GRTX_ERR_INVALID_ARG, "memory budget too small");
        arena = (budget - lists - tables) / 256 * 256;
    }
    grtx_server *v = new (std::nothrow) grtx_server();
    if (!v) return grtx_fail(GRTX_ERR_OOM, "host allocation failed");
    v->scenes.assign(scenes, scenes + n_scenes);
    v->p = *p;
    v->max_rays = max_rays;
    v->max_inflight = inflight_cap;
    v->budget = mem_budget_bytes;
    v->n_steps = n_steps;
    v->blocks = blocks;
    v->s = reinterpret_cast<cudaStream_t>(stream);
    TraceArgs &a = v->a;
    a = TraceArgs{};
    a.traversal = p->traversal;
    a.T_min = p->T_min;
    a.alpha_max = p->alpha_max;
    a.bg0 = p->bg[0];
    a.bg1 = p->bg[1];
    a.bg2 = p->bg[2];
    a.ckpt_cap = (int)C;
    a.evict_cap = (int)E;
    a.packet_stack = p->packet_stack > 0 ? std::min(p->packet_stack, kPacketStack) : kPacketStack;
    int n_slots = v->blocks * 128;
    size_t ws = (size_t)blocks * per_block;
    // earlier work on any stream (the scenes' builds) completes before steps run on the
    // server's own streams
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->queue, kSteps * kQueueStride * sizeof(unsigned));
    for (int i = 0; i < n_steps && e == cudaSuccess; ++i) {
        SrvStep &sst = v->steps[i];
        if (i == 0) {
            sst.s = v->s;
        } else {
            e = cudaStreamCreateWithFlags(&sst.s, cudaStreamNonBlocking);
            sst.own_stream = e == cudaSuccess;
        }
        if (e == cudaSuccess) e = cudaMalloc(&sst.ws, ws);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sst.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sst.h, sizeof(ServeSeg) * v->max_inflight);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d, sizeof(ServeSeg) * v->max_inflight);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d_done, sizeof(unsigned) * v->max_inflight);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sst.h_flag, sizeof(unsigned) * v->max_inflight,
                                                cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(sst.h_flag, 0, sizeof(unsigned) * v->max_inflight);
            e = cudaHostGetDevicePointer((void **)&sst.d_flag, sst.h_flag, 0);
        }
    }
    char *arena_base = nullptr;
    if (e == cudaSuccess && arena > 0) e = cudaMalloc((void **)&arena_base, arena);
    if (e != cudaSuccess) {
        cudaGetLastError();
        server_free(v);
        return grtx_fail(GRTX_ERR_OOM, "server allocation failed");
    }
    v->arena.reset(arena_base, arena);
    v->list_bytes = (size_t)n_steps * ws;
    v->device_bytes = v->list_bytes + arena + kSteps * kQueueStride * sizeof(unsigned) +
                      (size_t)n_steps * (sizeof(ServeSeg) + sizeof(unsigned)) * v->max_inflight;
    a.n_slots = n_slots;
    *out = v;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_submit(grtx_server *v, const grtx_request *reqs, int n)
{
    if (!v || (n > 0 && !reqs) || n < 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad submit arguments");
    if ((int64_t)v->pending.size() + n > kMaxPending) return grtx_fail(GRTX_ERR_BUSY, "pending queue is full");
    std::vector<SrvReq *> add;
    for (int i = 0; i < n; ++i) {
        const grtx_request &q = reqs[i];
        int st = GRTX_OK;
        size_t out_bytes = 0;
        if (!q.d_rgbT && q.cam.width > 0 && q.cam.height > 0)
            out_bytes = Arena::round((size_t)q.cam.width * (size_t)q.cam.height * 16);
        if (q.scene_id < 0 || q.scene_id >= (int)v->scenes.size()) st = grtx_fail(GRTX_ERR_NOT_FOUND, "unknown scene id");
        else if (!q.d_rgbT && v->arena.bytes == 0)
            st = grtx_fail(GRTX_ERR_INVALID_ARG, "a server-owned output (d_rgbT = NULL) needs a server memory budget");
        else if (!q.d_rgbT && out_bytes > v->arena.bytes)
            st = grtx_fail(GRTX_ERR_OOM, "the request's output (" + std::to_string(out_bytes) +
                                             " bytes) exceeds the server's output arena (" +
                                             std::to_string(v->arena.bytes) + " bytes)");
        else if ((uintptr_t)q.d_rgbT & 15) st = grtx_fail(GRTX_ERR_INVALID_ARG, "bad output buffer");
        SrvReq *r = nullptr;
        if (st == GRTX_OK) {
            r = new (std::nothrow) SrvReq();
            if (!r) st = grtx_fail(GRTX_ERR_OOM, "host allocation failed");
        }
        if (st == GRTX_OK) {
            r->r = q;
            r->out_bytes = out_bytes;
            st = grtx_fill_camera(r->cam, r->n_items, &q.cam);
        }
        if (st != GRTX_OK) {
            delete r;
            for (auto *x : add) delete x;
            return st;
        }
        add.push_back(r);
    }
    for (auto *r : add) v->pending.push_back(r);
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_poll(grtx_server *v, grtx_completion *done, int max_done, int *n_done, int wait)
{
    if (!v || !n_done || max_done < 0 || (max_done > 0 && !done)) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad poll arguments");
    *n_done = 0;
    int got = 0;
    // a segment is complete: the request is reported once all of its items have been
    // scheduled and all of its segments are complete
    auto segment_done = [&](SrvStep &st, size_t j, double t) {
        st.seg_seen[j] = 1;
        SrvReq *r = st.seg_req[j];
        if (--r->pending_segs > 0 || r->next < r->n_items) return;
        grtx_completion c;
        c.tag = r->r.tag;
        c.status = GRTX_OK;
        c.reserved = 0;
        c.t_admit = r->t_admit;
        c.t_done = t;
        c.d_rgbT = r->r.d_rgbT;
        v->backlog.push_back(c);
        v->active.erase(std::find(v->active.begin(), v->active.end(), r));
        delete r;
        ++got;
    };
    for (;;) {
        // segments finished inside running steps
        double t = now_s();
        for (int si : v->inflight) {
            SrvStep &st = v->steps[si];
            const volatile unsigned *flag = st.h_flag;
            for (size_t j = 0; j < st.seg_req.size(); ++j)
                if (!st.seg_seen[j] && flag[j] == st.seq) segment_done(st, j, t);
        }
        // finished steps free their slots (every segment is complete once the launch is)
        while (!v->inflight.empty()) {
            SrvStep &st = v->steps[v->inflight.front()];
            cudaError_t q = cudaEventQuery(st.ev);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return grtx_cuda_fail(q, "serve step");
            t = now_s();
            for (size_t j = 0; j < st.seg_req.size(); ++j)
                if (!st.seg_seen[j]) segment_done(st, j, t);
            st.seg_req.clear();
            st.seg_seen.clear();
            st.busy = false;
            v->inflight.pop_front();
        }
        // admission of pending requests into free slots, in submission order; a request
        // whose server-owned output does not fit the arena holds the ones behind it
        while ((int)v->active.size() < v->max_inflight && !v->pending.empty()) {
            SrvReq *r = v->pending.front();
            if (r->out_bytes) {
                char *o = v->arena.alloc(r->out_bytes);
                if (!o) break;
                r->r.d_rgbT = (float *)o;
            }
            v->pending.pop_front();
            r->t_admit = now_s();
            v->active.push_back(r);
        }
        // keep up to n_steps steps enqueued, one per slot
        while ((int)v->inflight.size() < v->n_steps && has_unscheduled(v)) {
            int si = -1;
            for (int i = 0; i < v->n_steps; ++i)
                if (!v->steps[i].busy) { si = i; break; }
            if (si < 0) break;
            int st = schedule_step(v, si);
            if (st != GRTX_OK) return st;
        }
        if (!wait || got > 0 || v->inflight.empty()) break;
        cudaError_t e = cudaEventSynchronize(v->steps[v->inflight.front()].ev);
        if (e != cudaSuccess) return grtx_cuda_fail(e, "serve step");
    }
    while (*n_done < max_done && !v->backlog.empty()) {
        done[(*n_done)++] = v->backlog.front();
        v->backlog.pop_front();
    }
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_render_requests(grtx_server *v, const grtx_request *reqs, int n, grtx_completion *done,
                                             int *n_done, void *stream)
{
    (void)stream;   // all server work runs on the server's stream
    if (!v || !n_done || (n > 0 && !done)) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad arguments");
    int st = grtx_server_submit(v, reqs, n);
    if (st) return st;
    *n_done = 0;
    while (*n_done < n) {
        int got = 0;
        st = grtx_server_poll(v, done + *n_done, n - *n_done, &got, 1);
        if (st) return st;
        *n_done += got;
        if (got == 0 && v->inflight.empty() && v->active.empty() && v->backlog.empty()) {
            if (!v->pending.empty())          // held until outputs are released, which cannot happen here
                return grtx_fail(GRTX_ERR_BUSY, "requests are held: the output arena is full until outputs are released");
            break;
        }
    }
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_load(const grtx_server *v, int *n_inflight, int *n_pending)
{
    if (!v) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    if (n_inflight) *n_inflight = (int)v->active.size();
    if (n_pending) *n_pending = (int)v->pending.size();
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_release(grtx_server *v, float *d_rgbT)
{
    if (!v) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    if (!v->arena.release((char *)d_rgbT)) return grtx_fail(GRTX_ERR_NOT_FOUND, "not a live server-owned output");
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_get_info(const grtx_server *v, grtx_server_info *info)
{
    if (!v || !info) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL argument");
    info->n_step_slots = v->n_steps;
    info->blocks_per_step = v->blocks;
    info->list_bytes = (int64_t)v->list_bytes;
    info->arena_bytes = (int64_t)v->arena.bytes;
    info->arena_used = (int64_t)v->arena.used;
    info->device_bytes = (int64_t)v->device_bytes;
    info->n_inflight = (int32_t)v->active.size();
    info->n_pending = (int32_t)v->pending.size();
    return GRTX_OK;
}

extern "C" GRTX_API void grtx_server_destroy(grtx_server *v)
{
    if (v) server_free(v);
}
