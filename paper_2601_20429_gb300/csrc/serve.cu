// Serving: several resident scenes and a stream of camera requests. Requests are admitted
// into a bounded set (continuous batching), and, under a memory budget, only while their
// outputs fit the server's output arena. One persistent launch (the live launch) traces the
// 32-ray tiles of every admitted request (mixed scenes and resolutions) from one queue; the
// host keeps publishing work to it while it runs, a little at a time and earliest deadline
// first, so that a request that arrives waits for little of the others' work, and the launch
// never drains into a tail while work is waiting. Its warps wait a short while for more work
// when there is none. A full or idle launch is closed and the next one starts in another step
// slot (own stream and lists), taking the SMs the old one's last warps leave.
// A scheduler thread of the server does all of this; callers only queue requests and take
// completions.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "serve_host.h"
#include "trace_impl.cuh"

using grtx_serve::Arena;

#define GRTX_EXTERN_SERVE(K)                                                                                 \
    extern template int serve_launch<K>(const TraceArgs &, const ServeSeg *, const unsigned *, int, int,            \
                                        cudaStream_t, ServeLive);                                                    \
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
constexpr int kSteps = 2;         // step slots (streams): the live launch and one finishing
constexpr int kQueueStride = 32;   // the slots' queue counters on separate 128-byte lines
constexpr unsigned kLingerNs = 2000000;   // default wait of a live launch's warps for new work
constexpr double kSizeNs = 5.0;           // default deadline weight: 5 ns per ray

double now_s()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int serve_launch_k(int k, const TraceArgs &a, const ServeSeg *segs, const unsigned *begins, int n, int blocks,
                   cudaStream_t s, const ServeLive &live)
{
    switch (k) {
    case 1: return serve_launch<1>(a, segs, begins, n, blocks, s, live);
    case 2: return serve_launch<2>(a, segs, begins, n, blocks, s, live);
    case 4: return serve_launch<4>(a, segs, begins, n, blocks, s, live);
    case 8: return serve_launch<8>(a, segs, begins, n, blocks, s, live);
    case 16: return serve_launch<16>(a, segs, begins, n, blocks, s, live);
    default: return serve_launch<32>(a, segs, begins, n, blocks, s, live);
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
    std::vector<std::pair<unsigned, unsigned>> retry;   // {first item, count}: ranges a launch did not trace
};


// A step slot: each has its own stream, per-slot lists and queue counter, so that the next
// launch's blocks take the SMs the previous launch's blocks leave while its slowest warps
// finish. Completion is per segment (a piece of a request): the warp that finishes a
// segment's last tile raises the segment's flag in pinned host memory, so a request is
// reported as soon as its own tiles are done, not when the launch ends.
struct SrvStep {
    cudaEvent_t ev = nullptr;
    cudaStream_t s = nullptr;  // slot 0: the server's stream; the others: created by the server
    bool own_stream = false;
    void *ws = nullptr;        // checkpoint and eviction lists of this slot's launches
    ServeSeg *h = nullptr;     // pinned host copy of the segment table
    ServeSeg *d = nullptr;     // device segment table
    unsigned *h_begins = nullptr, *d_begins = nullptr;   // each segment's first launch item (pinned / device)
    unsigned *d_done = nullptr;     // device: items finished per segment
    unsigned *h_flag = nullptr;     // pinned, mapped: the step's sequence number once a segment is done
    unsigned *d_flag = nullptr;     // device address of h_flag
    unsigned seq = 0;               // this launch's sequence number
    std::vector<SrvReq *> seg_req;  // request of each segment
    std::vector<char> seg_seen;     // segment completion already taken into account
    std::vector<unsigned> seg_begin, seg_item;   // each segment's first launch item and request item
    // appends to the running launch: published {items, closed} (device), the pinned staging of
    // the item counts (one word per publication, so that a copy still queued never reads a
    // later count), the list of claims given up, and the count of warps that gave up (device,
    // and its mapped host mirror)
    unsigned *d_avail = nullptr, *h_avail = nullptr, *d_lost = nullptr;
    unsigned *d_exited = nullptr, *h_exited = nullptr, *d_exited_host = nullptr;
    unsigned *h_claimed = nullptr, *d_claimed_host = nullptr;   // claims so far (mapped, approximate)
    cudaEvent_t ready = nullptr;    // recorded before the launch: appends are copied after it
    unsigned n_items = 0;           // items published to this launch
    int n_pub = 0;                  // publications used (staging words)
    bool closed = false;            // the host appends nothing more to this launch
    double t_pub = 0;               // host time of the launch's last publication
    unsigned claimed_max = 0;       // largest claim mirror the host has read
    bool busy = false;
};

}  // namespace

struct grtx_server {
    std::vector<grtx_scene *> scenes;
    grtx_params p;
    int64_t max_rays = 0;
    int max_inflight = 0;
    int seg_cap = 0;            // segment records per launch (4 per admitted request)
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
    cudaStream_t ctl = nullptr; // copies of segments appended to running launches
    unsigned lost_cap = 0;      // warps of a launch
    std::vector<unsigned> h_lost;
    unsigned *h_one = nullptr;  // pinned: word 1 (the copy that closes a launch), then read-back words
    int live = -1;              // slot of the launch new work is appended to (-1: none)
    int64_t n_launches = 0, n_appends = 0, n_retried = 0;
    unsigned linger_ns = kLingerNs;
    double size_ns = kSizeNs;   // deadline weight of a request's size (see take_pieces)
    bool append_guard = true;   // see grtx_server_set_append_guard
    // the scheduler thread: it admits, publishes, starts and closes launches, and collects
    // completions, every 20 us while there is work; callers only queue requests and take
    // completions. Every field above is guarded by mu.
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    bool admit_blocked = false; // pending requests wait for arena memory (after an admission pass)
    int dev = 0;
    int err = GRTX_OK;          // a failure of the scheduler thread, reported by every later poll
    std::string err_msg;
};

namespace {

void server_free(grtx_server *v)
{
    for (auto &st : v->steps)
        if (st.ev) cudaStreamSynchronize(st.s);     // (unused slots have no event)
    if (v->ctl) {
        cudaStreamSynchronize(v->ctl);
        cudaStreamDestroy(v->ctl);
    }
    for (auto &st : v->steps) {
        if (st.ev) cudaEventDestroy(st.ev);
        if (st.ready) cudaEventDestroy(st.ready);
        if (st.d_avail) cudaFree(st.d_avail);
        if (st.h_avail) cudaFreeHost(st.h_avail);
        if (st.d_lost) cudaFree(st.d_lost);
        if (st.d_exited) cudaFree(st.d_exited);
        if (st.h_exited) cudaFreeHost(st.h_exited);
        if (st.h_claimed) cudaFreeHost(st.h_claimed);
        if (st.h) cudaFreeHost(st.h);
        if (st.d) cudaFree(st.d);
        if (st.h_begins) cudaFreeHost(st.h_begins);
        if (st.d_begins) cudaFree(st.d_begins);
        if (st.d_done) cudaFree(st.d_done);
        if (st.h_flag) cudaFreeHost(st.h_flag);
        if (st.ws) cudaFree(st.ws);
        if (st.own_stream) cudaStreamDestroy(st.s);
    }
    if (v->queue) cudaFree(v->queue);
    if (v->h_one) cudaFreeHost(v->h_one);
    if (v->arena.base) cudaFree(v->arena.base);
    for (auto *r : v->pending) delete r;
    for (auto *r : v->active) delete r;
    delete v;
}

using Piece = grtx_serve::Piece<SrvReq>;


// Unscheduled work in deadline order (see grtx_serve::take_pieces).
std::vector<Piece> take_pieces(grtx_server *v, int64_t budget, int max_pieces)
{
    return grtx_serve::take_pieces<SrvReq>(v->active, v->size_ns, budget, max_pieces);
}

// Segment records (and begins entries) of `pieces`, after the launch's current segments and
// items.
void fill_segments(grtx_server *v, SrvStep &st, const std::vector<Piece> &pieces)
{
    for (const Piece &pc : pieces) {
        const int j = (int)st.seg_req.size();
        ServeSeg &g = st.h[j];
        g.sc = grtx_scene_ref(v->scenes[pc.r->r.scene_id]);
        g.cam = pc.r->cam;
        g.out = (float4 *)pc.r->r.d_rgbT;
        g.item_begin = pc.begin;
        g.step_begin = st.n_items;
        g.count = pc.count;
        g.pad = 0;
        st.h_begins[j] = st.n_items;
        st.seg_req.push_back(pc.r);
        st.seg_seen.push_back(0);
        st.seg_begin.push_back(st.n_items);
        st.seg_item.push_back(pc.begin);
        st.n_items += pc.count;
        pc.r->pending_segs++;
    }
}

// Launch one step over unscheduled work (up to max_rays items, least remaining work first);
// more is appended to it as its warps use up what was published.
int schedule_step(grtx_server *v, int si)
{
    SrvStep &st = v->steps[si];
    std::vector<Piece> pieces = take_pieces(v, v->max_rays, v->seg_cap);
    if (pieces.empty()) return GRTX_OK;
    st.seg_req.clear();
    st.seg_seen.clear();
    st.seg_begin.clear();
    st.seg_item.clear();
    st.n_items = 0;
    fill_segments(v, st, pieces);
    const int n = (int)st.seg_req.size();
    TraceArgs a = v->a;
    const size_t S = (size_t)a.n_slots;
    a.ck0 = (uint2 *)st.ws;
    a.ck1 = a.ck0 + S * a.ckpt_cap;
    a.ev = a.ck0 + S * 2 * a.ckpt_cap;
    a.queue = v->queue + kQueueStride * si;
    a.n_items = st.n_items;
    set_list_offsets(a, 2 * (size_t)a.ckpt_cap + (size_t)a.evict_cap);   // size checked at creation
    a.discard = lists_discardable(a);
    st.h_avail[0] = st.n_items;
    *reinterpret_cast<volatile unsigned *>(st.h_exited) = 0;
    *reinterpret_cast<volatile unsigned *>(st.h_claimed) = 0;
    GRTX_CUDA(cudaMemcpyAsync(st.d, st.h, sizeof(ServeSeg) * n, cudaMemcpyHostToDevice, st.s));
    GRTX_CUDA(cudaMemsetAsync(st.d_begins, 0xff, sizeof(unsigned) * v->seg_cap, st.s));
    GRTX_CUDA(cudaMemcpyAsync(st.d_begins, st.h_begins, sizeof(unsigned) * n, cudaMemcpyHostToDevice, st.s));
    GRTX_CUDA(cudaMemcpyAsync(st.d_avail, st.h_avail, sizeof(unsigned), cudaMemcpyHostToDevice, st.s));
    GRTX_CUDA(cudaMemsetAsync(st.d_avail + 1, 0, sizeof(unsigned), st.s));
    GRTX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), st.s));
    GRTX_CUDA(cudaMemsetAsync(st.d_done, 0, sizeof(unsigned) * v->seg_cap, st.s));
    GRTX_CUDA(cudaMemsetAsync(st.d_lost, 0, sizeof(unsigned), st.s));
    GRTX_CUDA(cudaMemsetAsync(st.d_exited, 0, sizeof(unsigned), st.s));
    GRTX_CUDA(cudaEventRecord(st.ready, st.s));
    st.n_pub = 1;
    st.seq = ++v->seq;
    ServeLive live;
    live.seg_done = st.d_done;
    live.seg_flag = st.d_flag;
    live.seq = st.seq;
    live.avail = st.d_avail;
    live.lost = st.d_lost;
    live.lost_cap = v->lost_cap;
    live.exited = st.d_exited;
    live.exited_host = st.d_exited_host;
    // the warps' own bound on a wait without any publication. With the guard (the default) it
    // is a backstop for a host that stops polling, well past the host's own linger, so that an
    // append never races with warps giving up; without it, the linger itself
    live.linger_ns = (!v->append_guard || v->linger_ns == 0)
                         ? v->linger_ns
                         : (unsigned)std::min<uint64_t>(1000000000ull,
                                                        std::max<uint64_t>(20000000ull, 16ull * v->linger_ns));
    live.claimed_host = st.d_claimed_host;
    if (serve_launch_k(v->p.k, a, st.d, st.d_begins, v->seg_cap, v->blocks, st.s, live) != GRTX_OK) {
        cudaError_t e = cudaGetLastError();
        return grtx_cuda_fail(e == cudaSuccess ? cudaErrorLaunchFailure : e, "serve step launch");
    }
    GRTX_CUDA(cudaEventRecord(st.ev, st.s));
    st.busy = true;
    st.closed = false;
    st.t_pub = now_s();
    st.claimed_max = 0;
    v->inflight.push_back(si);
    v->live = si;
    ++v->n_launches;
    return GRTX_OK;
}

// Append unscheduled work to the running launch of slot si (its warps pick it up without a
// new launch): the records and their entries of the begins array, then the item count, on
// the control stream after the launch's own copies. Returns false when the launch's segment
// table (or its staging) is full, or its item numbers would come near 2^31.
bool append_to_step(grtx_server *v, int si)
{
    SrvStep &st = v->steps[si];
    const int room = std::min(v->seg_cap - (int)st.seg_req.size(), v->seg_cap - st.n_pub);
    // (item numbers stay below 2^31, with room for the claims of every warp past the end)
    if (room <= 0 || (uint64_t)st.n_items + (uint64_t)v->max_rays + 32ull * v->lost_cap >= (1ull << 31)) return false;
    std::vector<Piece> pieces = take_pieces(v, v->max_rays, room);
    if (pieces.empty()) return false;
    const int j0 = (int)st.seg_req.size();
    fill_segments(v, st, pieces);
    const int n = (int)st.seg_req.size();
    unsigned *count = st.h_avail + st.n_pub++;
    *count = st.n_items;
    cudaStreamWaitEvent(v->ctl, st.ready, 0);
    cudaMemcpyAsync(st.d + j0, st.h + j0, sizeof(ServeSeg) * (n - j0), cudaMemcpyHostToDevice, v->ctl);
    cudaMemcpyAsync(st.d_begins + j0, st.h_begins + j0, sizeof(unsigned) * (n - j0), cudaMemcpyHostToDevice, v->ctl);
    cudaMemcpyAsync(st.d_avail, count, sizeof(unsigned), cudaMemcpyHostToDevice, v->ctl);
    st.t_pub = now_s();
    ++v->n_appends;
    return true;
}

// Nothing more is appended to the launch of slot si: its waiting warps stop (after the
// launch's appends, on the control stream).
void close_step(grtx_server *v, int si)
{
    SrvStep &st = v->steps[si];
    if (st.closed) return;
    cudaStreamWaitEvent(v->ctl, st.ready, 0);
    cudaMemcpyAsync(st.d_avail + 1, v->h_one, sizeof(unsigned), cudaMemcpyHostToDevice, v->ctl);
    st.closed = true;
    if (v->live == si) v->live = -1;
}

bool has_unscheduled(const grtx_server *v)
{
    for (const SrvReq *r : v->active)
        if (r->next < r->n_items || !r->retry.empty()) return true;
    return false;
}

}  // namespace

namespace {
void scheduler(grtx_server *v);

// Servers whose scheduler threads run: a process that exits without grtx_server_destroy stops
// them first (an exit handler registered after the CUDA runtime's own, so it runs before them).
std::mutex g_servers_mu;
std::vector<grtx_server *> g_servers;

void stop_servers_at_exit()
{
    std::lock_guard<std::mutex> g(g_servers_mu);
    for (grtx_server *v : g_servers) {
        {
            std::lock_guard<std::mutex> lk(v->mu);
            v->stop = true;
        }
        v->cv_work.notify_all();
        if (v->worker.joinable()) v->worker.join();
    }
    g_servers.clear();
}
}

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
    const int inflight_cap = max_inflight > 0 ? max_inflight : 64;
    const int seg_cap = 4 * inflight_cap;
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
    // segment tables, completion counts, publication words and given-up claims of each slot
    // (the tables: queue counters, and per slot the segment records, begins and completion
    // counts, four control words, and one given-up claim per warp)
    const grtx_serve::BudgetPlan plan = grtx_serve::plan_budget(
        (size_t)mem_budget_bytes, kSteps, blocks_full, per_block, kSteps * kQueueStride * sizeof(unsigned),
        (sizeof(ServeSeg) + 2 * sizeof(unsigned)) * seg_cap + 4 * sizeof(unsigned), sizeof(unsigned) * (kBlock / 32));
    if (plan.below_one_block)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "memory budget of " + std::to_string(mem_budget_bytes) +
                                                   " bytes is below twice one block of lists (" +
                                                   std::to_string(per_block) + " bytes)");
    if (!plan.fits) return grtx_fail(GRTX_ERR_INVALID_ARG, "memory budget too small");
    const int n_steps = plan.n_steps, blocks = plan.blocks;
    const size_t arena = plan.arena;
    grtx_server *v = new (std::nothrow) grtx_server();
    if (!v) return grtx_fail(GRTX_ERR_OOM, "host allocation failed");
    v->scenes.assign(scenes, scenes + n_scenes);
    v->p = *p;
    // work published to a launch at a time: by default two rounds of its warps' tiles
    v->max_rays = max_rays_per_step > 0 ? std::max<int64_t>(32, std::min<int64_t>(max_rays_per_step, (int64_t)1 << 28) / 32 * 32)
                                        : (int64_t)2 * 32 * blocks * (kBlock / 32);
    v->max_inflight = inflight_cap;
    v->seg_cap = seg_cap;
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
    v->lost_cap = (unsigned)blocks * (kBlock / 32);
    // earlier work on any stream (the scenes' builds) completes before steps run on the
    // server's own streams
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->queue, kSteps * kQueueStride * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v->ctl, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&v->h_one, 4 * sizeof(unsigned));
    if (e == cudaSuccess) *v->h_one = 1;
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
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sst.h, sizeof(ServeSeg) * seg_cap);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d, sizeof(ServeSeg) * seg_cap);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d_done, sizeof(unsigned) * seg_cap);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sst.h_flag, sizeof(unsigned) * seg_cap,
                                                cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(sst.h_flag, 0, sizeof(unsigned) * seg_cap);
            e = cudaHostGetDevicePointer((void **)&sst.d_flag, sst.h_flag, 0);
        }
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sst.h_begins, sizeof(unsigned) * seg_cap);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d_begins, sizeof(unsigned) * seg_cap);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d_avail, 2 * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sst.h_avail, sizeof(unsigned) * (seg_cap + 1));
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d_lost, sizeof(unsigned) * (1 + (size_t)v->lost_cap));
        if (e == cudaSuccess) e = cudaMalloc((void **)&sst.d_exited, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sst.h_exited, sizeof(unsigned), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            *sst.h_exited = 0;
            e = cudaHostGetDevicePointer((void **)&sst.d_exited_host, sst.h_exited, 0);
        }
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sst.h_claimed, sizeof(unsigned), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            *sst.h_claimed = 0;
            e = cudaHostGetDevicePointer((void **)&sst.d_claimed_host, sst.h_claimed, 0);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sst.ready, cudaEventDisableTiming);
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
    v->device_bytes = v->list_bytes + arena + plan.tables;
    a.n_slots = n_slots;
    cudaGetDevice(&v->dev);
    try {
        v->worker = std::thread(scheduler, v);
    } catch (...) {
        server_free(v);
        return grtx_fail(GRTX_ERR_OOM, "could not start the server's scheduler thread");
    }
    {
        static std::once_flag registered;
        std::call_once(registered, [] { std::atexit(stop_servers_at_exit); });
        std::lock_guard<std::mutex> g(g_servers_mu);
        g_servers.push_back(v);
    }
    *out = v;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_submit(grtx_server *v, const grtx_request *reqs, int n)
{
    if (!v || (n > 0 && !reqs) || n < 0) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad submit arguments");
    std::lock_guard<std::mutex> lk(v->mu);
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
    if (!add.empty()) {
        v->admit_blocked = false;          // until the scheduler's next admission pass
        v->cv_work.notify_one();
    }
    return GRTX_OK;
}

namespace {

// One pass of the scheduler (the caller holds v->mu): segments finished inside running
// launches, ended launches (their untraced tiles go back to their requests), admission,
// publication to the live launch, and a new launch when the live one is gone.
int advance(grtx_server *v)
{
    // a segment is complete (or its launch ended): the request is reported once all of its
    // items have been scheduled, traced, and all of its segments are complete
    auto segment_done = [&](SrvStep &st, size_t j, double t) {
        st.seg_seen[j] = 1;
        SrvReq *r = st.seg_req[j];
        if (--r->pending_segs > 0 || r->next < r->n_items || !r->retry.empty()) return;
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
    };
    // tiles of an ended launch that no warp traced (claims given up before the host published
    // them, or items published after the last warp stopped) go back to their requests, as
    // ranges of consecutive items
    auto recover = [&](SrvStep &st, int si) -> int {
        // (copies on the control stream, after the launch's appends; the launch has ended, and a
        // synchronous copy would also wait for the other streams' work)
        unsigned *qn = v->h_one + 1;                         // pinned: queue counter, lost count
        GRTX_CUDA(cudaMemcpyAsync(qn, v->queue + kQueueStride * si, sizeof(unsigned), cudaMemcpyDeviceToHost, v->ctl));
        GRTX_CUDA(cudaMemcpyAsync(qn + 1, st.d_lost, sizeof(unsigned), cudaMemcpyDeviceToHost, v->ctl));
        GRTX_CUDA(cudaStreamSynchronize(v->ctl));
        const unsigned q = qn[0];
        unsigned n_lost = std::min(qn[1], v->lost_cap);
        std::vector<std::pair<SrvReq *, unsigned>> tiles;    // {request, first item}
        auto add = [&](unsigned b) {
            const size_t j = (size_t)(std::upper_bound(st.seg_begin.begin(), st.seg_begin.end(), b) -
                                      st.seg_begin.begin()) - 1;
            tiles.push_back({st.seg_req[j], st.seg_item[j] + (b - st.seg_begin[j])});
        };
        if (n_lost) {
            v->h_lost.resize(n_lost);
            GRTX_CUDA(cudaMemcpyAsync(v->h_lost.data(), st.d_lost + 1, sizeof(unsigned) * n_lost, cudaMemcpyDeviceToHost,
                                      v->ctl));
            GRTX_CUDA(cudaStreamSynchronize(v->ctl));
            for (unsigned b : v->h_lost)
                if (b < st.n_items) add(b);
        }
        for (unsigned b = q / 32 * 32; b < st.n_items; b += 32) add(b);
        v->n_retried += (int64_t)grtx_serve::give_back_tiles(tiles);
        return GRTX_OK;
    };
    // segments finished inside running steps
    double t = now_s();
    for (int si : v->inflight) {
        SrvStep &st = v->steps[si];
        const volatile unsigned *flag = st.h_flag;
        for (size_t j = 0; j < st.seg_req.size(); ++j)
            if (!st.seg_seen[j] && flag[j] == st.seq) segment_done(st, j, t);
    }
    // ended launches free their slots: untraced tiles go back to their requests, and
    // every other segment of the launch is complete
    for (size_t i = 0; i < v->inflight.size();) {
        const int si = v->inflight[i];
        SrvStep &st = v->steps[si];
        cudaError_t q = cudaEventQuery(st.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess) return grtx_cuda_fail(q, "serve step");
        int rs = recover(st, si);
        if (rs != GRTX_OK) return rs;
        t = now_s();
        for (size_t j = 0; j < st.seg_req.size(); ++j)
            if (!st.seg_seen[j]) segment_done(st, j, t);
        st.seg_req.clear();
        st.seg_seen.clear();
        st.seg_begin.clear();
        st.seg_item.clear();
        st.busy = false;
        if (v->live == si) v->live = -1;
        v->inflight.erase(v->inflight.begin() + (long)i);
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
    // new work joins the live launch: the host publishes up to max_rays more items (in
    // deadline order) whenever less than half of that is left unclaimed, so that a request
    // that arrives waits for at most that much work of others. The launch's warps take it as
    // they come free and wait for more when there is none. The host closes the live launch
    // (its waiting warps stop, so that the next launch gets their SMs) when no admitted
    // request is left, when it has had no work for linger_ns, when its segment table is
    // full, or when some of its warps have stopped waiting on their own (a host that did not
    // poll for the warps' backstop); the next work starts a launch in a free slot. (Without
    // the append guard the warps stop linger_ns after the last publication and the host
    // appends all the same: appends then race with warps giving up, which tests use.)
    if (v->live >= 0) {
        SrvStep &st = v->steps[v->live];
        // the mirror's writes come from many warps and may land out of order: keep the
        // largest value read (a lower bound of the claims, so `left` errs high, which only
        // delays the next publication)
        const unsigned mirror = *reinterpret_cast<volatile unsigned *>(st.h_claimed);
        st.claimed_max = std::max(st.claimed_max, mirror);
        const int64_t left = (int64_t)st.n_items - (int64_t)st.claimed_max;
        if (*reinterpret_cast<volatile unsigned *>(st.h_exited) != 0 || v->active.empty()) {
            close_step(v, v->live);
        } else if (has_unscheduled(v)) {
            if (2 * left < v->max_rays && !append_to_step(v, v->live)) close_step(v, v->live);
        } else if (left <= 0 && now_s() - st.t_pub >= 1e-9 * v->linger_ns) {
            close_step(v, v->live);
        }
    }
    if (v->live < 0 && (int)v->inflight.size() < v->n_steps && has_unscheduled(v)) {
        int si = -1;
        for (int i = 0; i < v->n_steps; ++i)
            if (!v->steps[i].busy) { si = i; break; }
        if (si >= 0) {
            int st = schedule_step(v, si);
            if (st != GRTX_OK) return st;
        }
    }
    v->admit_blocked = !v->pending.empty();
    return GRTX_OK;
}

// The scheduler thread: passes every 20 us while requests are queued, admitted or launches run;
// otherwise it sleeps until a submit, a release or the server's end.
void scheduler(grtx_server *v)
{
    cudaSetDevice(v->dev);
    std::unique_lock<std::mutex> lk(v->mu);
    while (!v->stop) {
        const bool busy = !v->pending.empty() || !v->active.empty() || !v->inflight.empty();
        if (v->err != GRTX_OK || !busy || (v->admit_blocked && v->active.empty() && v->inflight.empty())) {
            v->cv_done.notify_all();
            v->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        const size_t before = v->backlog.size();
        const int st = advance(v);
        if (st != GRTX_OK) {
            v->err = st;
            v->err_msg = grtx_last_error();
        }
        if (v->backlog.size() != before || st != GRTX_OK || v->active.empty()) v->cv_done.notify_all();
        lk.unlock();
        timespec ts = {0, 20000};
        nanosleep(&ts, nullptr);
        lk.lock();
    }
}

}  // namespace

extern "C" GRTX_API int grtx_server_poll(grtx_server *v, grtx_completion *done, int max_done, int *n_done, int wait)
{
    if (!v || !n_done || max_done < 0 || (max_done > 0 && !done)) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad poll arguments");
    *n_done = 0;
    std::unique_lock<std::mutex> lk(v->mu);
    // (with wait: until a completion, a failure, or nothing admitted that could complete)
    auto ready = [&] {
        return !v->backlog.empty() || v->err != GRTX_OK ||
               (v->active.empty() && (v->pending.empty() || v->admit_blocked));
    };
    while (wait && !ready()) v->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    while (*n_done < max_done && !v->backlog.empty()) {
        done[(*n_done)++] = v->backlog.front();
        v->backlog.pop_front();
    }
    if (v->err != GRTX_OK && *n_done == 0) return grtx_fail(v->err, v->err_msg);
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_render_requests(grtx_server *v, const grtx_request *reqs, int n, grtx_completion *done,
                                             int *n_done, void *stream)
{
    (void)stream;   // all server work runs on the server's streams
    if (!v || !n_done || (n > 0 && !done)) return grtx_fail(GRTX_ERR_INVALID_ARG, "bad arguments");
    int st = grtx_server_submit(v, reqs, n);
    if (st) return st;
    *n_done = 0;
    while (*n_done < n) {
        int got = 0;
        st = grtx_server_poll(v, done + *n_done, n - *n_done, &got, 1);
        if (st) return st;
        *n_done += got;
        if (got == 0) {
            std::lock_guard<std::mutex> lk(v->mu);
            if (v->active.empty() && v->backlog.empty()) {
                if (!v->pending.empty())      // held until outputs are released, which cannot happen here
                    return grtx_fail(GRTX_ERR_BUSY, "requests are held: the output arena is full until outputs are released");
                break;
            }
        }
    }
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_load(const grtx_server *cv, int *n_inflight, int *n_pending)
{
    if (!cv) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    grtx_server *v = const_cast<grtx_server *>(cv);   // (the lock)
    std::lock_guard<std::mutex> lk(v->mu);
    if (n_inflight) *n_inflight = (int)(v->active.size() + v->backlog.size());
    if (n_pending) *n_pending = (int)v->pending.size();
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_release(grtx_server *v, float *d_rgbT)
{
    if (!v) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    if (!v->arena.release((char *)d_rgbT)) return grtx_fail(GRTX_ERR_NOT_FOUND, "not a live server-owned output");
    v->admit_blocked = false;
    v->cv_work.notify_one();
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_set_linger(grtx_server *v, int64_t linger_ns)
{
    if (!v) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    if (linger_ns < 0 || linger_ns > 1000000000) return grtx_fail(GRTX_ERR_INVALID_ARG, "linger_ns must be in [0, 1e9]");
    std::lock_guard<std::mutex> lk(v->mu);
    v->linger_ns = (unsigned)linger_ns;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_set_append_guard(grtx_server *v, int on)
{
    if (!v) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    v->append_guard = on != 0;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_set_order(grtx_server *v, double size_ns_per_ray)
{
    if (!v) return grtx_fail(GRTX_ERR_INVALID_ARG, "server is NULL");
    if (!(size_ns_per_ray >= 0.0 && size_ns_per_ray <= 1e9)) return grtx_fail(GRTX_ERR_INVALID_ARG, "size_ns_per_ray must be in [0, 1e9]");
    std::lock_guard<std::mutex> lk(v->mu);
    v->size_ns = size_ns_per_ray;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_server_get_info(const grtx_server *cv, grtx_server_info *info)
{
    if (!cv || !info) return grtx_fail(GRTX_ERR_INVALID_ARG, "NULL argument");
    grtx_server *v = const_cast<grtx_server *>(cv);   // (the lock)
    std::lock_guard<std::mutex> lk(v->mu);
    info->n_step_slots = v->n_steps;
    info->blocks_per_step = v->blocks;
    info->list_bytes = (int64_t)v->list_bytes;
    info->arena_bytes = (int64_t)v->arena.bytes;
    info->arena_used = (int64_t)v->arena.used;
    info->device_bytes = (int64_t)v->device_bytes;
    info->n_inflight = (int32_t)(v->active.size() + v->backlog.size());
    info->n_pending = (int32_t)v->pending.size();
    info->n_launches = v->n_launches;
    info->n_appends = v->n_appends;
    info->n_retried_tiles = v->n_retried;
    return GRTX_OK;
}

extern "C" GRTX_API void grtx_server_destroy(grtx_server *v)
{
    if (!v) return;
    {
        std::lock_guard<std::mutex> g(g_servers_mu);
        g_servers.erase(std::remove(g_servers.begin(), g_servers.end(), v), g_servers.end());
    }
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
    }
    v->cv_work.notify_all();
    if (v->worker.joinable()) v->worker.join();
    for (int si : v->inflight) close_step(v, si);
    server_free(v);
}
