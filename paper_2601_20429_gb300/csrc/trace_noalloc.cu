// grtx_trace_forward_noalloc: the forward trace with its scratch memory in a fixed,
// library-owned device array instead of a workspace the library allocates.
//
// Why it exists: grtx_trace_forward grows a per-scene workspace with a stream-ordered
// allocation the first time it needs more room. Some callers cannot allow any allocation
// during rendering: a renderer that reserves all of its device memory up front under a hard
// budget, or a host loop that must not stall on the allocator between frames. This entry
// point never allocates; the price is a fixed upper bound on its scratch, which caps the
// number of rays in flight (fewer resident ray slots than the regular path may use).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "trace_impl.cuh"

#define GRTX_EXTERN_NOALLOC(K)                                                                   \
    extern template int trace_launch<K>(const TraceArgs &, int, bool, int, int, cudaStream_t); \
    extern template int trace_occupancy<K>(int, bool, int, int *);
GRTX_EXTERN_NOALLOC(1)
GRTX_EXTERN_NOALLOC(2)
GRTX_EXTERN_NOALLOC(4)
GRTX_EXTERN_NOALLOC(8)
GRTX_EXTERN_NOALLOC(16)
GRTX_EXTERN_NOALLOC(32)

int grtx_fill_camera(CamRef &a, unsigned &n_items_out, const grtx_camera *cam);
SceneRef grtx_scene_ref(const grtx_scene *sc);
int grtx_check_params(const grtx_params *p);

// The scratch: 256 bytes for the ray-queue counter, then the per-slot checkpoint lists and
// eviction list. Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GRTX_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t kCounterBytes = 256;
constexpr int kMaxDevices = 64;

// Device address of g_noalloc_scratch and SM count per device. Host code only sees a
// stand-in for the symbol, so the address is looked up once per device, with that device
// current; the once-flag makes concurrent first calls from several host threads safe.
struct DeviceScratch {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char *addr = nullptr;
    int sms = 1;
};
DeviceScratch g_dev[kMaxDevices];

int scratch_for_current_device(unsigned char **out, int *sms)
{
    int dev = 0;
    GRTX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return grtx_fail(GRTX_ERR_INVALID_ARG, "device ordinal out of range");
    DeviceScratch &d = g_dev[dev];
    std::call_once(d.once, [&d, dev]() {
        void *p = nullptr;
        d.err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (d.err != cudaSuccess) return;
        int n = 0;
        d.err = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        d.sms = n > 0 ? n : 1;
        d.addr = (unsigned char *)p;
    });
    if (d.err != cudaSuccess) return grtx_cuda_fail(d.err, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = d.addr;
    *sms = d.sms;
    return GRTX_OK;
}

int launch_noalloc(int k, const TraceArgs &a, int form, int blocks, cudaStream_t s)
{
    switch (k) {
    case 1: return trace_launch<1>(a, form, false, PASS_FWD, blocks, s);
    case 2: return trace_launch<2>(a, form, false, PASS_FWD, blocks, s);
    case 4: return trace_launch<4>(a, form, false, PASS_FWD, blocks, s);
    case 8: return trace_launch<8>(a, form, false, PASS_FWD, blocks, s);
    case 16: return trace_launch<16>(a, form, false, PASS_FWD, blocks, s);
    default: return trace_launch<32>(a, form, false, PASS_FWD, blocks, s);
    }
}

int occupancy_noalloc(int k, int form, int *bps)
{
    switch (k) {
    case 1: return trace_occupancy<1>(form, false, PASS_FWD, bps);
    case 2: return trace_occupancy<2>(form, false, PASS_FWD, bps);
    case 4: return trace_occupancy<4>(form, false, PASS_FWD, bps);
    case 8: return trace_occupancy<8>(form, false, PASS_FWD, bps);
    case 16: return trace_occupancy<16>(form, false, PASS_FWD, bps);
    default: return trace_occupancy<32>(form, false, PASS_FWD, bps);
    }
}

}  // namespace

extern "C" GRTX_API int grtx_trace_forward_noalloc(grtx_scene *sc, const grtx_camera *cam, const grtx_params *p,
                                                   float *d_rgbT, void *stream)
{
    if (!sc) return grtx_fail(GRTX_ERR_INVALID_ARG, "scene is NULL");
    int st = grtx_check_params(p);
    if (st) return st;
    if (p->alpha_min != sc->alpha_min)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "alpha_min differs from the one the scene was built with");
    if (p->traversal == GRTX_TRAVERSAL_SINGLE)
        return grtx_fail(GRTX_ERR_INVALID_ARG, "the fixed-scratch trace supports checkpoint and restart traversal");
    if (!d_rgbT || ((uintptr_t)d_rgbT & 15)) return grtx_fail(GRTX_ERR_INVALID_ARG, "rgbT must be a 16-byte aligned pointer");
    TraceArgs a = {};
    st = grtx_fill_camera(a.cam, a.n_items, cam);
    if (st) return st;
    int form = kernel_form(sc->form);
    a.sc = grtx_scene_ref(sc);
    a.traversal = p->traversal;
    a.T_min = p->T_min;
    a.alpha_max = p->alpha_max;
    a.bg0 = p->bg[0];
    a.bg1 = p->bg[1];
    a.bg2 = p->bg[2];
    a.ckpt_cap = p->ckpt_capacity > 0 ? p->ckpt_capacity : GRTX_DEFAULT_CKPT_CAPACITY;
    a.evict_cap = p->evict_capacity > 0 ? p->evict_capacity : GRTX_DEFAULT_EVICT_CAPACITY;
    a.packet_stack = p->packet_stack > 0 ? std::min(p->packet_stack, kPacketStack) : kPacketStack;
    a.rgbT = (float4 *)d_rgbT;
    bool ckpt = a.traversal == GRTX_TRAVERSAL_CHECKPOINT;
    size_t C = ckpt ? (size_t)a.ckpt_cap : 1, E = ckpt ? (size_t)a.evict_cap : 1;
    size_t per_block = 128 * (2 * C + E) * sizeof(uint2);
    const size_t room = GRTX_NOALLOC_SCRATCH_BYTES - kCounterBytes;
    if (per_block > room)
        return grtx_fail(GRTX_ERR_INVALID_ARG,
                         "checkpoint/eviction capacities need " + std::to_string(per_block) +
                             " bytes per 128-ray block, more than the " + std::to_string(room) +
                             " bytes of fixed scratch; lower ckpt_capacity / evict_capacity");
    unsigned char *base = nullptr;
    int sms = 1;
    st = scratch_for_current_device(&base, &sms);
    if (st) return st;
    int bps = 0;
    if (occupancy_noalloc(p->k, form, &bps) != GRTX_OK || bps <= 0)
        return grtx_fail(GRTX_ERR_CUDA, "occupancy query failed");
    int blocks = (int)std::min<size_t>((size_t)sms * bps, room / per_block);
    int n_slots = blocks * 128;
    uint2 *ws = (uint2 *)(base + kCounterBytes);
    a.ck0 = ws;
    a.ck1 = ws + (size_t)n_slots * C;
    a.ev = ws + (size_t)n_slots * 2 * C;
    a.n_slots = n_slots;
    a.queue = (unsigned *)base;
    set_list_offsets(a, 2 * C + E);          // the fixed scratch holds far fewer than 2^31 entries
    a.discard = lists_discardable(a);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the counter must start at zero; the lists are always written before they are read
    GRTX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(unsigned), s));
    if (launch_noalloc(p->k, a, form, blocks, s) != GRTX_OK) {
        cudaError_t e = cudaGetLastError();
        return grtx_cuda_fail(e == cudaSuccess ? cudaErrorLaunchFailure : e, "trace launch");
    }
    return GRTX_OK;
}
