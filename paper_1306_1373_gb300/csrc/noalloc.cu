// dct_batch_run_noalloc: the batched codec pass for callers that must not
// allocate memory.
//
// dct_batch_prepare keeps its work list (item descriptors, tile offsets,
// quantiser tables) in device memory the plan allocates.  Some callers
// cannot allow that: a process whose device memory is reserved up front by
// another allocator (a framework's caching allocator holding nearly all of
// HBM), a latency-critical loop that cannot absorb the implicit device
// synchronisation of cudaMalloc / cudaFree, or a deployment with a fixed
// memory budget that forbids allocation after start-up.  This entry point
// runs the same kernels with the work list in a fixed-size array that is
// part of the loaded library image instead.
//
// The array lives in every device that loads the library, for the life of
// the process.  In host code its name is only a host-side stand-in, so the
// device address is looked up with cudaGetSymbolAddress once per device, on
// that device's first call, and kept in a per-device table.
//
// The descriptors and tables are staged in this call's stack frame and
// copied with cudaMemcpyAsync from that pageable memory: the driver may
// first wait for the work already queued on the stream, and the call refuses
// to run while the stream is being captured (a graph would replay copies
// from a frame that no longer exists).
#include <cstring>

#include "host_common.h"

namespace dctgb {

// Largest batch the static work list holds.
constexpr int kNoAllocMaxItems = 64;

struct NoAllocList {
    PlaneArg items[kNoAllocMaxItems];
    int32_t tile_begin[kNoAllocMaxItems + 1];
    int32_t pad[(256 - ((kNoAllocMaxItems + 1) * 4) % 256) / 4];
    QuantSet tabs[kNoAllocMaxItems];
};

// The scratch: one work list shared by every call on a device.
static __device__ __align__(256) NoAllocList g_noalloc_list;

// Kernels of batch.cu, launched unchanged.
__global__ void k_batch_init(const PlaneArg* __restrict__ items, int n, int do_sse, int do_stats,
                             unsigned int* counters, int ncounters);

constexpr int kMaxDevices = 64;
static NoAllocList* g_list_addr[kMaxDevices];   // device address per device, nullptr until set up

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_batch_run_noalloc(const dct_batch_item* items, int n, uint32_t ops, uint64_t* sse_out,
                                            dct_stream_t stream) {
    if (!items) return fail(DCT_ERR_INVALID_ARG, "null items");
    if (n < 1 || n > kNoAllocMaxItems) {
        return fail(DCT_ERR_INVALID_ARG, "dct_batch_run_noalloc takes 1.." + std::to_string(kNoAllocMaxItems) +
                                             " items (the size of its static work list); use dct_batch_prepare "
                                             "for larger batches");
    }
    const uint32_t known = DCT_OP_COMPRESS | DCT_OP_RECONSTRUCT | DCT_OP_SSE | DCT_OP_TWO_PASS;
    if (ops == 0 || (ops & ~known)) return fail(DCT_ERR_INVALID_ARG, "ops must be a non-empty mask of DCT_OP_*");
    if ((ops & DCT_OP_SSE) && !sse_out) return fail(DCT_ERR_INVALID_ARG, "DCT_OP_SSE needs sse_out");
    if (sse_out && (((uintptr_t)sse_out) & 7u)) return fail(DCT_ERR_INVALID_ARG, "sse_out must be 8-byte aligned");
    const bool comp = ops & DCT_OP_COMPRESS, rec = ops & DCT_OP_RECONSTRUCT, sse = ops & DCT_OP_SSE;
    const bool two = ops & DCT_OP_TWO_PASS;
    if (two && !(comp && rec)) return fail(DCT_ERR_INVALID_ARG, "DCT_OP_TWO_PASS needs COMPRESS|RECONSTRUCT");

    unsigned mode;
    if (two) mode = kLoadCoef | kInverse | kStoreRecon | (sse ? kSse : 0u) | kOwnCodes;   // reads its own codes
    else if (comp && !rec && !sse) mode = kLoadPix | kStoreCoef;
    else if (rec && !comp) mode = kLoadCoef | kInverse | kStoreRecon | (sse ? kSse : 0u);
    else mode = kLoadPix | kInverse | (sse ? kSse : 0u) | (comp ? kStoreCoef : 0u) | (rec ? kStoreRecon : 0u);

    // A plan on the stack carries the limits and launch shape the shared
    // launcher reads; nothing is allocated.  The shape is a new plan's
    // default (two lanes per block where the operation has a two-lane
    // kernel); without a tile counter those kernels give each warp a fixed
    // contiguous tile range, so no device word is needed.
    dct_plan_s plan;
    memset(&plan, 0, sizeof plan);
    plan.desc.max_width = 1 << 16;
    plan.desc.max_height = 1 << 16;
    plan.desc.layout = DCT_LAYOUT_GRAY8;
    plan.desc.max_batch = kNoAllocMaxItems;
    plan.shape = default_shape();

    // Pass 1, host only: check every item against the limits of
    // dct_plan_create (at most 65536 x 65536, below 2^31 samples per plane)
    // and dct_batch_prepare (source samples are needed only when the
    // operation reads them; at most 2^30 tiles), fill the descriptors in a
    // stack buffer and assign table slots.  Nothing touches the GPU until
    // every item is valid.
    struct {
        PlaneArg items[kNoAllocMaxItems];
        int32_t tile_begin[kNoAllocMaxItems + 1];
    } h;
    QuantSet tab;
    int cursor = 0, ntabs = 0;
    int tab_quality[kNoAllocMaxItems], tab_chroma[kNoAllocMaxItems], tab_item[kNoAllocMaxItems];
    const uint16_t* tab_custom[kNoAllocMaxItems];
    const bool need_src = (mode & kLoadPix) || (mode & kSse) || two;
    for (int i = 0; i < n; ++i) {
        const dct_batch_item& it = items[i];
        dct_status st = DCT_OK;
        if (need_src) {
            if ((st = check_plane(&plan, it.src, "item src")) != DCT_OK) return st;
        } else if (it.src.width < 1 || it.src.height < 1 || it.src.width > plan.desc.max_width ||
                   it.src.height > plan.desc.max_height) {
            return fail(DCT_ERR_INVALID_ARG, "item size outside 1..65536 x 1..65536");
        }
        if ((int64_t)it.src.width * it.src.height > (int64_t)1 << 31)
            return fail(DCT_ERR_INVALID_ARG, "item width * height must stay below 2^31 samples");
        PlaneArg& a = h.items[i];
        memset(&a, 0, sizeof a);
        fill_plane(a, it.src, cursor);
        if (cursor < 0 || cursor > (1 << 30)) return fail(DCT_ERR_INVALID_ARG, "batch too large");
        a.src = it.src.data;
        a.src_pitch = it.src.pitch;
        a.ref = it.src.data;
        a.ref_pitch = it.src.pitch;
        int fl = (it.src.data && (((uintptr_t)it.src.data) & 7u) == 0 && (it.src.pitch & 7) == 0) ? (kVecSrc | kVecRef)
                                                                                                  : 0;
        if ((mode & kStoreCoef) || (mode & kLoadCoef)) {
            if (!it.coeffs) return fail(DCT_ERR_INVALID_ARG, "item coeffs is null");
            if (((uintptr_t)it.coeffs) & 15u) return fail(DCT_ERR_INVALID_ARG, "item coeffs must be 16-byte aligned");
            a.coef = it.coeffs;
        }
        if (mode & kStoreRecon) {
            if (!it.recon) return fail(DCT_ERR_INVALID_ARG, "item recon is null");
            if (it.recon_pitch < it.src.width) return fail(DCT_ERR_INVALID_ARG, "item recon_pitch < width");
            a.dst = it.recon;
            a.dst_pitch = it.recon_pitch;
            if ((((uintptr_t)it.recon) & 7u) == 0 && (it.recon_pitch & 7) == 0) fl |= kVecDst;
        }
        a.flags = fl;
        a.sse = sse ? reinterpret_cast<unsigned long long*>(sse_out) + i : nullptr;
        if (it.quality < 0 || it.quality > 100) return fail(DCT_ERR_INVALID_ARG, "item quality must be 0..100");
        if (it.quality == 0 && !it.qtab_host) return fail(DCT_ERR_INVALID_ARG, "item quality 0 needs qtab_host");
        int t = -1;
        for (int k = 0; k < ntabs && t < 0; ++k) {
            if (it.quality > 0 && tab_quality[k] == it.quality && tab_chroma[k] == (it.chroma ? 1 : 0)) t = k;
            if (it.quality == 0 && tab_quality[k] == 0 && memcmp(tab_custom[k], it.qtab_host, 128) == 0) t = k;
        }
        if (t < 0) {
            st = build_tables(it.quality, it.qtab_host, 64, it.chroma, tab);   // validates custom tables
            if (st != DCT_OK) return st;
            tab_quality[ntabs] = it.quality;
            tab_chroma[ntabs] = it.chroma ? 1 : 0;
            tab_custom[ntabs] = it.qtab_host;
            tab_item[ntabs] = i;
            t = ntabs++;
        }
        a.table = t;
        h.tile_begin[i] = a.tile_begin;
    }
    h.tile_begin[n] = cursor;

    // The descriptors are copied from this call's stack frame.  Captured into
    // a graph, those copies would read a frame that is gone when the graph
    // replays, so the call refuses to run on a stream that is capturing.
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(DCT_ERR_UNSUPPORTED, "dct_batch_run_noalloc does not run on a stream that is being captured "
                                         "(its descriptors are copied from the caller's stack)");

    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(DCT_ERR_UNSUPPORTED, "device index beyond 63");
    if (!g_list_addr[dev]) {
        // first call on this device: find where the array lives on it
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_list);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_list_addr[dev] = static_cast<NoAllocList*>(p);
    }
    NoAllocList* dlist = g_list_addr[dev];
    e = cudaDeviceGetAttribute(&plan.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    plan.device = dev;

    // Pass 2: upload the distinct tables from one stack buffer each, then
    // the descriptors (pageable copies: cudaMemcpyAsync has read them when
    // it returns).
    for (int k = 0; k < ntabs; ++k) {
        const dct_batch_item& it = items[tab_item[k]];
        build_tables(it.quality, it.qtab_host, 64, it.chroma, tab);
        e = cudaMemcpyAsync(dlist->tabs + k, &tab, sizeof(QuantSet), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "table upload");
    }
    e = cudaMemcpyAsync(dlist->items, h.items, sizeof(PlaneArg) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dlist->tile_begin, h.tile_begin, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "work list upload");
    if (sse) {
        k_batch_init<<<1, 64, 0, s>>>(dlist->items, n, 1, 0, nullptr, 0);   // the SSE outputs start at zero
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "SSE clear launch");
    }
    if (two) {
        e = batch_launch(kLoadPix | kStoreCoef, dlist->items, dlist->tile_begin, dlist->tabs, n, cursor, &plan, s);
        if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    }
    e = batch_launch(mode, dlist->items, dlist->tile_begin, dlist->tabs, n, cursor, &plan, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return DCT_OK;
}
