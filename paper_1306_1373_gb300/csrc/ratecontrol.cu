// Learned rate control and the plain pipeline's quality bisection (no
// counterpart in the paper: they pick the quality factor of the Sec. 3.2
// pipeline for a target PSNR of Eq. 23).
//
// Every pass over the frames is the batched persistent kernel in its fused
// "SSE only" mode (transform, quantiser, dequantiser, inverse, SSE; nothing
// stored).  A frame's quality is switched on the device by rewriting the
// table index of its planes' work-list entries into a bank of 200 tables
// (luma then chroma, qualities 1..100), so the 8 bisection steps run
// without host round trips.  All decisions compare integer SSEs with
// thresholds computed on the host in float64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_common.h"

namespace dctgb {

constexpr int kBank = 200;      // luma q = 1..100 at [0, 100), chroma at [100, 200)
constexpr int kBisectSteps = 8;

// One work list (descriptors + tile offsets) in device and pinned host memory.
struct WorkList {
    PlaneArg* d_items = nullptr;
    int32_t* d_tb = nullptr;
    int32_t* d_frame = nullptr;   // slot frame -> global frame
    PlaneArg* h_items = nullptr;
    int32_t* h_tb = nullptr;
    int32_t* h_frame = nullptr;
    int nitems = 0, ntiles = 0, nframes = 0;
};

struct RcState {
    int cap = 0;                  // items (planes)
    QuantSet* d_bank = nullptr;
    WorkList all, luma, sub;
    unsigned long long* d_item_sse = nullptr;
    unsigned long long* d_stats = nullptr;
    float* d_feats = nullptr;
    float* d_target = nullptr;
    int32_t* d_w = nullptr;
    int32_t* d_h = nullptr;
    int32_t* d_q = nullptr;       // per global frame: chosen quality
    unsigned long long* d_sse = nullptr;   // per global frame: SSE at the chosen quality
    uint8_t* d_fell = nullptr;
    unsigned long long* d_thr = nullptr;   // SSE <= thr  <=>  PSNR >= target
    unsigned long long* d_blo = nullptr;   // band of |PSNR - target| <= 0.25
    unsigned long long* d_bhi = nullptr;
    int32_t* d_lo = nullptr;      // per slot frame bisection state
    int32_t* d_hi = nullptr;
    int32_t* d_mid = nullptr;
    int32_t* d_rej = nullptr;     // last rejected quality (0: none) and its SSE
    unsigned long long* d_rej_sse = nullptr;
    unsigned long long* d_fsse = nullptr;
    unsigned int* d_counter = nullptr;   // tile counter of the SSE passes
    // pinned host staging
    unsigned long long* h_thr = nullptr;
    unsigned long long* h_blo = nullptr;
    unsigned long long* h_bhi = nullptr;
    float* h_target = nullptr;
    int32_t* h_w = nullptr;
    int32_t* h_h = nullptr;
    uint8_t* h_fell = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// table index of every plane of a slot frame for that frame's quality; clears
// the planes' SSE words and the next pass's tile counter
__global__ void k_rc_set_quality(PlaneArg* items, int nitems, int k, const int32_t* __restrict__ frame,
                                 const int32_t* __restrict__ q_slot, const int32_t* __restrict__ q_global,
                                 unsigned int* tile_counter) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *tile_counter = 0u;
    if (i >= nitems) return;
    const int f = i / k;
    const int q = q_slot ? q_slot[f] : q_global[frame[f]];
    items[i].table = (i % k ? 100 : 0) + q - 1;
    *items[i].sse = 0ull;
}

__global__ void k_rc_frame_sse(const PlaneArg* __restrict__ items, int nframes, int k,
                               unsigned long long* __restrict__ fsse) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nframes) return;
    unsigned long long s = 0ull;
    for (int p = 0; p < k; ++p) s += *items[f * k + p].sse;
    fsse[f] = s;
}

// learned path: keep the prediction when its SSE lies in the 0.25 dB band
__global__ void k_rc_decide(const unsigned long long* __restrict__ fsse, const unsigned long long* __restrict__ blo,
                            const unsigned long long* __restrict__ bhi, int n, unsigned long long* __restrict__ sse,
                            uint8_t* __restrict__ fell) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const unsigned long long s = fsse[f];
    sse[f] = s;
    fell[f] = (s >= blo[f] && s <= bhi[f]) ? 0 : 1;
}

__global__ void k_bisect_init(int32_t* lo, int32_t* hi, int32_t* rej, int n) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) {
        lo[f] = 1;
        hi[f] = 100;
        rej[f] = 0;
    }
}

__global__ void k_bisect_mid(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi, int32_t* mid, int n) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < n) mid[f] = min(100, (lo[f] + hi[f]) >> 1);
}

__global__ void k_bisect_update(const unsigned long long* __restrict__ fsse, const int32_t* __restrict__ frame,
                                const unsigned long long* __restrict__ thr, const int32_t* __restrict__ mid,
                                int32_t* lo, int32_t* hi, int32_t* rej, unsigned long long* rej_sse, int n) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    if (fsse[f] <= thr[frame[f]]) {
        hi[f] = mid[f];
    } else {
        lo[f] = mid[f] + 1;
        rej[f] = mid[f];
        rej_sse[f] = fsse[f];
    }
}

// Results to the global arrays.  The last step's mid is Q*; when its PSNR
// lies outside the +-0.25 dB band but the last rejected quality (Q* - 1
// whenever a step rejected) lies inside it, that quality is the result.
__global__ void k_bisect_finish(const unsigned long long* __restrict__ fsse, const int32_t* __restrict__ frame,
                                const int32_t* __restrict__ mid, const int32_t* __restrict__ rej,
                                const unsigned long long* __restrict__ rej_sse, const unsigned long long* __restrict__ blo,
                                const unsigned long long* __restrict__ bhi, int n, int32_t* q, unsigned long long* sse) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const int g = frame[f];
    int qq = mid[f];
    unsigned long long s = fsse[f];
    const bool in_band = s >= blo[g] && s <= bhi[g];
    if (!in_band && rej[f] > 0 && rej_sse[f] >= blo[g] && rej_sse[f] <= bhi[g]) {
        qq = rej[f];
        s = rej_sse[f];
    }
    q[g] = qq;
    sse[g] = s;
}

// clears the statistics words of the luma list (min words to all ones)
__global__ void k_rc_clear_stats(unsigned long long* st, int nframes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nframes * kStatsWords) st[i] = (i % kStatsWords == kStMin) ? ~0ull : 0ull;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

static void free_list(WorkList& w) {
    cudaFree(w.d_items);
    cudaFree(w.d_tb);
    cudaFree(w.d_frame);
    cudaFreeHost(w.h_items);
    cudaFreeHost(w.h_tb);
    cudaFreeHost(w.h_frame);
    w = WorkList();
}

static void release_rc(RcState* r) {
    if (!r) return;
    cudaFree(r->d_bank);
    free_list(r->all);
    free_list(r->luma);
    free_list(r->sub);
    void* dev[] = {r->d_item_sse, r->d_stats, r->d_feats, r->d_target, r->d_w, r->d_h, r->d_q, r->d_sse,
                   r->d_fell, r->d_thr, r->d_blo, r->d_bhi, r->d_lo, r->d_hi, r->d_mid, r->d_rej, r->d_rej_sse,
                   r->d_fsse, r->d_counter};
    for (void* p : dev) cudaFree(p);
    void* host[] = {r->h_thr, r->h_blo, r->h_bhi, r->h_target, r->h_w, r->h_h, r->h_fell};
    for (void* p : host) cudaFreeHost(p);
    if (r->ev0) cudaEventDestroy(r->ev0);
    if (r->ev1) cudaEventDestroy(r->ev1);
    delete r;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) { return ws_malloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1)); }
template <typename T>
static cudaError_t halloc(T** p, size_t n) {
    return ws_malloc_host(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1));
}

static cudaError_t alloc_list(WorkList& w, int cap) {
    cudaError_t e = dalloc(&w.d_items, cap);
    if (e == cudaSuccess) e = dalloc(&w.d_tb, cap + 1);
    if (e == cudaSuccess) e = dalloc(&w.d_frame, cap);
    if (e == cudaSuccess) e = halloc(&w.h_items, cap);
    if (e == cudaSuccess) e = halloc(&w.h_tb, cap + 1);
    if (e == cudaSuccess) e = halloc(&w.h_frame, cap);
    return e;
}

static dct_status ensure_rc(dct_plan_t plan, cudaStream_t s) {
    if (plan->rc) return DCT_OK;
    const int cap = plan->desc.max_batch;
    if (cap < 1) return fail(DCT_ERR_STATE, "plan was created with max_batch = 0");
    RcState* r = new (std::nothrow) RcState();
    if (!r) return fail(DCT_ERR_ALLOC, "host allocation failed");
    r->cap = cap;
    cudaError_t e = dalloc(&r->d_bank, kBank);
    if (e == cudaSuccess) e = alloc_list(r->all, cap);
    if (e == cudaSuccess) e = alloc_list(r->luma, cap);
    if (e == cudaSuccess) e = alloc_list(r->sub, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_item_sse, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_stats, (size_t)cap * kStatsWords);
    if (e == cudaSuccess) e = dalloc(&r->d_feats, (size_t)cap * DCT_MLP_INPUTS);
    if (e == cudaSuccess) e = dalloc(&r->d_target, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_w, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_h, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_q, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_sse, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_fell, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_thr, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_blo, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_bhi, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_lo, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_hi, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_mid, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_rej, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_rej_sse, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_fsse, cap);
    if (e == cudaSuccess) e = dalloc(&r->d_counter, 1);
    if (e == cudaSuccess) e = halloc(&r->h_thr, cap);
    if (e == cudaSuccess) e = halloc(&r->h_blo, cap);
    if (e == cudaSuccess) e = halloc(&r->h_bhi, cap);
    if (e == cudaSuccess) e = halloc(&r->h_target, cap);
    if (e == cudaSuccess) e = halloc(&r->h_w, cap);
    if (e == cudaSuccess) e = halloc(&r->h_h, cap);
    if (e == cudaSuccess) e = halloc(&r->h_fell, cap);
    if (e == cudaSuccess) e = ws_event_create(&r->ev0);
    if (e == cudaSuccess) e = ws_event_create(&r->ev1);
    if (e != cudaSuccess) {
        release_rc(r);
        return fail(DCT_ERR_ALLOC, std::string("rate-control workspace: ") + cudaGetErrorString(e));
    }
    // table bank: luma then chroma for every quality
    std::vector<QuantSet> bank(kBank);
    for (int c = 0; c < 2; ++c)
        for (int q = 1; q <= 100; ++q) build_tables(q, nullptr, 0, c, bank[c * 100 + q - 1]);
    e = cudaMemcpyAsync(r->d_bank, bank.data(), sizeof(QuantSet) * kBank, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release_rc(r);
        return cuda_fail(e, "table bank upload");
    }
    plan->rc = r;
    return DCT_OK;
}

// Fills a work list with the planes of the given frames (all k planes, or
// plane 0 only) and uploads it.
static dct_status build_list(RcState* r, WorkList& w, const dct_plane* planes, int k, const std::vector<int>& frames,
                             bool luma_only, cudaStream_t s) {
    int cursor = 0, n = 0;
    const int per = luma_only ? 1 : k;
    for (size_t fi = 0; fi < frames.size(); ++fi) {
        const int f = frames[fi];
        w.h_frame[fi] = f;
        for (int p = 0; p < per; ++p) {
            const dct_plane& pl = planes[(size_t)f * k + p];
            PlaneArg& a = w.h_items[n];
            memset(&a, 0, sizeof a);
            fill_plane(a, pl, cursor);
            a.src = pl.data;
            a.src_pitch = pl.pitch;
            a.flags = ((((uintptr_t)pl.data) & 7u) == 0 && (pl.pitch & 7) == 0) ? kVecSrc : 0;
            a.table = p ? 100 : 0;
            a.sse = r->d_item_sse + n;
            a.stats = r->d_stats + (size_t)fi * kStatsWords;
            w.h_tb[n] = a.tile_begin;
            ++n;
        }
    }
    w.h_tb[n] = cursor;
    w.nitems = n;
    w.ntiles = cursor;
    w.nframes = (int)frames.size();
    cudaError_t e = cudaMemcpyAsync(w.d_items, w.h_items, sizeof(PlaneArg) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.d_tb, w.h_tb, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.d_frame, w.h_frame, sizeof(int32_t) * w.nframes, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "work list upload");
}

static inline int blocks_for(int n) { return (n + 127) / 128; }

// 8-step bisection over the frames of list w; results to d_q / d_sse.
static dct_status run_bisection(dct_plan_t plan, RcState* r, WorkList& w, int k, cudaStream_t s) {
    const int n = w.nframes;
    k_bisect_init<<<blocks_for(n), 128, 0, s>>>(r->d_lo, r->d_hi, r->d_rej, n);
    for (int step = 0; step < kBisectSteps; ++step) {
        k_bisect_mid<<<blocks_for(n), 128, 0, s>>>(r->d_lo, r->d_hi, r->d_mid, n);
        k_rc_set_quality<<<blocks_for(w.nitems), 128, 0, s>>>(w.d_items, w.nitems, k, w.d_frame, r->d_mid, nullptr,
                                                              r->d_counter);
        cudaError_t e = batch_launch(kLoadPix | kInverse | kSse, w.d_items, w.d_tb, r->d_bank, w.nitems, w.ntiles,
                                     plan, s, r->d_counter);
        if (e != cudaSuccess) return cuda_fail(e, "bisection pass");
        k_rc_frame_sse<<<blocks_for(n), 128, 0, s>>>(w.d_items, n, k, r->d_fsse);
        if (step + 1 < kBisectSteps)
            k_bisect_update<<<blocks_for(n), 128, 0, s>>>(r->d_fsse, w.d_frame, r->d_thr, r->d_mid, r->d_lo, r->d_hi,
                                                          r->d_rej, r->d_rej_sse, n);
    }
    // after 7 steps lo == hi on 1..100, so the 8th step evaluated Q*
    k_bisect_finish<<<blocks_for(n), 128, 0, s>>>(r->d_fsse, w.d_frame, r->d_mid, r->d_rej, r->d_rej_sse, r->d_blo,
                                                  r->d_bhi, n, r->d_q, r->d_sse);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "bisection launch");
}

static dct_status check_frames(dct_plan_t plan, const dct_plane* planes, int k, int nframes, const float* target) {
    if (!plan) return fail(DCT_ERR_INVALID_ARG, "null plan");
    if (!planes || !target) return fail(DCT_ERR_INVALID_ARG, "null planes or targets");
    if (k != 1 && k != 3) return fail(DCT_ERR_INVALID_ARG, "planes_per_frame must be 1 or 3");
    if (nframes < 1 || (long long)nframes * k > plan->desc.max_batch)
        return fail(DCT_ERR_INVALID_ARG, "nframes * planes_per_frame must be 1..max_batch");
    long long tiles = 0;
    for (long long i = 0; i < (long long)nframes * k; ++i) {
        dct_status st = check_plane(plan, planes[i], "rate-control plane");
        if (st != DCT_OK) return st;
        const long long nblk = (long long)((planes[i].width + 7) / 8) * ((planes[i].height + 7) / 8);
        tiles += (nblk + kTileBlocks - 1) / kTileBlocks;
    }
    if (tiles > (1ll << 30)) return fail(DCT_ERR_INVALID_ARG, "frames too large for one pass (more than 2^30 tiles)");
    for (int f = 0; f < nframes; ++f)
        if (!(target[f] > 0.0f && target[f] < 200.0f)) return fail(DCT_ERR_INVALID_ARG, "targets must be in (0, 200) dB");
    return DCT_OK;
}

// statistics pass + features of every frame's plane 0 into r->d_feats
static dct_status features_pass(dct_plan_t plan, RcState* r, const dct_plane* planes, int k, int nframes,
                                const float* target, cudaStream_t s) {
    std::vector<int> all(nframes);
    for (int f = 0; f < nframes; ++f) all[f] = f;
    dct_status st = build_list(r, r->luma, planes, k, all, true, s);
    if (st != DCT_OK) return st;
    for (int f = 0; f < nframes; ++f) {
        r->h_w[f] = planes[(size_t)f * k].width;
        r->h_h[f] = planes[(size_t)f * k].height;
        r->h_target[f] = target[f];
    }
    cudaError_t e = cudaMemcpyAsync(r->d_w, r->h_w, sizeof(int32_t) * nframes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_h, r->h_h, sizeof(int32_t) * nframes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_target, r->h_target, sizeof(float) * nframes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "feature inputs upload");
    k_rc_clear_stats<<<blocks_for(nframes * kStatsWords), 128, 0, s>>>(r->d_stats, nframes);
    e = batch_launch(kLoadPix | kStats, r->luma.d_items, r->luma.d_tb, r->d_bank, r->luma.nitems, r->luma.ntiles,
                     plan, s);
    if (e == cudaSuccess) e = launch_features(r->d_stats, r->d_w, r->d_h, r->d_target, nframes, r->d_feats, s);
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "statistics pass");
}

}  // namespace dctgb

using namespace dctgb;

namespace dctgb {
void rc_release(dct_plan_t plan) {
    if (plan && plan->rc) {
        release_rc(plan->rc);
        plan->rc = nullptr;
    }
}
}  // namespace dctgb

extern "C" {

dct_status dct_rate_features(dct_plan_t plan, const dct_plane* planes, int planes_per_frame, int nframes,
                             const float* target_host, float* feats_out, dct_stream_t stream) {
    dct_status st = check_frames(plan, planes, planes_per_frame, nframes, target_host);
    if (st != DCT_OK) return st;
    if (!feats_out) return fail(DCT_ERR_INVALID_ARG, "null feats_out");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_rc(plan, s)) != DCT_OK) return st;
    RcState* r = plan->rc;
    if ((st = features_pass(plan, r, planes, planes_per_frame, nframes, target_host, s)) != DCT_OK) return st;
    cudaError_t e = cudaMemcpyAsync(feats_out, r->d_feats, sizeof(float) * (size_t)nframes * DCT_MLP_INPUTS,
                                    cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // staging buffers are reused by the next call
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "features copy");
}

dct_status dct_rate_control(dct_plan_t plan, const dct_plane* planes, int planes_per_frame, int nframes,
                            const float* target_host, const dct_mlp* net, int32_t* quality_host,
                            uint64_t* sse_host, uint8_t* fell_back_host, dct_rc_summary* summary,
                            dct_stream_t stream) {
    const int k = planes_per_frame;
    dct_status st = check_frames(plan, planes, k, nframes, target_host);
    if (st != DCT_OK) return st;
    if (net && (!net->params || !net->feat_mean || !net->feat_std))
        return fail(DCT_ERR_INVALID_ARG, "network pointers are null");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_rc(plan, s)) != DCT_OK) return st;
    RcState* r = plan->rc;

    // thresholds on the integer SSE (float64, on the host)
    std::vector<long long> nsamp(nframes, 0);
    for (int f = 0; f < nframes; ++f) {
        for (int p = 0; p < k; ++p) {
            const dct_plane& pl = planes[(size_t)f * k + p];
            nsamp[f] += (long long)pl.width * pl.height;
        }
        const double n = (double)nsamp[f], t = (double)target_host[f];
        r->h_thr[f] = (unsigned long long)std::floor(65025.0 * n / std::pow(10.0, t / 10.0));
        r->h_blo[f] = (unsigned long long)std::ceil(65025.0 * n / std::pow(10.0, (t + 0.25) / 10.0));
        r->h_bhi[f] = (unsigned long long)std::floor(65025.0 * n / std::pow(10.0, (t - 0.25) / 10.0));
    }
    cudaEventRecord(r->ev0, s);
    cudaError_t e = cudaMemcpyAsync(r->d_thr, r->h_thr, 8 * nframes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_blo, r->h_blo, 8 * nframes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_bhi, r->h_bhi, 8 * nframes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "threshold upload");

    std::vector<int> all(nframes);
    for (int f = 0; f < nframes; ++f) all[f] = f;
    int passes = 0, fell = 0;
    if (net) {
        if ((st = features_pass(plan, r, planes, k, nframes, target_host, s)) != DCT_OK) return st;
        if ((e = launch_mlp_forward(net, r->d_feats, nframes, nullptr, r->d_q, s)) != cudaSuccess)
            return cuda_fail(e, "network launch");
        if ((st = build_list(r, r->all, planes, k, all, false, s)) != DCT_OK) return st;
        k_rc_set_quality<<<blocks_for(r->all.nitems), 128, 0, s>>>(r->all.d_items, r->all.nitems, k, r->all.d_frame,
                                                                   nullptr, r->d_q, r->d_counter);
        e = batch_launch(kLoadPix | kInverse | kSse, r->all.d_items, r->all.d_tb, r->d_bank, r->all.nitems,
                         r->all.ntiles, plan, s, r->d_counter);
        if (e != cudaSuccess) return cuda_fail(e, "verification pass");
        k_rc_frame_sse<<<blocks_for(nframes), 128, 0, s>>>(r->all.d_items, nframes, k, r->d_fsse);
        k_rc_decide<<<blocks_for(nframes), 128, 0, s>>>(r->d_fsse, r->d_blo, r->d_bhi, nframes, r->d_sse, r->d_fell);
        passes += nframes;
        e = cudaMemcpyAsync(r->h_fell, r->d_fell, nframes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "fallback mask");
        std::vector<int> sub;
        for (int f = 0; f < nframes; ++f)
            if (r->h_fell[f]) sub.push_back(f);
        fell = (int)sub.size();
        if (!sub.empty()) {
            if ((st = build_list(r, r->sub, planes, k, sub, false, s)) != DCT_OK) return st;
            if ((st = run_bisection(plan, r, r->sub, k, s)) != DCT_OK) return st;
            passes += kBisectSteps * fell;
        }
    } else {
        if ((st = build_list(r, r->all, planes, k, all, false, s)) != DCT_OK) return st;
        if ((st = run_bisection(plan, r, r->all, k, s)) != DCT_OK) return st;
        cudaMemsetAsync(r->d_fell, 1, nframes, s);
        passes += kBisectSteps * nframes;
        fell = nframes;
    }
    cudaEventRecord(r->ev1, s);
    std::vector<int32_t> q(nframes);
    std::vector<unsigned long long> sse(nframes);
    e = cudaMemcpyAsync(q.data(), r->d_q, 4 * nframes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sse.data(), r->d_sse, 8 * nframes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_fell, r->d_fell, nframes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "result copy");
    int unreachable = 0, within = 0;
    for (int f = 0; f < nframes; ++f) {
        if (quality_host) quality_host[f] = q[f];
        if (sse_host) sse_host[f] = sse[f];
        if (fell_back_host) fell_back_host[f] = r->h_fell[f];
        // a final PSNR outside the band comes from the bisection, which
        // evaluated the qualities on both sides of the band (or stopped at
        // 1 or 100): no quality lands in it while PSNR rises with quality
        if (sse[f] >= r->h_blo[f] && sse[f] <= r->h_bhi[f]) ++within;
        else ++unreachable;
    }
    if (summary) {
        summary->frames = nframes;
        summary->fell_back = fell;
        summary->unreachable = unreachable;
        summary->within_tol = within;
        summary->passes = passes;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r->ev0, r->ev1);
        summary->gpu_ms = ms;
    }
    return DCT_OK;
}

}  // extern "C"
