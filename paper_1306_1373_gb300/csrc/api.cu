// C ABI of the codec: spec query, tables, plans, compress / reconstruct /
// fused / PSNR entry points.  Every argument is checked here before anything
// is enqueued; the kernels themselves never trap.
#include <atomic>
#include <cmath>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>

#include "host_common.h"

namespace dctgb {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

dct_status fail(dct_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

dct_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    set_error(m);
    return e == cudaErrorMemoryAllocation ? DCT_ERR_ALLOC : DCT_ERR_CUDA;
}

// Fault injection of the workspace allocations: 0 = off; n > 0 = the n-th
// attempt from now fails (and disarms the hook).
static std::atomic<int> g_fail_at{0};
static std::atomic<long long> g_alloc_attempts{0};

static bool injected_failure() {
    g_alloc_attempts.fetch_add(1);
    int n = g_fail_at.load();
    while (n > 0) {
        if (g_fail_at.compare_exchange_weak(n, n - 1)) return n == 1;
    }
    return false;
}

cudaError_t ws_malloc(void** p, size_t bytes) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t ws_malloc_host(void** p, size_t bytes) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, bytes);
}

cudaError_t ws_stream_create(cudaStream_t* s) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}

cudaError_t ws_event_create(cudaEvent_t* e) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaEventCreate(e);
}

// ITU-T T.81 Annex K, Table K.1 (luminance) and Table K.2 (chrominance),
// natural order.
static const uint16_t kLumaBase[64] = {
    16, 11, 10, 16, 24, 40, 51, 61,      12, 12, 14, 19, 26, 58, 60, 55,
    14, 13, 16, 24, 40, 57, 69, 56,      14, 17, 22, 29, 51, 87, 80, 62,
    18, 22, 37, 56, 68, 109, 103, 77,    24, 35, 55, 64, 81, 104, 113, 92,
    49, 64, 78, 87, 103, 121, 120, 101,  72, 92, 95, 98, 112, 100, 103, 99};
static const uint16_t kChromaBase[64] = {
    17, 18, 24, 47, 99, 99, 99, 99,  18, 21, 26, 66, 99, 99, 99, 99,
    24, 26, 56, 99, 99, 99, 99, 99,  47, 66, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,  99, 99, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99,  99, 99, 99, 99, 99, 99, 99, 99};

// Per-output gain of one pass relative to sqrt(8) * orthonormal DCT:
// [1, K, K/sqrt2, K/sqrt2, 1, K/sqrt2, K/sqrt2, K], K = prod sqrt(1 + 4^-i).
static void pass_gains(double g[8]) {
    double k = 1.0;
    for (int i = 1; i <= kN; ++i) k *= std::sqrt(1.0 + std::ldexp(1.0, -2 * i));
    const double kr = k / std::sqrt(2.0);
    const double v[8] = {1.0, k, kr, kr, 1.0, kr, kr, k};
    for (int i = 0; i < 8; ++i) g[i] = v[i];
}

dct_status build_tables(int quality, const uint16_t* qtab, int qtab_entries, int chroma, QuantSet& out) {
    int q[64];
    if (quality < 0 || quality > 100) return fail(DCT_ERR_INVALID_ARG, "quality must be 0..100");
    if (quality == 0) {
        if (!qtab) return fail(DCT_ERR_INVALID_ARG, "quality 0 needs qtab_host");
        if (qtab_entries != 64 && qtab_entries != 128)
            return fail(DCT_ERR_INVALID_ARG, "qtab_entries must be 64 or 128");
        const uint16_t* t = (chroma && qtab_entries == 128) ? qtab + 64 : qtab;
        for (int i = 0; i < 64; ++i) {
            if (t[i] < 1 || t[i] > 255) return fail(DCT_ERR_INVALID_ARG, "quant table entries must be 1..255");
            q[i] = t[i];
        }
    } else {
        // IJG scaling: s = 5000/q below 50, else 200 - 2q; Q = clamp((b s + 50) / 100, 1, 255)
        const int s = quality < 50 ? 5000 / quality : 200 - 2 * quality;
        const uint16_t* base = chroma ? kChromaBase : kLumaBase;
        for (int i = 0; i < 64; ++i) {
            int v = ((int)base[i] * s + 50) / 100;
            q[i] = v < 1 ? 1 : (v > 255 ? 255 : v);
        }
    }
    double g[8];
    pass_gains(g);
    for (int u = 0; u < 8; ++u) {
        for (int v = 0; v < 8; ++v) {
            const int i = u * 8 + v;
            const double gg = g[u] * g[v];
            // M = rint(2^32 / (8 * 2^P * gg * Q)); the power of two is exact
            const double den = gg * (double)q[i];
            const double m = std::nearbyint(std::ldexp(1.0, kQuantShift - 3 - kP) / den);
            const double w = std::nearbyint(std::ldexp(1.0, kR) / gg);
            out.Q[i] = q[i];
            out.M[i] = (uint32_t)m;
            out.W[i] = (int32_t)w;
            out.QW[i] = q[i] * (int32_t)w;
            // the kernels quantise the non-tie entries without the sign term,
            // which is exact only while M has at most 11 trailing zero bits
            // (tie_entry); every Q in 1..255 satisfies this
            if (!tie_entry(u, v) && (out.M[i] & kTieFreeBits) == 0)
                return fail(DCT_ERR_UNSUPPORTED, "quantiser multiplier outside the tie-free range");
        }
    }
    return DCT_OK;
}

dct_status check_plane(const dct_plan_s* plan, const dct_plane& p, const char* what) {
    char buf[160];
    if (!p.data) {
        snprintf(buf, sizeof buf, "%s: null data pointer", what);
        return fail(DCT_ERR_INVALID_ARG, buf);
    }
    if (p.width < 1 || p.height < 1 || p.width > plan->desc.max_width || p.height > plan->desc.max_height) {
        snprintf(buf, sizeof buf, "%s: size %dx%d outside 1..%dx%d", what, p.width, p.height,
                 plan->desc.max_width, plan->desc.max_height);
        return fail(DCT_ERR_INVALID_ARG, buf);
    }
    if (p.pitch < p.width) {
        snprintf(buf, sizeof buf, "%s: pitch %d < width %d", what, p.pitch, p.width);
        return fail(DCT_ERR_INVALID_ARG, buf);
    }
    return DCT_OK;
}

static int64_t plane_blocks(const dct_plane& p) {
    return (int64_t)((p.width + 7) / 8) * (int64_t)((p.height + 7) / 8);
}

void fill_plane(PlaneArg& a, const dct_plane& p, int& tile_cursor) {
    a.width = p.width;
    a.height = p.height;
    a.nbx = (p.width + 7) / 8;
    a.nblk = (int)plane_blocks(p);
    a.tile_begin = tile_cursor;
    tile_cursor += (a.nblk + kTileBlocks - 1) / kTileBlocks;
}

static bool aligned8(const void* ptr, int pitch) {
    return (((uintptr_t)ptr) & 7u) == 0 && (pitch & 7) == 0;
}

}  // namespace dctgb

using namespace dctgb;

extern "C" {

const char* dct_last_error(void) { return g_last_error.c_str(); }

dct_status dct_debug_fail_alloc(int nth, int64_t* attempts_host) {
    if (nth < 0) return fail(DCT_ERR_INVALID_ARG, "nth must be >= 0");
    g_fail_at.store(nth);
    if (attempts_host) *attempts_host = g_alloc_attempts.load();
    return DCT_OK;
}

dct_status dct_spec_query(dct_spec_info* out) {
    if (!out) return fail(DCT_ERR_INVALID_ARG, "out is null");
    out->P = kP;
    out->N = kN;
    out->R = kR;
    out->quant_shift = kQuantShift;
    out->dequant_clamp = kDequantClamp;
    out->psnr_max = kPsnrMax;
    out->sigma_odd_upper = kSigOddUpper;
    out->sigma_odd_lower = kSigOddLower;
    out->sigma_even = kSigEven;
    out->stats_words = kStatsWords;
    return DCT_OK;
}

dct_status dct_tables(int quality, const uint16_t* qtab_host, int qtab_entries, int chroma,
                      uint16_t* Q_host, uint32_t* M_host, int32_t* W_host) {
    QuantSet t;
    dct_status st = build_tables(quality, qtab_host, qtab_entries, chroma, t);
    if (st != DCT_OK) return st;
    for (int i = 0; i < 64; ++i) {
        if (Q_host) Q_host[i] = (uint16_t)t.Q[i];
        if (M_host) M_host[i] = t.M[i];
        if (W_host) W_host[i] = t.W[i];
    }
    return DCT_OK;
}

double dct_psnr_from_sse(uint64_t sse, int64_t n_samples, double max_value) {
    const double mx = max_value > 0.0 ? max_value : (double)kPsnrMax;
    if (sse == 0) return INFINITY;
    return 10.0 * std::log10(mx * mx * (double)n_samples / (double)sse);
}

dct_status dct_psnr_from_sse_list(const uint64_t* sse_host, const int64_t* samples_host, int n, double max_value,
                                  double* psnr_host) {
    if (!sse_host || !samples_host || !psnr_host) return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (n < 1) return fail(DCT_ERR_INVALID_ARG, "n must be >= 1");
    uint64_t tot = 0;
    int64_t ns = 0;
    for (int i = 0; i < n; ++i) {
        if (samples_host[i] < 1) return fail(DCT_ERR_INVALID_ARG, "sample counts must be >= 1");
        psnr_host[i] = dct_psnr_from_sse(sse_host[i], samples_host[i], max_value);
        tot += sse_host[i];
        ns += samples_host[i];
    }
    psnr_host[n] = dct_psnr_from_sse(tot, ns, max_value);
    return DCT_OK;
}

dct_status dct_plan_create(dct_plan_t* out, const dct_plan_desc* desc, dct_stream_t stream) {
    (void)stream;
    if (!out || !desc) return fail(DCT_ERR_INVALID_ARG, "null out or desc");
    *out = nullptr;
    if (desc->max_width < 1 || desc->max_height < 1 || desc->max_width > (1 << 16) || desc->max_height > (1 << 16))
        return fail(DCT_ERR_INVALID_ARG, "max_width/max_height must be 1..65536");
    if ((int64_t)desc->max_width * desc->max_height > (int64_t)1 << 31)
        return fail(DCT_ERR_INVALID_ARG, "max_width * max_height must stay below 2^31 samples");
    if (desc->layout != DCT_LAYOUT_GRAY8 && desc->layout != DCT_LAYOUT_YUV420)
        return fail(DCT_ERR_INVALID_ARG, "unknown layout");
    if (desc->max_batch < 0 || desc->max_batch > (1 << 20)) return fail(DCT_ERR_INVALID_ARG, "max_batch must be 0..2^20");
    if (desc->flags != 0) return fail(DCT_ERR_INVALID_ARG, "flags must be 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    dct_plan_s* p = new (std::nothrow) dct_plan_s();
    if (!p) return fail(DCT_ERR_ALLOC, "host allocation failed");
    p->desc = *desc;
    p->device = dev;
    p->num_sms = sms;
    p->shape = default_shape();
    p->batch = nullptr;
    p->rc = nullptr;
    *out = p;
    return DCT_OK;
}

dct_status dct_plan_destroy(dct_plan_t plan) {
    if (!plan) return fail(DCT_ERR_INVALID_ARG, "null plan");
    cudaDeviceSynchronize();
    batch_release(plan);
    rc_release(plan);
    delete plan;
    return DCT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// shared argument handling for the plane calls
// ---------------------------------------------------------------------------

static dct_status prepare_planes(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                                 const uint16_t* qtab, int qtab_entries, DirectArgs& a) {
    if (!plan) return fail(DCT_ERR_INVALID_ARG, "null plan");
    if (!planes) return fail(DCT_ERR_INVALID_ARG, "null planes");
    if (nplanes < 1 || nplanes > kMaxPlanes) return fail(DCT_ERR_INVALID_ARG, "nplanes must be 1..4");
    memset(&a, 0, sizeof a);
    dct_status st = build_tables(quality, qtab, qtab_entries, 0, a.tabs[0]);
    if (st != DCT_OK) return st;
    const bool yuv = plan->desc.layout == DCT_LAYOUT_YUV420;
    st = build_tables(quality, qtab, qtab_entries, yuv ? 1 : 0, a.tabs[1]);
    if (st != DCT_OK) return st;
    int cursor = 0;
    for (int i = 0; i < nplanes; ++i) {
        st = check_plane(plan, planes[i], "plane");
        if (st != DCT_OK) return st;
        fill_plane(a.p[i], planes[i], cursor);
        a.p[i].table = (yuv && i > 0) ? 1 : 0;
    }
    a.nplanes = nplanes;
    a.ntiles = cursor;
    return DCT_OK;
}

static dct_status set_coef_pointers(DirectArgs& a, int16_t* coeffs) {
    if (((uintptr_t)coeffs) & 15u) return fail(DCT_ERR_INVALID_ARG, "coeffs must be 16-byte aligned");
    size_t off = 0;
    for (int i = 0; i < a.nplanes; ++i) {
        a.p[i].coef = coeffs + off;
        off += (size_t)a.p[i].nblk * 64;
    }
    return DCT_OK;
}

extern "C" {

dct_status dct_compress(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                        const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                        uint64_t* stats_out, dct_stream_t stream) {
    DirectArgs a;
    dct_status st = prepare_planes(plan, planes, nplanes, quality, qtab_host, qtab_entries, a);
    if (st != DCT_OK) return st;
    if (!coeffs) return fail(DCT_ERR_INVALID_ARG, "null coeffs");
    if ((st = set_coef_pointers(a, coeffs)) != DCT_OK) return st;
    if (stats_out && (((uintptr_t)stats_out) & 7u)) return fail(DCT_ERR_INVALID_ARG, "stats_out must be 8-byte aligned");
    for (int i = 0; i < nplanes; ++i) {
        a.p[i].src = planes[i].data;
        a.p[i].src_pitch = planes[i].pitch;
        a.p[i].flags = aligned8(planes[i].data, planes[i].pitch) ? kVecSrc : 0;
        a.p[i].stats = stats_out ? reinterpret_cast<unsigned long long*>(stats_out) + (size_t)i * kStatsWords : nullptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = kDirectThreads;
    cudaError_t e;
    if (stats_out) {
        k_init_acc<<<1, 128, 0, s>>>(a, 0, 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "init launch");
    }
    e = launch_compress(a, stats_out != nullptr, plan->num_sms, threads, s);
    if (e != cudaSuccess) return cuda_fail(e, "compress launch");
    return DCT_OK;
}

dct_status dct_reconstruct(dct_plan_t plan, const int16_t* coeffs, const dct_plane* out_planes, int nplanes,
                           int quality, const uint16_t* qtab_host, int qtab_entries,
                           const dct_plane* ref_planes, uint64_t* sse_out, dct_stream_t stream) {
    DirectArgs a;
    dct_status st = prepare_planes(plan, out_planes, nplanes, quality, qtab_host, qtab_entries, a);
    if (st != DCT_OK) return st;
    if (!coeffs) return fail(DCT_ERR_INVALID_ARG, "null coeffs");
    if ((st = set_coef_pointers(a, const_cast<int16_t*>(coeffs))) != DCT_OK) return st;
    if ((ref_planes != nullptr) != (sse_out != nullptr))
        return fail(DCT_ERR_INVALID_ARG, "ref_planes and sse_out go together");
    if (sse_out && (((uintptr_t)sse_out) & 7u)) return fail(DCT_ERR_INVALID_ARG, "sse_out must be 8-byte aligned");
    for (int i = 0; i < nplanes; ++i) {
        a.p[i].dst = out_planes[i].data;
        a.p[i].dst_pitch = out_planes[i].pitch;
        int fl = aligned8(out_planes[i].data, out_planes[i].pitch) ? kVecDst : 0;
        if (ref_planes) {
            st = check_plane(plan, ref_planes[i], "ref plane");
            if (st != DCT_OK) return st;
            if (ref_planes[i].width != out_planes[i].width || ref_planes[i].height != out_planes[i].height)
                return fail(DCT_ERR_INVALID_ARG, "ref plane size differs from output plane");
            a.p[i].ref = ref_planes[i].data;
            a.p[i].ref_pitch = ref_planes[i].pitch;
            if (aligned8(ref_planes[i].data, ref_planes[i].pitch)) fl |= kVecRef;
            a.p[i].sse = reinterpret_cast<unsigned long long*>(sse_out) + i;
        }
        a.p[i].flags = fl;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = kDirectThreads;
    cudaError_t e;
    if (sse_out) {
        k_init_acc<<<1, 32, 0, s>>>(a, 1, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "init launch");
    }
    e = launch_reconstruct(a, sse_out != nullptr, plan->num_sms, threads, s);
    if (e != cudaSuccess) return cuda_fail(e, "reconstruct launch");
    return DCT_OK;
}

dct_status dct_codec_fused(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                           const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                           const dct_plane* recon_planes, uint64_t* sse_out, dct_stream_t stream) {
    DirectArgs a;
    dct_status st = prepare_planes(plan, planes, nplanes, quality, qtab_host, qtab_entries, a);
    if (st != DCT_OK) return st;
    if (!sse_out) return fail(DCT_ERR_INVALID_ARG, "sse_out is required");
    if (((uintptr_t)sse_out) & 7u) return fail(DCT_ERR_INVALID_ARG, "sse_out must be 8-byte aligned");
    if (coeffs && (st = set_coef_pointers(a, coeffs)) != DCT_OK) return st;
    for (int i = 0; i < nplanes; ++i) {
        a.p[i].src = planes[i].data;
        a.p[i].src_pitch = planes[i].pitch;
        int fl = aligned8(planes[i].data, planes[i].pitch) ? kVecSrc : 0;
        if (recon_planes) {
            st = check_plane(plan, recon_planes[i], "recon plane");
            if (st != DCT_OK) return st;
            if (recon_planes[i].width != planes[i].width || recon_planes[i].height != planes[i].height)
                return fail(DCT_ERR_INVALID_ARG, "recon plane size differs from input plane");
            a.p[i].dst = recon_planes[i].data;
            a.p[i].dst_pitch = recon_planes[i].pitch;
            if (aligned8(recon_planes[i].data, recon_planes[i].pitch)) fl |= kVecDst;
        }
        a.p[i].flags = fl;
        a.p[i].sse = reinterpret_cast<unsigned long long*>(sse_out) + i;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = kDirectThreads;
    k_init_acc<<<1, 32, 0, s>>>(a, 1, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    e = launch_fused(a, coeffs != nullptr, recon_planes != nullptr, plan->num_sms, threads, s);
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return DCT_OK;
}

}  // extern "C"
