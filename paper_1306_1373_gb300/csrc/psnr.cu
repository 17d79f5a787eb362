// SSE between two sets of planes (the sum in Eq. 24) and PSNR (Eq. 23).
#include <cmath>
#include <cstring>

#include "host_common.h"

namespace dctgb {

struct SseArgs {
    const uint8_t* a[kMaxPlanes];
    const uint8_t* b[kMaxPlanes];
    int32_t pa[kMaxPlanes], pb[kMaxPlanes], w[kMaxPlanes];
    int32_t vec16[kMaxPlanes];
    int32_t row_begin[kMaxPlanes + 1];
    unsigned long long* sse;
    int32_t nplanes;
};

__device__ __forceinline__ unsigned sq_diff_bytes(uint32_t x, uint32_t y) {
    unsigned e = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int d = (int)((x >> (8 * j)) & 0xFFu) - (int)((y >> (8 * j)) & 0xFFu);
        e += d * d;
    }
    return e;
}

// One warp per row, grid-stride over the rows of all planes.  Rows of planes
// whose base and pitch are 16-byte aligned are read 16 bytes per lane; the
// last (w mod 16) bytes, and unaligned planes, bytewise.
__global__ void __launch_bounds__(256) k_sse(const __grid_constant__ SseArgs args) {
    __shared__ unsigned long long acc[kMaxPlanes];
    if (threadIdx.x < kMaxPlanes) acc[threadIdx.x] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int total_rows = args.row_begin[args.nplanes];
    for (int row = blockIdx.x * warps + (threadIdx.x >> 5); row < total_rows; row += gridDim.x * warps) {
        int pl = 0;
        while (pl + 1 < args.nplanes && row >= args.row_begin[pl + 1]) ++pl;
        const int y = row - args.row_begin[pl];
        const uint8_t* ra = args.a[pl] + (size_t)y * args.pa[pl];
        const uint8_t* rb = args.b[pl] + (size_t)y * args.pb[pl];
        const int w = args.w[pl];
        unsigned e = 0;
        int tail = 0;
        if (args.vec16[pl]) {
            const int chunks = w >> 4;
            for (int c = lane; c < chunks; c += 32) {
                const uint4 va = __ldg(reinterpret_cast<const uint4*>(ra) + c);
                const uint4 vb = __ldg(reinterpret_cast<const uint4*>(rb) + c);
                e += sq_diff_bytes(va.x, vb.x) + sq_diff_bytes(va.y, vb.y) +
                     sq_diff_bytes(va.z, vb.z) + sq_diff_bytes(va.w, vb.w);
            }
            tail = chunks << 4;
        }
        for (int c = tail + lane; c < w; c += 32) {
            const int d = (int)ra[c] - (int)rb[c];
            e += d * d;
        }
        const unsigned tot = __reduce_add_sync(0xffffffffu, e);
        if (lane == 0 && tot) atomicAdd(&acc[pl], (unsigned long long)tot);
    }
    __syncthreads();
    if (threadIdx.x < args.nplanes && acc[threadIdx.x]) atomicAdd(args.sse + threadIdx.x, acc[threadIdx.x]);
}

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_psnr(dct_plan_t plan, const dct_plane* a, const dct_plane* b, int nplanes,
                               uint64_t* sse_out, double* psnr_host, double max_value, dct_stream_t stream) {
    if (!plan) return fail(DCT_ERR_INVALID_ARG, "null plan");
    if (!a || !b || !sse_out) return fail(DCT_ERR_INVALID_ARG, "null planes or sse_out");
    if (nplanes < 1 || nplanes > kMaxPlanes) return fail(DCT_ERR_INVALID_ARG, "nplanes must be 1..4");
    if (((uintptr_t)sse_out) & 7u) return fail(DCT_ERR_INVALID_ARG, "sse_out must be 8-byte aligned");
    if (max_value < 0.0) return fail(DCT_ERR_INVALID_ARG, "max_value must be >= 0");
    SseArgs args;
    memset(&args, 0, sizeof args);
    int rows = 0;
    int64_t n_samples[kMaxPlanes];
    for (int i = 0; i < nplanes; ++i) {
        dct_status st = check_plane(plan, a[i], "plane a");
        if (st != DCT_OK) return st;
        st = check_plane(plan, b[i], "plane b");
        if (st != DCT_OK) return st;
        if (a[i].width != b[i].width || a[i].height != b[i].height)
            return fail(DCT_ERR_INVALID_ARG, "plane sizes differ");
        args.a[i] = a[i].data;
        args.b[i] = b[i].data;
        args.pa[i] = a[i].pitch;
        args.pb[i] = b[i].pitch;
        args.w[i] = a[i].width;
        args.vec16[i] = ((((uintptr_t)a[i].data) | ((uintptr_t)b[i].data)) & 15u) == 0 &&
                        ((a[i].pitch | b[i].pitch) & 15) == 0;
        args.row_begin[i] = rows;
        rows += a[i].height;
        n_samples[i] = (int64_t)a[i].width * a[i].height;
    }
    args.row_begin[nplanes] = rows;
    args.sse = reinterpret_cast<unsigned long long*>(sse_out);
    args.nplanes = nplanes;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(sse_out, 0, sizeof(uint64_t) * nplanes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const int threads = 256;
    int grid = (rows + 7) / 8;
    const int cap = plan->num_sms * 8;
    if (grid > cap) grid = cap;
    k_sse<<<grid, threads, 0, s>>>(args);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sse launch");
    if (psnr_host) {
        uint64_t h[kMaxPlanes];
        e = cudaMemcpyAsync(h, sse_out, sizeof(uint64_t) * nplanes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        uint64_t tot = 0;
        int64_t n = 0;
        for (int i = 0; i < nplanes; ++i) {
            psnr_host[i] = dct_psnr_from_sse(h[i], n_samples[i], max_value);
            tot += h[i];
            n += n_samples[i];
        }
        psnr_host[nplanes] = dct_psnr_from_sse(tot, n, max_value);
    }
    return DCT_OK;
}
