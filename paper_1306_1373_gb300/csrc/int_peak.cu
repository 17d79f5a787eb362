// Integer issue-rate probe (no counterpart in the paper): the throughput of
// the codec's dominant operation, the CORDIC micro-rotation
// (a, b) <- (a + (b >> i), b - (a >> i)) of Sec. 2.5.2's rotation blocks,
// measured on this GPU in four instruction forms.  The codec is bound by
// integer instruction issue, so this rate (not HBM bandwidth) is the
// roofline its kernels are held against.
//
//   kind 0  shift + add for both halves            (4 instructions; the
//           form of the codec kernels)
//   kind 1  one half as mad.hi.s32, one shift+add  (3 instructions)
//   kind 2  both halves as mad.hi.s32 (the second on ~a, exact:
//           b - (a >> i) = b + ((~a) >> i) + 1 folded as a constant)
//                                                  (2 instructions + 1 not)
//   kind 3  both halves as float32 fused multiply-adds with directed
//           rounding (the forward kernels' form for micro-rotations
//           2..N: on biased values in [2^23, 2^24) they round to exactly
//           a + floor(b / 2^i))                    (2 instructions)
//
// Every thread runs 8 independent micro-rotation chains; the grid fills
// every SM with resident CTAs.  Cycles come from clock64() per CTA, so the
// rate per clock does not depend on the clock the GPU ran at.
#include "host_common.h"

namespace dctgb {

static __constant__ int32_t kPeakMul[8] = {0, 0, 1 << 30, 1 << 29, 1 << 28, 1 << 27, 1 << 26, 1 << 25};

template <int I>
__device__ __forceinline__ int peak_madhi(int acc, int v) {
    int r;
    asm("mad.hi.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(v), "r"(kPeakMul[I]), "r"(acc));
    return r;
}

template <int KIND, int I>
__device__ __forceinline__ void peak_step(int& a, int& b) {
    if constexpr (KIND == 3) {
        constexpr float sc = 1.0f / float(1 << I);
        const float fa = __int_as_float(a), fb = __int_as_float(b);
        b = __float_as_int(__fmaf_ru(fa, -sc, fb));
        a = __float_as_int(__fmaf_rd(fb, sc, fa));
    } else if constexpr (KIND == 0) {
        const int na = a + (b >> I);
        b = b - (a >> I);
        a = na;
    } else if constexpr (KIND == 1) {
        const int na = peak_madhi<I>(a, b);
        b = b - (a >> I);
        a = na;
    } else {
        const int na = peak_madhi<I>(a, b);
        b = peak_madhi<I>(b, ~a);
        a = na;
    }
}

constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 4;

template <int KIND>
__global__ void __launch_bounds__(256) k_int_peak(int iters, int* sink, long long* cycles) {
    int a[kPeakChains], b[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) {
        a[k] = (int)(threadIdx.x * 2654435761u) ^ (k * 40503);
        b[k] = (int)(blockIdx.x * 97u + k * 1013904223u);
        if (KIND == 3) {            // floats of magnitude near 2^23 (finite)
            a[k] = (int)(0x4B000000u + ((unsigned)a[k] & 0xFFFFu));
            b[k] = (int)(0xCB000000u + ((unsigned)b[k] & 0xFFFFu));
        }
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) {
                switch ((u + k) % 5) {      // shifts 2..6, as in a rotation block
                    case 0: peak_step<KIND, 2>(a[k], b[k]); break;
                    case 1: peak_step<KIND, 3>(a[k], b[k]); break;
                    case 2: peak_step<KIND, 4>(a[k], b[k]); break;
                    case 3: peak_step<KIND, 5>(a[k], b[k]); break;
                    default: peak_step<KIND, 6>(a[k], b[k]); break;
                }
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    int acc = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc ^= a[k] + b[k];
    if (acc == 0x7f3a5c11) sink[threadIdx.x] = acc;      // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_int_peak(int kind, int iters, double* ops_per_clk_sm_host, double* tops_host,
                                   float* ms_host, dct_stream_t stream) {
    if (kind < 0 || kind > 3) return fail(DCT_ERR_INVALID_ARG, "kind must be 0, 1, 2 or 3");
    if (iters < 1 || iters > (1 << 24)) return fail(DCT_ERR_INVALID_ARG, "iters must be 1..2^24");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    void (*kp)(int, int*, long long*) =
        kind == 0 ? k_int_peak<0> : (kind == 1 ? k_int_peak<1> : (kind == 2 ? k_int_peak<2> : k_int_peak<3>));
    const int threads = 256;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kp, threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (occ < 1) occ = 1;
    const int grid = sms * occ;
    int* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    dct_status st = DCT_OK;
    std::vector<long long> hc(grid);
    float ms = 0.f;
    if ((e = cudaMalloc(&sink, threads * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&cyc, grid * sizeof(long long))) != cudaSuccess) {
        st = fail(DCT_ERR_ALLOC, std::string("probe buffers: ") + cudaGetErrorString(e));
        goto done;
    }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        st = cuda_fail(e, "cudaEventCreate");
        goto done;
    }
    kp<<<grid, threads, 0, s>>>(iters / 8 + 1, sink, cyc);           // warm-up
    cudaEventRecord(e0, s);
    kp<<<grid, threads, 0, s>>>(iters, sink, cyc);
    cudaEventRecord(e1, s);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = cuda_fail(e, "probe launch");
        goto done;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if ((e = cudaMemcpy(hc.data(), cyc, grid * sizeof(long long), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        st = cuda_fail(e, "probe readback");
        goto done;
    }
    {
        long long span = 0;
        for (long long c : hc) span = c > span ? c : span;
        // 4 algorithmic integer operations (2 floor shifts, 2 adds) per micro-rotation
        const double ops = 4.0 * kPeakChains * kPeakUnroll * (double)iters * threads * grid;
        if (ops_per_clk_sm_host) *ops_per_clk_sm_host = ops / sms / (double)(span > 0 ? span : 1);
        if (tops_host) *tops_host = ops / (ms * 1e-3) / 1e12;
        if (ms_host) *ms_host = ms;
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    return st;
}
