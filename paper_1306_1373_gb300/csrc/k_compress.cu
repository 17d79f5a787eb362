// Forward-path kernels: level shift, 2-D Cordic-Loeffler DCT, quantiser,
// coefficient store (Sec. 2.5.2, Sec. 3.2): one lane per 8x8 block, with
// the optional statistics pass.
#include "kernels_pair.cuh"

namespace dctgb {

template <unsigned MODE>
static cudaError_t launch_mode(const DirectArgs& a, int num_sms, int threads, cudaStream_t s) {
    const size_t smem = codec_smem_bytes(threads);
    cudaError_t e = cudaFuncSetAttribute(k_codec<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_codec<MODE>, threads, smem);
    if (e != cudaSuccess) return e;
    k_codec<MODE><<<persistent_grid(a.ntiles, threads, num_sms, occ), threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_compress(const DirectArgs& a, bool stats, int num_sms, int threads, cudaStream_t s) {
    if (stats) return launch_mode<kLoadPix | kStoreCoef | kStats>(a, num_sms, threads, s);
    // one lane per block: its forward pass runs the float micro-rotations
    // (measured 849 against 803 GPix/s for the two-lane kernel on the
    // benchmark planes)
    return launch_mode<kLoadPix | kStoreCoef>(a, num_sms, threads, s);
}

__global__ void k_init_acc(DirectArgs args, int do_sse, int do_stats) {
    for (int pl = 0; pl < args.nplanes; ++pl) {
        if (do_sse && threadIdx.x == 0) *args.p[pl].sse = 0ull;
        if (do_stats)
            for (int w = threadIdx.x; w < kStatsWords; w += blockDim.x)
                args.p[pl].stats[w] = (w == kStMin) ? ~0ull : 0ull;
    }
}

}  // namespace dctgb
