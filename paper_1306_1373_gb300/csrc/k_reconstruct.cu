// Inverse-path kernels: coefficient load, dequantiser, transposed
// Cordic-Loeffler graph, descale, store (Sec. 3.2), with the SSE of Eq. 24
// against a reference fused in.
#include "kernels.cuh"

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

cudaError_t launch_reconstruct(const DirectArgs& a, bool sse, int num_sms, int threads, cudaStream_t s) {
    if (sse) return launch_mode<kLoadCoef | kInverse | kStoreRecon | kSse>(a, num_sms, threads, s);
    return launch_mode<kLoadCoef | kInverse | kStoreRecon>(a, num_sms, threads, s);
}

}  // namespace dctgb
