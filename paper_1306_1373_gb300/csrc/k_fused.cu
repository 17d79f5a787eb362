// Fused kernels: the whole Sec. 3.2 pipeline (transform, quantiser,
// dequantiser, inverse) and the SSE of Eq. 24 in one pass over the samples.
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

cudaError_t launch_fused(const DirectArgs& a, bool coef, bool recon, int num_sms, int threads, cudaStream_t s) {
    constexpr unsigned base = kLoadPix | kInverse | kSse;
    if (coef && recon) return launch_mode<base | kStoreCoef | kStoreRecon>(a, num_sms, threads, s);
    if (coef) return launch_mode<base | kStoreCoef>(a, num_sms, threads, s);
    if (recon) return launch_mode<base | kStoreRecon>(a, num_sms, threads, s);
    return launch_mode<base>(a, num_sms, threads, s);
}

}  // namespace dctgb
