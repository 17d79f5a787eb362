// Fused kernels: the whole Sec. 3.2 pipeline (transform, quantiser,
// dequantiser, inverse) and the SSE of Eq. 24 in one pass over the samples,
// two lanes per 8x8 block (kernels_pair.cuh).
#include "kernels_pair.cuh"

namespace dctgb {

cudaError_t launch_fused(const DirectArgs& a, bool coef, bool recon, int num_sms, int threads, cudaStream_t s) {
    constexpr unsigned base = kLoadPix | kInverse | kSse;
    if (coef && recon) return launch_codec_pair<base | kStoreCoef | kStoreRecon>(a, num_sms, threads, s);
    if (coef) return launch_codec_pair<base | kStoreCoef>(a, num_sms, threads, s);
    if (recon) return launch_codec_pair<base | kStoreRecon>(a, num_sms, threads, s);
    return launch_codec_pair<base>(a, num_sms, threads, s);
}

}  // namespace dctgb
