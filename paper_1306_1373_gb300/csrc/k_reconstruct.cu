// Inverse-path kernels: coefficient load, dequantiser, transposed
// Cordic-Loeffler graph, descale, store (Sec. 3.2), with the SSE of Eq. 24
// against a reference fused in; two lanes per 8x8 block.
#include "kernels_pair.cuh"

namespace dctgb {

cudaError_t launch_reconstruct(const DirectArgs& a, bool sse, int num_sms, int threads, cudaStream_t s) {
    if (sse) return launch_codec_pair<kLoadCoef | kInverse | kStoreRecon | kSse>(a, num_sms, threads, s);
    return launch_codec_pair<kLoadCoef | kInverse | kStoreRecon>(a, num_sms, threads, s);
}

}  // namespace dctgb
