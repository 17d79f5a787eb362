// Learned rate controller, network side: the 80 features, input
// normalisation, forward pass, back-propagation with deterministic
// (fixed-order) minibatch sums, and Adam.  The network is tiny (9409
// parameters), so it runs on plain FMA units: one thread per sample for
// inference, one warp per minibatch row for the training forward and delta
// pass, one thread per parameter for the gradient sums and the update.
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "host_common.h"

namespace dctgb {

constexpr int kIn = DCT_MLP_INPUTS, kHid = DCT_MLP_HIDDEN, kParams = DCT_MLP_PARAMS;
constexpr int oW1 = 0, oB1 = kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid;
static_assert(oB3 + 1 == kParams, "parameter layout");

// per-sample cache (floats): xn[80] a1[64] h1[64] a2[64] h2[64] y dz da2[64] da1[64]
constexpr int cXn = 0, cA1 = cXn + kIn, cH1 = cA1 + kHid, cA2 = cH1 + kHid, cH2 = cA2 + kHid, cY = cH2 + kHid,
              cDz = cY + 1, cDa2 = cDz + 1, cDa1 = cDa2 + kHid, kCache = ((cDa1 + kHid + 3) / 4) * 4;

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float a) {
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}
__device__ __forceinline__ float act(float h, int bf16) {
    return bf16 ? __bfloat162float(__float2bfloat16_rn(h)) : h;
}

// Forward pass of one sample; fills the cache when c != nullptr.
__device__ float forward_sample(const float* __restrict__ P, const float* __restrict__ x,
                                const float* __restrict__ mean, const float* __restrict__ stdv, int bf16,
                                float* __restrict__ c) {
    float xn[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        xn[i] = (x[i] - mean[i]) / stdv[i];
        if (c) c[cXn + i] = xn[i];
    }
    float h1[kHid];
    for (int j = 0; j < kHid; ++j) {
        float a = P[oB1 + j];
        const float* w = P + oW1 + j * kIn;
#pragma unroll
        for (int i = 0; i < kIn; ++i) a = fmaf(w[i], xn[i], a);
        h1[j] = act(gelu(a), bf16);
        if (c) {
            c[cA1 + j] = a;
            c[cH1 + j] = h1[j];
        }
    }
    float z = P[oB3];
    for (int j = 0; j < kHid; ++j) {
        float a = P[oB2 + j];
        const float* w = P + oW2 + j * kHid;
#pragma unroll
        for (int i = 0; i < kHid; ++i) a = fmaf(w[i], h1[i], a);
        const float h = act(gelu(a), bf16);
        if (c) {
            c[cA2 + j] = a;
            c[cH2 + j] = h;
        }
        z = fmaf(P[oW3 + j], h, z);
    }
    const float y = 1.0f / (1.0f + expf(-z));
    if (c) c[cY] = y;
    return y;
}

__global__ void k_mlp_forward(const float* __restrict__ P, const float* __restrict__ feats,
                              const float* __restrict__ mean, const float* __restrict__ stdv, int bf16, int n,
                              float* __restrict__ y_out, int* __restrict__ q_out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float y = forward_sample(P, feats + (size_t)s * kIn, mean, stdv, bf16, nullptr);
    if (y_out) y_out[s] = y;
    if (q_out) {
        const float q = rintf(1.0f + 99.0f * y);
        q_out[s] = (int)fminf(100.0f, fmaxf(1.0f, q));
    }
}

// forward + output delta + hidden deltas of one minibatch row per warp:
// lane l owns hidden units l and l + 32 of both layers; every sum runs over
// its inputs in ascending order as forward_sample's does (the inputs a lane
// does not hold come by shuffle), so the cache holds the same values.
__global__ void k_mlp_delta(const float* __restrict__ P, const float* __restrict__ feats,
                            const float* __restrict__ labels, const int* __restrict__ index,
                            const float* __restrict__ mean, const float* __restrict__ stdv, int bf16, int batch,
                            float* __restrict__ cache) {
    const int lane = threadIdx.x & 31;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= batch) return;                                   // warp-uniform
    const int s = index[b];
    float* c = cache + (size_t)b * kCache;
    const float* x = feats + (size_t)s * kIn;
    float xn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = lane + 32 * k;
        xn[k] = i < kIn ? (x[i] - mean[i]) / stdv[i] : 0.0f;
        if (i < kIn) c[cXn + i] = xn[k];
    }
    // layer 1
    float a1[2], h1[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) a1[k] = P[oB1 + lane + 32 * k];
    for (int i = 0; i < kIn; ++i) {
        const float v = __shfl_sync(0xffffffffu, xn[i >> 5], i & 31);
#pragma unroll
        for (int k = 0; k < 2; ++k) a1[k] = fmaf(P[oW1 + (lane + 32 * k) * kIn + i], v, a1[k]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        h1[k] = act(gelu(a1[k]), bf16);
        c[cA1 + lane + 32 * k] = a1[k];
        c[cH1 + lane + 32 * k] = h1[k];
    }
    // layer 2
    float a2[2], h2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) a2[k] = P[oB2 + lane + 32 * k];
    for (int i = 0; i < kHid; ++i) {
        const float v = __shfl_sync(0xffffffffu, h1[i >> 5], i & 31);
#pragma unroll
        for (int k = 0; k < 2; ++k) a2[k] = fmaf(P[oW2 + (lane + 32 * k) * kHid + i], v, a2[k]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        h2[k] = act(gelu(a2[k]), bf16);
        c[cA2 + lane + 32 * k] = a2[k];
        c[cH2 + lane + 32 * k] = h2[k];
    }
    // output, in the same order on every lane
    float z = P[oB3];
    for (int j = 0; j < kHid; ++j) z = fmaf(P[oW3 + j], __shfl_sync(0xffffffffu, h2[j >> 5], j & 31), z);
    const float y = 1.0f / (1.0f + expf(-z));
    const float dz = 2.0f * (y - labels[s]) / (float)batch * y * (1.0f - y);
    if (lane == 0) {
        c[cY] = y;
        c[cDz] = dz;
    }
    float da2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        da2[k] = dz * P[oW3 + lane + 32 * k] * gelu_grad(a2[k]);
        c[cDa2 + lane + 32 * k] = da2[k];
    }
    float s2[2] = {0.0f, 0.0f};
    for (int j = 0; j < kHid; ++j) {
        const float d = __shfl_sync(0xffffffffu, da2[j >> 5], j & 31);
#pragma unroll
        for (int k = 0; k < 2; ++k) s2[k] = fmaf(d, P[oW2 + j * kHid + lane + 32 * k], s2[k]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) c[cDa1 + lane + 32 * k] = s2[k] * gelu_grad(a1[k]);
}

// one thread per parameter (plus one for the loss): sums over the minibatch
// in row order
__global__ void k_mlp_grad(const float* __restrict__ cache, const float* __restrict__ labels,
                           const int* __restrict__ index, int batch, float* __restrict__ grad,
                           float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kParams) return;
    float g = 0.0f;
    if (p == kParams) {
        for (int b = 0; b < batch; ++b) {
            const float d = cache[(size_t)b * kCache + cY] - labels[index[b]];
            g = fmaf(d, d, g);
        }
        *loss = g / (float)batch;
        return;
    }
    if (p < oB1) {
        const int j = p / kIn, i = p - j * kIn;
        for (int b = 0; b < batch; ++b) {
            const float* c = cache + (size_t)b * kCache;
            g = fmaf(c[cDa1 + j], c[cXn + i], g);
        }
    } else if (p < oW2) {
        const int j = p - oB1;
        for (int b = 0; b < batch; ++b) g += cache[(size_t)b * kCache + cDa1 + j];
    } else if (p < oB2) {
        const int q = p - oW2, j = q / kHid, i = q - j * kHid;
        for (int b = 0; b < batch; ++b) {
            const float* c = cache + (size_t)b * kCache;
            g = fmaf(c[cDa2 + j], c[cH1 + i], g);
        }
    } else if (p < oW3) {
        const int j = p - oB2;
        for (int b = 0; b < batch; ++b) g += cache[(size_t)b * kCache + cDa2 + j];
    } else if (p < oB3) {
        const int j = p - oW3;
        for (int b = 0; b < batch; ++b) {
            const float* c = cache + (size_t)b * kCache;
            g = fmaf(c[cDz], c[cH2 + j], g);
        }
    } else {
        for (int b = 0; b < batch; ++b) g += cache[(size_t)b * kCache + cDz];
    }
    grad[p] = g;
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float gi = g[p];
    const float mi = b1 * m[p] + (1.0f - b1) * gi;
    const float vi = b2 * v[p] + (1.0f - b2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    P[p] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// training target of a quality label: (Q - 1) / 99 (IEEE division, as the
// host would compute it in float32)
__global__ void k_quality_labels(const int32_t* __restrict__ q, int n, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(q[i] - 1) / 99.0f;
}

// mean and standard deviation of every feature (one thread per feature, in
// row order, float64); a standard deviation below 1e-6 becomes 1
__global__ void k_feat_norm(const float* __restrict__ feats, int n, float* __restrict__ mean,
                            float* __restrict__ stdv) {
    const int i = threadIdx.x;
    if (i >= kIn) return;
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += (double)feats[(size_t)r * kIn + i];
    const double mu = s / n;
    double v = 0.0;
    for (int r = 0; r < n; ++r) {
        const double d = (double)feats[(size_t)r * kIn + i] - mu;
        v += d * d;
    }
    const double sd = sqrt(v / n);
    mean[i] = (float)mu;
    stdv[i] = sd < 1e-6 ? 1.0f : (float)sd;
}

// the 80 features of one frame from its statistics words (float64 arithmetic)
__global__ void k_features(const unsigned long long* __restrict__ stats, const int* __restrict__ width,
                           const int* __restrict__ height, const float* __restrict__ target, int n,
                           float* __restrict__ out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const unsigned long long* st = stats + (size_t)f * kStatsWords;
    float* o = out + (size_t)f * kIn;
    const double nb = (double)st[kStBlocks], ns = (double)st[kStSamples];
    for (int k = 0; k < 64; ++k) o[k] = (float)log1p((double)st[k] / nb);
    const double mean = (double)st[kStSum] / ns;
    double var = (double)st[kStSum2] / ns - mean * mean;
    if (var < 0.0) var = 0.0;
    o[64] = (float)(mean / 128.0);
    o[65] = (float)(sqrt(var) / 64.0);
    o[66] = (float)((double)st[kStMin] / 255.0);
    o[67] = (float)((double)st[kStMax] / 255.0);
    const double nd = nb * 56.0;
    o[68] = (float)((double)st[kStAbsDx] / nd / 32.0);
    o[69] = (float)((double)st[kStAbsDy] / nd / 32.0);
    o[70] = (float)(sqrt((double)st[kStDx2] / nd) / 32.0);
    o[71] = (float)(sqrt((double)st[kStDy2] / nd) / 32.0);
    for (int k = 0; k < 4; ++k) o[72 + k] = (float)((double)st[kStLowAc + k] / nb);
    o[76] = (float)(log2((double)width[f]) / 11.0);
    o[77] = (float)(log2((double)height[f]) / 11.0);
    o[78] = (float)(((double)target[f] - 35.0) / 7.0);
    o[79] = 1.0f;
}

cudaError_t launch_features(const unsigned long long* stats, const int* w, const int* h, const float* t, int n,
                            float* out, cudaStream_t s) {
    k_features<<<(n + 127) / 128, 128, 0, s>>>(stats, w, h, t, n, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const dct_mlp* net, const float* feats, int n, float* y, int* q, cudaStream_t s) {
    k_mlp_forward<<<(n + 63) / 64, 64, 0, s>>>(net->params, feats, net->feat_mean, net->feat_std, net->act_bf16, n,
                                               y, q);
    return cudaGetLastError();
}

static dct_status check_net(const dct_mlp* net, bool train) {
    if (!net || !net->params || !net->feat_mean || !net->feat_std)
        return fail(DCT_ERR_INVALID_ARG, "network pointers are null");
    if (train && (!net->adam_m || !net->adam_v)) return fail(DCT_ERR_INVALID_ARG, "Adam state pointers are null");
    if (net->act_bf16 != 0 && net->act_bf16 != 1) return fail(DCT_ERR_INVALID_ARG, "act_bf16 must be 0 or 1");
    return DCT_OK;
}

}  // namespace dctgb

using namespace dctgb;

extern "C" {

dct_status dct_features(const uint64_t* stats, const int32_t* width, const int32_t* height, const float* target,
                        int n, float* feats_out, dct_stream_t stream) {
    if (!stats || !width || !height || !target || !feats_out) return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (n < 1) return fail(DCT_ERR_INVALID_ARG, "n must be >= 1");
    cudaError_t e = launch_features(reinterpret_cast<const unsigned long long*>(stats), width, height, target, n,
                                    feats_out, (cudaStream_t)stream);
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "features launch");
}

dct_status dct_mlp_set_norm(dct_mlp* net, const float* feats, int n, dct_stream_t stream) {
    dct_status st = check_net(net, false);
    if (st != DCT_OK) return st;
    if (!feats || n < 1) return fail(DCT_ERR_INVALID_ARG, "feats null or n < 1");
    k_feat_norm<<<1, 128, 0, (cudaStream_t)stream>>>(feats, n, net->feat_mean, net->feat_std);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "norm launch");
}

dct_status dct_mlp_forward(const dct_mlp* net, const float* feats, int n, float* y_out, int32_t* quality_out,
                           dct_stream_t stream) {
    dct_status st = check_net(net, false);
    if (st != DCT_OK) return st;
    if (!feats || n < 1) return fail(DCT_ERR_INVALID_ARG, "feats null or n < 1");
    cudaError_t e = launch_mlp_forward(net, feats, n, y_out, quality_out, (cudaStream_t)stream);
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "forward launch");
}

dct_status dct_mlp_labels(const int32_t* quality, int n, float* labels_out, dct_stream_t stream) {
    if (!quality || !labels_out) return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (n < 1) return fail(DCT_ERR_INVALID_ARG, "n must be >= 1");
    k_quality_labels<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(quality, n, labels_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "labels launch");
}

size_t dct_mlp_workspace_bytes(int batch) {
    if (batch < 1) return 0;
    return sizeof(float) * ((size_t)batch * kCache + kParams + 4);
}

dct_status dct_mlp_loss_grad(const dct_mlp* net, const float* feats, const float* labels, const int32_t* index,
                             int batch, float* grad_out, float* loss_out, void* workspace, dct_stream_t stream) {
    dct_status st = check_net(net, false);
    if (st != DCT_OK) return st;
    if (!feats || !labels || !index || !grad_out || !loss_out || !workspace)
        return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (batch < 1 || batch > (1 << 20)) return fail(DCT_ERR_INVALID_ARG, "batch must be 1..2^20");
    cudaStream_t s = (cudaStream_t)stream;
    float* cache = static_cast<float*>(workspace);
    // one warp per row (4 rows per CTA); 64-thread CTAs for the per-parameter
    // sums so that they spread over every SM
    k_mlp_delta<<<(batch + 3) / 4, 128, 0, s>>>(net->params, feats, labels, index, net->feat_mean, net->feat_std,
                                                net->act_bf16, batch, cache);
    k_mlp_grad<<<(kParams + 1 + 63) / 64, 64, 0, s>>>(cache, labels, index, batch, grad_out, loss_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "gradient launch");
}

dct_status dct_mlp_adam(dct_mlp* net, const float* grad, float lr, float beta1, float beta2, float eps,
                        dct_stream_t stream) {
    dct_status st = check_net(net, true);
    if (st != DCT_OK) return st;
    if (!grad) return fail(DCT_ERR_INVALID_ARG, "null grad");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(DCT_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    net->step += 1;
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, net->step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, net->step));
    k_adam<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(net->params, net->adam_m, net->adam_v, grad, lr,
                                                                    beta1, beta2, eps, (float)c1, (float)c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "adam launch");
}

dct_status dct_mlp_train_epoch(dct_mlp* net, const float* feats, const float* labels, const int32_t* order, int n,
                               int batch, float lr, float* loss_out, void* workspace, dct_stream_t stream) {
    dct_status st = check_net(net, true);
    if (st != DCT_OK) return st;
    if (!feats || !labels || !order || !loss_out || !workspace) return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || batch < 1) return fail(DCT_ERR_INVALID_ARG, "n and batch must be >= 1");
    float* grad = reinterpret_cast<float*>(static_cast<char*>(workspace) + dct_mlp_workspace_bytes(batch));
    for (int b0 = 0, k = 0; b0 < n; b0 += batch, ++k) {
        const int cnt = n - b0 < batch ? n - b0 : batch;
        st = dct_mlp_loss_grad(net, feats, labels, order + b0, cnt, grad, loss_out + k, workspace, stream);
        if (st != DCT_OK) return st;
        st = dct_mlp_adam(net, grad, lr, 0.9f, 0.999f, 1e-8f, stream);
        if (st != DCT_OK) return st;
    }
    return DCT_OK;
}

}  // extern "C"
