// Learned rate controller, network side: the 80 features, input
// normalisation, forward pass, back-propagation with deterministic
// (fixed-order) minibatch sums, and Adam.  The network is tiny (9409
// parameters), so it runs on plain FMA units: one thread per sample for
// inference, one warp per minibatch row for the training forward and delta
// pass, one thread per parameter for the gradient sums (in tiles that stage
// the minibatch in shared memory) and the update.
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "host_common.h"

namespace dctgb {

constexpr int kIn = DCT_MLP_INPUTS, kHid = DCT_MLP_HIDDEN, kParams = DCT_MLP_PARAMS;
constexpr int oW1 = 0, oB1 = kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid;
static_assert(oB3 + 1 == kParams, "parameter layout");
static_assert(oW1 % 4 == 0 && oW2 % 4 == 0 && kIn % 4 == 0 && kHid % 4 == 0, "16-byte weight rows");

// per-sample cache (floats): xn[80] a1[64] h1[64] a2[64] h2[64] da2[64]
// da1[64] y dz, every vector 16-byte aligned (the row is 468 floats)
constexpr int cXn = 0, cA1 = cXn + kIn, cH1 = cA1 + kHid, cA2 = cH1 + kHid, cH2 = cA2 + kHid, cDa2 = cH2 + kHid,
              cDa1 = cDa2 + kHid, cY = cDa1 + kHid, cDz = cY + 1, kCache = ((cDz + 1 + 3) / 4) * 4;
static_assert(cH1 % 4 == 0 && cH2 % 4 == 0 && cDa2 % 4 == 0 && cDa1 % 4 == 0 && kCache % 4 == 0, "cache alignment");

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
// does not hold come by shuffle), so the cache holds the same values.  The
// CTA first stages W1 and W2 transposed in shared memory with rows padded
// to 65 floats: the forward sums read W^T[i][lane] and the backward sum
// reads W2[j][lane] = W2^T[lane][j], both free of bank conflicts (reading
// W1 straight from global memory touched 32 cache lines per warp access).
constexpr int kDeltaRows = 8;                  // minibatch rows (warps) per CTA
constexpr int kTStride = kHid + 1;             // padded row of a transposed weight matrix

__global__ void __launch_bounds__(kDeltaRows * 32)
k_mlp_delta(const float* __restrict__ P, const float* __restrict__ feats, const float* __restrict__ labels,
            const int* __restrict__ index, const float* __restrict__ mean, const float* __restrict__ stdv, int bf16,
            int batch, float* __restrict__ cache) {
    __shared__ float w1t[kIn * kTStride];       // w1t[i * 65 + j] = W1[j][i]
    __shared__ float w2t[kHid * kTStride];      // w2t[i * 65 + j] = W2[j][i]
    {
        // 16-byte loads along the rows of W1 and W2 (both start 16-byte
        // aligned), all issued before the first shared-memory store
        constexpr int n1 = kHid * kIn / 4, n2 = kHid * kHid / 4, nv = n1 + n2;
        constexpr int per = (nv + kDeltaRows * 32 - 1) / (kDeltaRows * 32);
        const float4* P4 = reinterpret_cast<const float4*>(P);
        float4 v[per];
#pragma unroll
        for (int u = 0; u < per; ++u) {
            const int e = threadIdx.x + u * kDeltaRows * 32;
            if (e < n1) v[u] = P4[oW1 / 4 + e];
            else if (e < nv) v[u] = P4[oW2 / 4 + e - n1];
        }
#pragma unroll
        for (int u = 0; u < per; ++u) {
            const int e = threadIdx.x + u * kDeltaRows * 32;
            if (e < n1) {
                const int j = (4 * e) / kIn, i = 4 * e - j * kIn;
                w1t[(i + 0) * kTStride + j] = v[u].x;
                w1t[(i + 1) * kTStride + j] = v[u].y;
                w1t[(i + 2) * kTStride + j] = v[u].z;
                w1t[(i + 3) * kTStride + j] = v[u].w;
            } else if (e < nv) {
                const int f = 4 * (e - n1), j = f / kHid, i = f - j * kHid;
                w2t[(i + 0) * kTStride + j] = v[u].x;
                w2t[(i + 1) * kTStride + j] = v[u].y;
                w2t[(i + 2) * kTStride + j] = v[u].z;
                w2t[(i + 3) * kTStride + j] = v[u].w;
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= batch) return;                                   // warp-uniform, after the only barrier
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
        for (int k = 0; k < 2; ++k) a1[k] = fmaf(w1t[i * kTStride + lane + 32 * k], v, a1[k]);
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
        for (int k = 0; k < 2; ++k) a2[k] = fmaf(w2t[i * kTStride + lane + 32 * k], v, a2[k]);
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
        for (int k = 0; k < 2; ++k) s2[k] = fmaf(d, w2t[(lane + 32 * k) * kTStride + j], s2[k]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) c[cDa1 + lane + 32 * k] = s2[k] * gelu_grad(a1[k]);
}

// Per-parameter minibatch sums, one output per thread, each over the rows
// in ascending order (deterministic).  CTAs 0..15 own the W1 gradients of
// four hidden units (320 outputs), CTAs 16..31 the W2 gradients of four
// units (256), CTA 32 the b1 sums, CTA 33 the b2 sums and CTA 34 the W3 and
// b3 sums and the loss.  Each CTA stages the cache columns it needs for
// kGradRows rows at a time in shared memory (contiguous reads), then every
// thread runs its sum over the staged rows.
constexpr int kGradUnits = 4;
constexpr int kGradRows = 128;
constexpr int kW1Tiles = kHid / kGradUnits, kW2Tiles = kHid / kGradUnits;
constexpr int kGradCtas = kW1Tiles + kW2Tiles + 3;
constexpr int kGradThreads = kGradUnits * kIn;               // the widest tile
static_assert(kHid % kGradUnits == 0 && kGradThreads >= kHid + 2, "gradient tiling");

// Adam step for one parameter (k_adam and the fused gradient kernel)
struct AdamArgs {
    float* P;
    float* m;
    float* v;
    float lr, b1, b2, eps, c1, c2;
};

__device__ __forceinline__ void adam_update(const AdamArgs& a, int p, float gi) {
    const float mi = a.b1 * a.m[p] + (1.0f - a.b1) * gi;
    const float vi = a.b2 * a.v[p] + (1.0f - a.b2) * gi * gi;
    a.m[p] = mi;
    a.v[p] = vi;
    a.P[p] -= a.lr * (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps);
}

// ADAM: also apply the Adam step to each parameter as soon as its sum is
// final (each parameter belongs to one thread; nothing in this kernel reads
// the parameters), saving the separate update launch of a training step.
template <bool ADAM>
__global__ void __launch_bounds__(kGradThreads)
k_mlp_grad(const float* __restrict__ cache, const float* __restrict__ labels, const int* __restrict__ index,
           int batch, float* __restrict__ grad, float* __restrict__ loss, AdamArgs adam) {
    __shared__ __align__(16) float sm[kGradRows * (kGradUnits + kIn)];
    const int t = threadIdx.x;
    const int blk = blockIdx.x;
    // the staged row: `ncol` floats (a multiple of 4) = na float4 from cache
    // column ca, then nb float4 from column cb; the last CTA's rows end with
    // (dz, y - label, 0, 0)
    int ncol, ca, na, cb, nb;
    const bool last = blk == kW1Tiles + kW2Tiles + 2;
    if (blk < kW1Tiles) {
        ca = cDa1 + kGradUnits * blk; na = kGradUnits / 4; cb = cXn; nb = kIn / 4;
    } else if (blk < kW1Tiles + kW2Tiles) {
        ca = cDa2 + kGradUnits * (blk - kW1Tiles); na = kGradUnits / 4; cb = cH1; nb = kHid / 4;
    } else if (blk == kW1Tiles + kW2Tiles) {
        ca = cDa1; na = kHid / 4; cb = 0; nb = 0;
    } else if (blk == kW1Tiles + kW2Tiles + 1) {
        ca = cDa2; na = kHid / 4; cb = 0; nb = 0;
    } else {
        ca = cH2; na = kHid / 4; cb = 0; nb = 0;
    }
    const int nv = na + nb + (last ? 1 : 0);
    ncol = 4 * nv;
    float4* sm4 = reinterpret_cast<float4*>(sm);
    const float4* cache4 = reinterpret_cast<const float4*>(cache);
    float g = 0.0f;
    for (int r0 = 0; r0 < batch; r0 += kGradRows) {
        const int rows = min(kGradRows, batch - r0);
        const int total = rows * nv;
        __syncthreads();
        // 16-byte loads, eight in flight per thread before the stores
        for (int e0 = t; e0 < total; e0 += 8 * kGradThreads) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * kGradThreads;
                if (e < total) {
                    const int r = e / nv, k = e - r * nv;
                    const size_t row4 = (size_t)(r0 + r) * (kCache / 4);
                    if (k < na) {
                        v[u] = cache4[row4 + ca / 4 + k];
                    } else if (k < na + nb) {
                        v[u] = cache4[row4 + cb / 4 + k - na];
                    } else {
                        const float* row = cache + (size_t)(r0 + r) * kCache;
                        v[u] = make_float4(row[cDz], row[cY] - labels[index[r0 + r]], 0.0f, 0.0f);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * kGradThreads;
                if (e < total) sm4[e] = v[u];
            }
        }
        __syncthreads();
        if (blk < kW1Tiles + kW2Tiles) {
            const int nin = blk < kW1Tiles ? kIn : kHid;
            if (t < kGradUnits * nin) {
                const int u = t / nin, i = t - u * nin;
                for (int r = 0; r < rows; ++r) g = fmaf(sm[r * ncol + u], sm[r * ncol + kGradUnits + i], g);
            }
        } else if (blk < kW1Tiles + kW2Tiles + 2) {
            if (t < kHid)
                for (int r = 0; r < rows; ++r) g += sm[r * ncol + t];
        } else if (t < kHid) {                           // W3
            for (int r = 0; r < rows; ++r) g = fmaf(sm[r * ncol + kHid], sm[r * ncol + t], g);
        } else if (t == kHid) {                          // b3
            for (int r = 0; r < rows; ++r) g += sm[r * ncol + kHid];
        } else if (t == kHid + 1) {                      // loss
            for (int r = 0; r < rows; ++r) {
                const float d = sm[r * ncol + kHid + 1];
                g = fmaf(d, d, g);
            }
        }
    }
    int p = -1;
    if (blk < kW1Tiles) {
        if (t < kGradUnits * kIn) p = oW1 + (kGradUnits * blk) * kIn + t;
    } else if (blk < kW1Tiles + kW2Tiles) {
        if (t < kGradUnits * kHid) p = oW2 + (kGradUnits * (blk - kW1Tiles)) * kHid + t;
    } else if (blk == kW1Tiles + kW2Tiles) {
        if (t < kHid) p = oB1 + t;
    } else if (blk == kW1Tiles + kW2Tiles + 1) {
        if (t < kHid) p = oB2 + t;
    } else if (t < kHid) {
        p = oW3 + t;
    } else if (t == kHid) {
        p = oB3;
    } else if (t == kHid + 1) {
        *loss = g / (float)batch;
    }
    if (p >= 0) {
        grad[p] = g;
        if (ADAM) adam_update(adam, p, g);
    }
}

__global__ void k_adam(AdamArgs a, const float* __restrict__ g) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    adam_update(a, p, g[p]);
}

// training target of a quality label: (Q - 1) / 99 (IEEE division, as the
// host would compute it in float32)
__global__ void k_quality_labels(const int32_t* __restrict__ q, int n, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(q[i] - 1) / 99.0f;
}

// mean and standard deviation of every feature (float64): one CTA per
// feature, each thread summing a fixed stride of rows, the partial sums
// combined in a fixed tree (deterministic); a standard deviation below 1e-6
// becomes 1
constexpr int kNormThreads = 256;

__device__ double cta_sum_fixed(double v, double* red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kNormThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kNormThreads)
k_feat_norm(const float* __restrict__ feats, int n, float* __restrict__ mean, float* __restrict__ stdv) {
    __shared__ double red[kNormThreads];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < n; r += kNormThreads) s += (double)feats[(size_t)r * kIn + i];
    const double mu = cta_sum_fixed(s, red) / n;
    double v = 0.0;
    for (int r = threadIdx.x; r < n; r += kNormThreads) {
        const double d = (double)feats[(size_t)r * kIn + i] - mu;
        v += d * d;
    }
    const double sd = sqrt(cta_sum_fixed(v, red) / n);
    if (threadIdx.x == 0) {
        mean[i] = (float)mu;
        stdv[i] = sd < 1e-6 ? 1.0f : (float)sd;
    }
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

static bool adam_params_ok(float lr, float beta1, float beta2, float eps) {
    return lr > 0.f && beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f;
}

// advances the network's step count and returns the Adam arguments of that
// step (bias corrections computed on the host in float64)
static AdamArgs next_adam_step(dct_mlp* net, float lr, float beta1, float beta2, float eps) {
    net->step += 1;
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, net->step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, net->step));
    return AdamArgs{net->params, net->adam_m, net->adam_v, lr, beta1, beta2, eps, (float)c1, (float)c2};
}

// one minibatch: forward and deltas (one warp per row, 8 rows per CTA,
// weights staged once per CTA), then one CTA per gradient tile
template <bool ADAM>
static cudaError_t launch_train_step(const dct_mlp* net, const float* feats, const float* labels, const int* index,
                                     int batch, float* grad, float* loss, void* workspace, AdamArgs adam,
                                     cudaStream_t s) {
    float* cache = static_cast<float*>(workspace);
    k_mlp_delta<<<(batch + kDeltaRows - 1) / kDeltaRows, kDeltaRows * 32, 0, s>>>(
        net->params, feats, labels, index, net->feat_mean, net->feat_std, net->act_bf16, batch, cache);
    k_mlp_grad<ADAM><<<kGradCtas, kGradThreads, 0, s>>>(cache, labels, index, batch, grad, loss, adam);
    return cudaGetLastError();
}

static dct_status check_net(const dct_mlp* net, bool train) {
    if (!net || !net->params || !net->feat_mean || !net->feat_std)
        return fail(DCT_ERR_INVALID_ARG, "network pointers are null");
    if (train && (!net->adam_m || !net->adam_v)) return fail(DCT_ERR_INVALID_ARG, "Adam state pointers are null");
    if (net->act_bf16 != 0 && net->act_bf16 != 1) return fail(DCT_ERR_INVALID_ARG, "act_bf16 must be 0 or 1");
    if (((uintptr_t)net->params) & 15u) return fail(DCT_ERR_INVALID_ARG, "params must be 16-byte aligned");
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
    k_feat_norm<<<kIn, kNormThreads, 0, (cudaStream_t)stream>>>(feats, n, net->feat_mean, net->feat_std);
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
    if (((uintptr_t)workspace) & 15u) return fail(DCT_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    cudaError_t e = launch_train_step<false>(net, feats, labels, index, batch, grad_out, loss_out, workspace,
                                             AdamArgs{}, (cudaStream_t)stream);
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "gradient launch");
}

dct_status dct_mlp_adam(dct_mlp* net, const float* grad, float lr, float beta1, float beta2, float eps,
                        dct_stream_t stream) {
    dct_status st = check_net(net, true);
    if (st != DCT_OK) return st;
    if (!grad) return fail(DCT_ERR_INVALID_ARG, "null grad");
    if (!adam_params_ok(lr, beta1, beta2, eps)) return fail(DCT_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    k_adam<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(next_adam_step(net, lr, beta1, beta2, eps), grad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "adam launch");
}

dct_status dct_mlp_train_epoch(dct_mlp* net, const float* feats, const float* labels, const int32_t* order, int n,
                               int batch, float lr, float* loss_out, void* workspace, dct_stream_t stream) {
    dct_status st = check_net(net, true);
    if (st != DCT_OK) return st;
    if (!feats || !labels || !order || !loss_out || !workspace) return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || batch < 1 || batch > (1 << 20)) return fail(DCT_ERR_INVALID_ARG, "n >= 1 and batch in 1..2^20");
    if (!adam_params_ok(lr, 0.9f, 0.999f, 1e-8f)) return fail(DCT_ERR_INVALID_ARG, "learning rate must be > 0");
    if (((uintptr_t)workspace) & 15u) return fail(DCT_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    float* grad = reinterpret_cast<float*>(static_cast<char*>(workspace) + dct_mlp_workspace_bytes(batch));
    // per minibatch: the delta kernel, then the gradient sums with the Adam
    // step fused (same arithmetic as dct_mlp_loss_grad + dct_mlp_adam)
    for (int b0 = 0, k = 0; b0 < n; b0 += batch, ++k) {
        const int cnt = n - b0 < batch ? n - b0 : batch;
        cudaError_t e = launch_train_step<true>(net, feats, labels, order + b0, cnt, grad, loss_out + k, workspace,
                                                next_adam_step(net, lr, 0.9f, 0.999f, 1e-8f), (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "training step launch");
    }
    return DCT_OK;
}

}  // extern "C"
