// Exact-DCT pipeline on the GPU: the "DCT" rows of Tables 3 and 4, i.e. the
// orthonormal 2-D DCT of Eq. 6, quantiser, dequantiser and inverse, in
// float32 with a fixed order of operations (each product and sum rounded on
// its own, no fused multiply-add), so that the quantised codes and the
// rounded pixels are reproducible:
//   rows    Z[i][v] = sum_k C[v][k] x[i][k]     (k ascending), x = p - 128
//   columns X[u][v] = sum_k C[u][k] Z[k][v]
//   q = sgn(X) floor(|X| / Q + 0.5),  D = q Q
//   columns T[i][v] = sum_u C[u][i] D[u][v];  rows y[i][j] = sum_v C[v][j] T[i][v]
//   r = clamp(floor((y + 128) + 0.5), 0, 255)
// One thread owns one 8x8 block (warp tiles of 32 blocks as in the Cordic
// kernels); the 64 float multiplies and adds per output run on the FMA pipes.
#include <cmath>
#include <cstring>

#include "host_common.h"

namespace dctgb {

struct ExactArgs {
    PlaneArg p[kMaxPlanes];
    float C[64];          // C[u * 8 + i] = sqrt(2/8) alpha(u) cos(pi u (2i + 1) / 16), rounded to float
    float Q[2][64];       // quantiser steps (luma, chroma)
    int32_t nplanes;
    int32_t ntiles;
};

__device__ __forceinline__ float dot8_rows(const float* __restrict__ c, const float (&x)[8]) {
    float acc = __fmul_rn(c[0], x[0]);
#pragma unroll
    for (int k = 1; k < 8; ++k) acc = __fadd_rn(acc, __fmul_rn(c[k], x[k]));
    return acc;
}

template <bool STORE_COEF, bool STORE_RECON>
__global__ void __launch_bounds__(256, 1) k_exact(const __grid_constant__ ExactArgs a) {
    __shared__ unsigned long long sse_acc[kMaxPlanes];
    if (threadIdx.x < kMaxPlanes) sse_acc[threadIdx.x] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int tile = blockIdx.x * warps + (threadIdx.x >> 5); tile < a.ntiles; tile += gridDim.x * warps) {
        int pi = 0;
#pragma unroll
        for (int k = 1; k < kMaxPlanes; ++k)
            if (k < a.nplanes && tile >= a.p[k].tile_begin) pi = k;
        const PlaneArg& P = a.p[pi];
        const float* Qt = a.Q[P.table];
        const int b = (tile - P.tile_begin) * kTileBlocks + lane;
        unsigned e = 0;
        if (b < P.nblk) {
            const int by = b / P.nbx, bx = b - by * P.nbx;
            uint32_t pix[8][2];
            load_block(P.src, P.src_pitch, P.width, P.height, by, bx, (P.flags & kVecSrc) != 0, pix);
            float x[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) x[r][c] = (float)sample(pix, r, c) - 128.0f;
            // rows: Z[i][v] = sum_k C[v][k] x[i][k]
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float t[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) t[v] = dot8_rows(a.C + v * 8, x[i]);
#pragma unroll
                for (int v = 0; v < 8; ++v) x[i][v] = t[v];
            }
            // columns: X[u][v] = sum_k C[u][k] Z[k][v]
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                float col[8], t[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) col[k] = x[k][v];
#pragma unroll
                for (int u = 0; u < 8; ++u) t[u] = dot8_rows(a.C + u * 8, col);
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u][v] = t[u];
            }
            // quantise (codes kept as exact small integers in float), store
            int16_t* cg = STORE_COEF ? P.coef + (size_t)b * 64 : nullptr;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint32_t w[4];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const float X = x[u][v];
                    const float t = floorf(__fadd_rn(__fdiv_rn(fabsf(X), Qt[u * 8 + v]), 0.5f));
                    const float q = X < 0.0f ? -t : t;
                    x[u][v] = __fmul_rn(q, Qt[u * 8 + v]);                 // dequantised D
                    if (STORE_COEF) {
                        const uint32_t h = (uint32_t)(int)q & 0xFFFFu;
                        if (v & 1) w[v >> 1] |= h << 16;
                        else w[v >> 1] = h;
                    }
                }
                if (STORE_COEF) *reinterpret_cast<uint4*>(cg + u * 8) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            // columns: T[i][v] = sum_u C[u][i] D[u][v]
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                float col[8], t[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) col[k] = x[k][v];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float acc = __fmul_rn(a.C[0 * 8 + i], col[0]);
#pragma unroll
                    for (int u = 1; u < 8; ++u) acc = __fadd_rn(acc, __fmul_rn(a.C[u * 8 + i], col[u]));
                    t[i] = acc;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i][v] = t[i];
            }
            // rows: y[i][j] = sum_v C[v][j] T[i][v]; pixels
            uint32_t out[8][2];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t wd[2] = {0u, 0u};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float acc = __fmul_rn(a.C[0 * 8 + j], x[i][0]);
#pragma unroll
                    for (int v = 1; v < 8; ++v) acc = __fadd_rn(acc, __fmul_rn(a.C[v * 8 + j], x[i][v]));
                    const float r = floorf(__fadd_rn(__fadd_rn(acc, 128.0f), 0.5f));
                    const int ri = (int)fminf(255.0f, fmaxf(0.0f, r));
                    wd[j >> 2] |= (uint32_t)ri << (8 * (j & 3));
                }
                out[i][0] = wd[0];
                out[i][1] = wd[1];
            }
            if (STORE_RECON) store_block(P.dst, P.dst_pitch, P.width, P.height, by, bx, (P.flags & kVecDst) != 0, out);
            const int nr = min(8, P.height - by * 8), nc = min(8, P.width - bx * 8);
            for (int r = 0; r < nr; ++r)
                for (int c = 0; c < nc; ++c) {
                    const int d = sample(out, r, c) - sample(pix, r, c);
                    e += d * d;
                }
        }
        const unsigned tot = warp_sum(e);
        if (lane == 0 && tot) atomicAdd(&sse_acc[pi], (unsigned long long)tot);
    }
    __syncthreads();
    if (threadIdx.x < a.nplanes && sse_acc[threadIdx.x]) atomicAdd(a.p[threadIdx.x].sse, sse_acc[threadIdx.x]);
}

// float32 basis, from the FP64 values sqrt(2/8) alpha(u) cos(pi u (2i+1) / 16)
static void basis(float C[64]) {
    const double pi = 3.14159265358979323846;
    for (int u = 0; u < 8; ++u)
        for (int i = 0; i < 8; ++i) {
            const double alpha = u == 0 ? 1.0 / std::sqrt(2.0) : 1.0;
            C[u * 8 + i] = (float)(std::sqrt(2.0 / 8) * alpha * std::cos(pi * u * (2 * i + 1) / 16.0));
        }
}

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_exact_fused(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                                      const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                                      const dct_plane* recon_planes, uint64_t* sse_out, dct_stream_t stream) {
    if (!plan) return fail(DCT_ERR_INVALID_ARG, "null plan");
    if (!planes || !sse_out) return fail(DCT_ERR_INVALID_ARG, "null planes or sse_out");
    if (nplanes < 1 || nplanes > kMaxPlanes) return fail(DCT_ERR_INVALID_ARG, "nplanes must be 1..4");
    if (((uintptr_t)sse_out) & 7u) return fail(DCT_ERR_INVALID_ARG, "sse_out must be 8-byte aligned");
    if (coeffs && (((uintptr_t)coeffs) & 15u)) return fail(DCT_ERR_INVALID_ARG, "coeffs must be 16-byte aligned");
    ExactArgs a;
    memset(&a, 0, sizeof a);
    const bool yuv = plan->desc.layout == DCT_LAYOUT_YUV420;
    for (int t = 0; t < 2; ++t) {
        QuantSet qs;
        dct_status st = build_tables(quality, qtab_host, qtab_entries, (t == 1 && yuv) ? 1 : 0, qs);
        if (st != DCT_OK) return st;
        for (int k = 0; k < 64; ++k) a.Q[t][k] = (float)qs.Q[k];
    }
    basis(a.C);
    int cursor = 0;
    size_t coef_off = 0;
    for (int i = 0; i < nplanes; ++i) {
        dct_status st = check_plane(plan, planes[i], "plane");
        if (st != DCT_OK) return st;
        PlaneArg& p = a.p[i];
        fill_plane(p, planes[i], cursor);
        p.src = planes[i].data;
        p.src_pitch = planes[i].pitch;
        p.table = (yuv && i > 0) ? 1 : 0;
        int fl = ((((uintptr_t)planes[i].data) & 7u) == 0 && (planes[i].pitch & 7) == 0) ? kVecSrc : 0;
        if (recon_planes) {
            st = check_plane(plan, recon_planes[i], "recon plane");
            if (st != DCT_OK) return st;
            if (recon_planes[i].width != planes[i].width || recon_planes[i].height != planes[i].height)
                return fail(DCT_ERR_INVALID_ARG, "recon plane size differs from input plane");
            p.dst = recon_planes[i].data;
            p.dst_pitch = recon_planes[i].pitch;
            if ((((uintptr_t)recon_planes[i].data) & 7u) == 0 && (recon_planes[i].pitch & 7) == 0) fl |= kVecDst;
        }
        p.flags = fl;
        p.coef = coeffs ? coeffs + coef_off : nullptr;
        coef_off += (size_t)p.nblk * 64;
        p.sse = reinterpret_cast<unsigned long long*>(sse_out) + i;
    }
    a.nplanes = nplanes;
    a.ntiles = cursor;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(sse_out, 0, sizeof(uint64_t) * nplanes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const int threads = 256;
    int grid = (cursor + 7) / 8;
    if (grid > plan->num_sms * 2) grid = plan->num_sms * 2;
    if (grid < 1) grid = 1;
    if (coeffs && recon_planes) k_exact<true, true><<<grid, threads, 0, s>>>(a);
    else if (coeffs) k_exact<true, false><<<grid, threads, 0, s>>>(a);
    else if (recon_planes) k_exact<false, true><<<grid, threads, 0, s>>>(a);
    else k_exact<false, false><<<grid, threads, 0, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "exact launch");
}
