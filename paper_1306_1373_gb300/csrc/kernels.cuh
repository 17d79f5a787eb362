// Codec kernels: forward path (Sec. 2.5.2 transform + Sec. 3.2 quantiser),
// inverse path (Sec. 3.2 dequantiser + IDCT) and the SSE of Eq. 24, for
// uint8 planes, all in integer arithmetic.
//
// Work decomposition: a plane of nbx x nby 8x8 blocks is cut into warp tiles
// of kTileBlocks consecutive blocks in block-major order (b = by * nbx + bx,
// wrapping across block rows).  Lane l of a warp owns block b0 + l and keeps
// its 64 samples in registers, so the row/column transpose between the two
// 1-D passes is free.  Pixel rows are loaded and stored 8 bytes per lane
// (a warp covers 256 contiguous bytes of a row); int16 coefficients go
// through a padded per-warp shared-memory stage so that the global side is
// 16 bytes per lane over contiguous 512-byte spans.  The grid is persistent:
// warps stride over all tiles of all planes of the launch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cordic_loeffler.cuh"
#include "dctgb_spec.h"

namespace dctgb {

constexpr int kMaxPlanes = 4;
constexpr int kTileBlocks = 32;      // blocks per warp tile (one per lane)
constexpr int kStageStride = 144;    // bytes per block in the stage (128 + 16 pad)
constexpr int kStageBytesPerWarp = kTileBlocks * kStageStride;

// Per-plane quantiser / dequantiser tables (natural order u*8+v).
struct QuantSet {
    uint32_t M[64];   // rint(2^32 / (8 * 2^P * g_u g_v Q))
    int32_t Q[64];    // 1..255
    int32_t W[64];    // rint(2^R / (g_u g_v))
};

struct PlaneArg {
    const uint8_t* src;       // samples (forward path, SSE reference in fused mode)
    int16_t* coef;            // block-major coefficients of this plane
    uint8_t* dst;             // reconstruction
    const uint8_t* ref;       // SSE reference for the inverse-only path
    unsigned long long* sse;  // per-plane SSE accumulator (global)
    unsigned long long* stats;// per-plane statistics words (global)
    int32_t src_pitch, dst_pitch, ref_pitch;
    int32_t width, height, nbx, nblk;
    int32_t table;            // index into the launch's QuantSet array
    int32_t tile_begin;       // first global tile index of this plane
    int32_t flags;            // kVecSrc | kVecDst | kVecRef
};
constexpr int kVecSrc = 1, kVecDst = 2, kVecRef = 4;

struct DirectArgs {
    PlaneArg p[kMaxPlanes];
    QuantSet tabs[2];
    int32_t nplanes;
    int32_t ntiles;
};

// Mode bits of the kernel template.
enum : unsigned {
    kLoadPix = 1u,     // read samples, forward transform, quantise
    kStoreCoef = 2u,   // write the quantised coefficients
    kLoadCoef = 4u,    // read quantised coefficients
    kInverse = 8u,     // dequantise, inverse transform, descale
    kStoreRecon = 16u, // write the reconstruction
    kSse = 32u,        // accumulate the SSE
    kStats = 64u       // accumulate band-energy and pixel statistics
};

// statistics word layout (per plane)
enum : int {
    kStBand = 0,         // 64 words: sum over blocks of (|Y_uv| >> kBandShift)^2
    kStSum = 64, kStSum2 = 65, kStMin = 66, kStMax = 67,
    kStAbsDx = 68, kStAbsDy = 69, kStDx2 = 70, kStDy2 = 71,
    kStLowAc = 72,       // 4 words: blocks whose AC energy < 2^10, 2^14, 2^18, 2^22
    kStBlocks = 76, kStSamples = 77
};

// --------------------------------------------------------------------------
// sample I/O
// --------------------------------------------------------------------------

// Loads block (by, bx) as 8 rows of two little-endian uint32 words.  Samples
// outside the plane repeat the nearest edge sample (edge replication).
__device__ __forceinline__ void load_block(const uint8_t* __restrict__ src, int pitch, int w, int h,
                                           int by, int bx, bool vec, uint32_t (&pix)[8][2]) {
    const int x0 = bx * 8, y0 = by * 8;
    if (vec && x0 + 8 <= w && y0 + 8 <= h) {
        const uint8_t* p = src + (size_t)y0 * pitch + x0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(p + (size_t)r * pitch));
            pix[r][0] = v.x;
            pix[r][1] = v.y;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int yy = min(y0 + r, h - 1);
            const uint8_t* row = src + (size_t)yy * pitch;
            uint32_t wd[2] = {0u, 0u};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int xx = min(x0 + c, w - 1);
                wd[c >> 2] |= (uint32_t)__ldg(row + xx) << (8 * (c & 3));
            }
            pix[r][0] = wd[0];
            pix[r][1] = wd[1];
        }
    }
}

// Stores the in-plane part of block (by, bx).
__device__ __forceinline__ void store_block(uint8_t* __restrict__ dst, int pitch, int w, int h,
                                            int by, int bx, bool vec, const uint32_t (&pix)[8][2]) {
    const int x0 = bx * 8, y0 = by * 8;
    if (vec && x0 + 8 <= w && y0 + 8 <= h) {
        uint8_t* p = dst + (size_t)y0 * pitch + x0;
#pragma unroll
        for (int r = 0; r < 8; ++r)
            *reinterpret_cast<uint2*>(p + (size_t)r * pitch) = make_uint2(pix[r][0], pix[r][1]);
    } else {
        const int nr = min(8, h - y0), nc = min(8, w - x0);
        for (int r = 0; r < nr; ++r) {
            uint8_t* row = dst + (size_t)(y0 + r) * pitch + x0;
            for (int c = 0; c < nc; ++c) row[c] = (uint8_t)(pix[r][c >> 2] >> (8 * (c & 3)));
        }
    }
}

__device__ __forceinline__ int sample(const uint32_t (&pix)[8][2], int r, int c) {
    return (int)((pix[r][c >> 2] >> (8 * (c & 3))) & 0xFFu);
}

// --------------------------------------------------------------------------
// per-CTA accumulators (shared memory), flushed to global at the end
// --------------------------------------------------------------------------

struct CtaAcc {
    unsigned long long sse[kMaxPlanes];
    unsigned long long st[kMaxPlanes][kStatsWords];
};

__device__ __forceinline__ unsigned warp_sum(unsigned v) { return __reduce_add_sync(0xffffffffu, v); }

// --------------------------------------------------------------------------
// one warp tile
// --------------------------------------------------------------------------

// Processes warp tile `tile_in_plane` of plane P.  Statistics go to the 80
// words at `st` (shared or global memory); the return value is the tile's
// SSE (the same in every lane; 0 without kSse).
template <unsigned MODE>
__device__ __forceinline__ unsigned process_tile(const PlaneArg& P, const QuantSet& T, int tile_in_plane,
                                                 int lane, uint8_t* stage, unsigned long long* st) {
    const int b0 = tile_in_plane * kTileBlocks;
    const int nvalid = min(kTileBlocks, P.nblk - b0);
    const bool active = lane < nvalid;
    const int b = b0 + lane;
    int by = 0, bx = 0;
    if (active) {
        by = b / P.nbx;
        bx = b - by * P.nbx;
    }

    int x[8][8];
    uint32_t pix[8][2];

    if (MODE & kLoadPix) {
        if (active) {
            load_block(P.src, P.src_pitch, P.width, P.height, by, bx, (P.flags & kVecSrc) != 0, pix);
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) pix[r][0] = pix[r][1] = 0x80808080u;
        }

        if (MODE & kStats) {
            unsigned s = 0, s2 = 0, mn = 255, mx = 0, adx = 0, ady = 0, dx2 = 0, dy2 = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int p = sample(pix, r, c);
                    s += p;
                    s2 += p * p;
                    mn = min(mn, (unsigned)p);
                    mx = max(mx, (unsigned)p);
                    if (c < 7) {
                        const int d = sample(pix, r, c + 1) - p;
                        adx += abs(d);
                        dx2 += d * d;
                    }
                    if (r < 7) {
                        const int d = sample(pix, r + 1, c) - p;
                        ady += abs(d);
                        dy2 += d * d;
                    }
                }
            }
            if (!active) { s = s2 = adx = ady = dx2 = dy2 = 0; mn = 255; mx = 0; }
            const unsigned vals[8] = {warp_sum(s), warp_sum(s2), __reduce_min_sync(0xffffffffu, mn),
                                      __reduce_max_sync(0xffffffffu, mx), warp_sum(adx), warp_sum(ady),
                                      warp_sum(dx2), warp_sum(dy2)};
            if (lane == 0) {
                atomicAdd(&st[kStSum], (unsigned long long)vals[0]);
                atomicAdd(&st[kStSum2], (unsigned long long)vals[1]);
                atomicMin(&st[kStMin], (unsigned long long)vals[2]);
                atomicMax(&st[kStMax], (unsigned long long)vals[3]);
                atomicAdd(&st[kStAbsDx], (unsigned long long)vals[4]);
                atomicAdd(&st[kStAbsDy], (unsigned long long)vals[5]);
                atomicAdd(&st[kStDx2], (unsigned long long)vals[6]);
                atomicAdd(&st[kStDy2], (unsigned long long)vals[7]);
                atomicAdd(&st[kStBlocks], (unsigned long long)nvalid);
                atomicAdd(&st[kStSamples], (unsigned long long)nvalid * 64ull);
            }
        }

        // level shift: x = (p - 128) << P
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[r][c] = (sample(pix, r, c) - 128) * (1 << kP);

        fwd2d(x);

        if (MODE & kStats) {
            unsigned ac = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const unsigned a = (unsigned)abs(x[u][v]) >> kBandShift;
                    const unsigned e = active ? a * a : 0u;
                    if (u | v) ac += e;
                    const unsigned tot = warp_sum(e);
                    if (lane == 0) atomicAdd(&st[kStBand + u * 8 + v], (unsigned long long)tot);
                }
            }
            const unsigned thr[4] = {1u << 10, 1u << 14, 1u << 18, 1u << 22};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned n = warp_sum((active && ac < thr[k]) ? 1u : 0u);
                if (lane == 0) atomicAdd(&st[kStLowAc + k], (unsigned long long)n);
            }
        }

        // quantiser: q = sgn(Y) * ((|Y| * M + 2^31) >> 32)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int y = x[u][v];
                const uint32_t a = (uint32_t)abs(y);
                const uint32_t q = (uint32_t)(((unsigned long long)a * T.M[u * 8 + v] + 0x80000000ull) >> 32);
                x[u][v] = y < 0 ? -(int)q : (int)q;
            }
        }

        if (MODE & kStoreCoef) {
            uint8_t* mine = stage + lane * kStageStride;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint4 w;
                w.x = ((uint32_t)x[u][0] & 0xFFFFu) | ((uint32_t)x[u][1] << 16);
                w.y = ((uint32_t)x[u][2] & 0xFFFFu) | ((uint32_t)x[u][3] << 16);
                w.z = ((uint32_t)x[u][4] & 0xFFFFu) | ((uint32_t)x[u][5] << 16);
                w.w = ((uint32_t)x[u][6] & 0xFFFFu) | ((uint32_t)x[u][7] << 16);
                *reinterpret_cast<uint4*>(mine + 16 * u) = w;
            }
            __syncwarp();
            uint4* g = reinterpret_cast<uint4*>(P.coef + (size_t)b0 * 64);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = k * 32 + lane;
                const int blk = c >> 3;
                if (blk < nvalid) g[c] = *reinterpret_cast<const uint4*>(stage + blk * kStageStride + (c & 7) * 16);
            }
            __syncwarp();
        }
    }

    if (MODE & kLoadCoef) {
        const uint4* g = reinterpret_cast<const uint4*>(P.coef + (size_t)b0 * 64);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int c = k * 32 + lane;
            const int blk = c >> 3;
            if (blk < nvalid)
                *reinterpret_cast<uint4*>(stage + blk * kStageStride + (c & 7) * 16) = __ldg(g + c);
        }
        __syncwarp();
        const uint8_t* mine = stage + lane * kStageStride;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint4 w = *reinterpret_cast<const uint4*>(mine + 16 * u);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                x[u][2 * k] = (int)(int16_t)(ws[k] & 0xFFFFu);
                x[u][2 * k + 1] = (int)ws[k] >> 16;
            }
        }
        __syncwarp();
        if (!active) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) x[u][v] = 0;
        }
    }

    if (MODE & kInverse) {
        // dequantiser: G = clamp(q * Q, -4096, 4096) * W
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                int t = x[u][v] * T.Q[u * 8 + v];
                t = max(-kDequantClamp, min(kDequantClamp, t));
                x[u][v] = t * T.W[u * 8 + v];
            }
        }
        // The DC input reaches every output through additions only, so the
        // descale rounding term 2^(R+2) and the +128 level (128 << (R+3))
        // are added once here instead of at each of the 64 outputs.
        x[0][0] += (1 << (kR + 2)) + (128 << (kR + 3));
        inv2d(x);
        uint32_t out[8][2];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t wd = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int v = max(0, min(255, x[r][4 * h + k] >> (kR + 3)));
                    wd |= (uint32_t)v << (8 * k);
                }
                out[r][h] = wd;
            }
        }
        if ((MODE & kStoreRecon) && active)
            store_block(P.dst, P.dst_pitch, P.width, P.height, by, bx, (P.flags & kVecDst) != 0, out);

        if (MODE & kSse) {
            if (!(MODE & kLoadPix)) {
                if (active)
                    load_block(P.ref, P.ref_pitch, P.width, P.height, by, bx, (P.flags & kVecRef) != 0, pix);
            }
            unsigned e = 0;
            if (active) {
                const int nr = min(8, P.height - by * 8), nc = min(8, P.width - bx * 8);
                if (nr == 8 && nc == 8) {
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const int d = sample(out, r, c) - sample(pix, r, c);
                            e += d * d;
                        }
                } else {
                    for (int r = 0; r < nr; ++r)
                        for (int c = 0; c < nc; ++c) {
                            const int d = sample(out, r, c) - sample(pix, r, c);
                            e += d * d;
                        }
                }
            }
            return warp_sum(e);
        }
    }
    return 0u;
}

// --------------------------------------------------------------------------
// persistent kernel over all tiles of up to kMaxPlanes planes
// --------------------------------------------------------------------------

template <unsigned MODE>
__global__ void __launch_bounds__(256) k_codec(const __grid_constant__ DirectArgs args) {
    extern __shared__ __align__(16) uint8_t smem[];
    QuantSet* tabs = reinterpret_cast<QuantSet*>(smem);                       // 2 sets
    CtaAcc* acc = reinterpret_cast<CtaAcc*>(smem + 2 * sizeof(QuantSet));
    uint8_t* stage_all = smem + 2 * sizeof(QuantSet) + sizeof(CtaAcc);

    // tables -> shared memory
    {
        const uint32_t* s = reinterpret_cast<const uint32_t*>(args.tabs);
        uint32_t* d = reinterpret_cast<uint32_t*>(tabs);
        for (int i = threadIdx.x; i < (int)(2 * sizeof(QuantSet) / 4); i += blockDim.x) d[i] = s[i];
        unsigned long long* a = reinterpret_cast<unsigned long long*>(acc);
        for (int i = threadIdx.x; i < (int)(sizeof(CtaAcc) / 8); i += blockDim.x) a[i] = 0ull;
        __syncthreads();
        if (MODE & kStats)
            if (threadIdx.x < kMaxPlanes) acc->st[threadIdx.x][kStMin] = ~0ull;
        __syncthreads();
    }

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint8_t* stage = stage_all + warp * kStageBytesPerWarp;
    const int warps_per_cta = blockDim.x >> 5;
    const int total_warps = gridDim.x * warps_per_cta;

    for (int tile = blockIdx.x * warps_per_cta + warp; tile < args.ntiles; tile += total_warps) {
        int pi = 0;
#pragma unroll
        for (int k = 1; k < kMaxPlanes; ++k)
            if (k < args.nplanes && tile >= args.p[k].tile_begin) pi = k;
        const PlaneArg& P = args.p[pi];
        const unsigned e = process_tile<MODE>(P, tabs[P.table], tile - P.tile_begin, lane, stage, acc->st[pi]);
        if ((MODE & kSse) && lane == 0 && e) atomicAdd(&acc->sse[pi], (unsigned long long)e);
    }

    __syncthreads();
    if (MODE & kSse) {
        if (threadIdx.x < args.nplanes && acc->sse[threadIdx.x])
            atomicAdd(args.p[threadIdx.x].sse, acc->sse[threadIdx.x]);
    }
    if (MODE & kStats) {
        for (int i = threadIdx.x; i < args.nplanes * kStatsWords; i += blockDim.x) {
            const int pl = i / kStatsWords, w = i - pl * kStatsWords;
            const unsigned long long v = acc->st[pl][w];
            unsigned long long* g = args.p[pl].stats + w;
            if (w == kStMin) {
                if (v != ~0ull) atomicMin(g, v);
            } else if (w == kStMax) {
                atomicMax(g, v);
            } else if (v) {
                atomicAdd(g, v);
            }
        }
    }
}

// zero the SSE words and the statistics (min words to all ones)
__global__ void k_init_acc(DirectArgs args, int do_sse, int do_stats);

inline size_t codec_smem_bytes(int threads) {
    return 2 * sizeof(QuantSet) + sizeof(CtaAcc) + (size_t)(threads / 32) * kStageBytesPerWarp;
}

// Persistent grid: enough CTAs for every tile, at most num_sms * occupancy.
inline int persistent_grid(int ntiles, int threads, int num_sms, int occ) {
    const int warps = threads / 32;
    const int need = (ntiles + warps - 1) / warps;
    const int cap = num_sms * (occ > 0 ? occ : 1);
    return need < 1 ? 1 : (need < cap ? need : cap);
}

// host launchers (one translation unit per family); kDirectThreads per CTA
constexpr int kDirectThreads = 256;
cudaError_t launch_compress(const DirectArgs& a, bool stats, int num_sms, int threads, cudaStream_t s);
cudaError_t launch_reconstruct(const DirectArgs& a, bool sse, int num_sms, int threads, cudaStream_t s);
cudaError_t launch_fused(const DirectArgs& a, bool coef, bool recon, int num_sms, int threads, cudaStream_t s);

}  // namespace dctgb
