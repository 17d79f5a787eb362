// Codec kernels: forward path (Sec. 2.5.2 transform + Sec. 3.2 quantiser),
// inverse path (Sec. 3.2 dequantiser + IDCT) and the SSE of Eq. 24, for
// uint8 planes, all in integer arithmetic.
//
// Work decomposition: a plane of nbx x nby 8x8 blocks is cut into warp tiles
// of kTileBlocks consecutive blocks in block-major order (b = by * nbx + bx,
// wrapping across block rows).  Lane l of a warp owns block b0 + l and keeps
// its 64 samples in registers, so the row/column transpose between the two
// 1-D passes is free.  Pixel rows move 8 bytes per lane (a warp covers 256
// contiguous bytes of an image row); int16 coefficients go through a
// swizzled per-warp shared-memory stage so the global side moves 16 bytes
// per lane over contiguous 512-byte spans.  The batched kernel prefetches
// the next tile's pixels / coefficients with cp.async while the current
// tile computes.  The path is bound by integer issue, not by HBM, so the
// code is arranged to minimise instructions per sample.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cordic_loeffler.cuh"
#include "dctgb_spec.h"

#ifndef DCTGB_MINB
#define DCTGB_MINB 2        // minimum resident CTAs per SM (launch bounds: <= 128 registers)
#endif

namespace dctgb {

constexpr int kMaxPlanes = 4;
constexpr int kTileBlocks = 32;                   // blocks per warp tile (one per lane)
constexpr int kStageBytes = kTileBlocks * 128;    // one tile of int16 coefficients
constexpr int kPixBytes = kTileBlocks * 64;       // one tile of uint8 samples

// Per-plane quantiser / dequantiser tables (natural order u*8+v).
struct QuantSet {
    uint32_t M[64];   // rint(2^32 / (8 * 2^P * g_u g_v Q))
    int32_t Q[64];    // 1..255
    int32_t W[64];    // rint(2^R / (g_u g_v))
    int32_t QW[64];   // Q * W
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

// Mode bits of the kernel templates.
enum : unsigned {
    kLoadPix = 1u,     // read samples, forward transform, quantise
    kStoreCoef = 2u,   // write the quantised coefficients
    kLoadCoef = 4u,    // read quantised coefficients
    kInverse = 8u,     // dequantise, inverse transform, descale
    kStoreRecon = 16u, // write the reconstruction
    kSse = 32u,        // accumulate the SSE
    kStats = 64u,      // accumulate band-energy and pixel statistics
    kStatsPrivate = 128u, // the statistics sink is this warp's own: plain adds, no atomics
    kOwnCodes = 256u      // the coefficients read back are this library's own codes, written by the
                          // forward kernel of the same graph: the dequantiser clamp never acts
};

// Forward micro-rotations 2..N in the float form (cordic_loeffler.cuh) for
// kernels that run the forward transform without the inverse: measured on
// the benchmark planes, the compress-only pass runs 5-7% faster with it
// (the FMA pipes take the shift-adds off the integer ALU pipe), while the
// fused forward + inverse kernel runs 1.7% slower (its instruction count
// falls only 1.6% and issue drops from 80.6% to 77.8% of cycles), so the
// fused kernels keep the integer form.
__host__ __device__ constexpr bool fwd_in_float(unsigned mode) { return (mode & kLoadPix) && !(mode & kInverse); }

// Quantiser entries that can meet an exact rounding tie.  The definition
// q = sgn(Y) ((|Y| M + 2^31) >> 32) equals the high word of the signed
// Y M + 2^31 for Y >= 0 always, and for Y < 0 unless |Y| M = 2^31 (mod 2^32),
// which needs |Y| = 2^(31-k) * odd, k = trailing zero bits of M.  The forward
// graph keeps |Y| <= 719380 < 2^20 (interval bound), so an entry with k <= 11
// never ties.  Where u and v are both 0 or 4, g_u g_v = 1 and
// M = rint(2^25 / Q) is a high power of two for Q = 1, 2, 4, ...: these four
// entries keep the sign-aware form.  For the other 60, every Q in 1..255
// gives k <= 11 (build_tables checks each table), so the plain high word is
// the exact quantiser there: one 64-bit multiply-add per coefficient.
__host__ __device__ constexpr bool tie_entry(int u, int v) { return (u & 3) == 0 && (v & 3) == 0; }
constexpr uint32_t kTieFreeBits = 0xFFFu;   // (M & kTieFreeBits) != 0  <=>  k <= 11

// Clamp to 0..255 in one instruction: max(min(v, 255), 0).
__device__ __forceinline__ int clamp_u8(int v) { return __vimin_s32_relu(v, 255); }

// statistics word layout (per plane)
enum : int {
    kStBand = 0,         // 64 words: sum over blocks of (|Y_uv| >> kBandShift)^2
    kStSum = 64, kStSum2 = 65, kStMin = 66, kStMax = 67,
    kStAbsDx = 68, kStAbsDy = 69, kStDx2 = 70, kStDy2 = 71,
    kStLowAc = 72,       // 4 words: blocks whose AC energy < 2^10, 2^14, 2^18, 2^22
    kStBlocks = 76, kStSamples = 77
};

// --------------------------------------------------------------------------
// shared-memory layouts (swizzled, conflict-free for both access patterns)
// --------------------------------------------------------------------------

// Coefficient stage: block `blk` occupies 128 bytes; its row u (8 int16) sits
// in 16-byte slot u ^ (blk & 7).  A lane writing/reading the 8 rows of its own
// block and 8 lanes reading one block's 8 slots both hit 8 distinct
// 16-byte bank groups.
__device__ __forceinline__ int stage_off(int blk, int row) { return blk * 128 + ((row ^ (blk & 7)) << 4); }

// Pixel buffer: lane l's 8 rows of 8 bytes at l * 64; row r in 8-byte slot
// r ^ ((l >> 1) & 7), so 16 lanes reading one row each touch 32 distinct banks.
__device__ __forceinline__ int pix_off(int lane, int r) { return lane * 64 + ((r ^ ((lane >> 1) & 7)) << 3); }

// --------------------------------------------------------------------------
// asynchronous copies (completion via cp.async.wait_group: no spin loops)
// --------------------------------------------------------------------------

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// --------------------------------------------------------------------------
// sample I/O
// --------------------------------------------------------------------------

__device__ __forceinline__ bool interior(const PlaneArg& P, int by, int bx) {
    return bx * 8 + 8 <= P.width && by * 8 + 8 <= P.height;
}

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

// Issues cp.async copies of this lane's block of tile `tile_in_plane` into
// `buf` (a kPixBytes region) when the block is interior and the plane's rows
// are 8-byte aligned; the consumer re-evaluates the same condition.
__device__ __forceinline__ void prefetch_block(const PlaneArg& P, const uint8_t* base, int pitch, int vec_flag,
                                               int tile_in_plane, int lane, uint8_t* buf) {
    const int b = tile_in_plane * kTileBlocks + lane;
    if (b < P.nblk && (P.flags & vec_flag)) {
        const int by = b / P.nbx, bx = b - by * P.nbx;
        if (interior(P, by, bx)) {
            const uint8_t* p = base + (size_t)(by * 8) * pitch + bx * 8;
#pragma unroll
            for (int r = 0; r < 8; ++r) cp_async8(buf + pix_off(lane, r), p + (size_t)r * pitch);
        }
    }
}

// Issues cp.async copies of tile `tile_in_plane`'s coefficients into `stage`.
__device__ __forceinline__ void prefetch_coef(const PlaneArg& P, int tile_in_plane, int lane, uint8_t* stage) {
    const int b0 = tile_in_plane * kTileBlocks;
    const int nvalid = min(kTileBlocks, P.nblk - b0);
    const uint8_t* g = reinterpret_cast<const uint8_t*>(P.coef + (size_t)b0 * 64);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int c = k * 32 + lane;
        const int blk = c >> 3;
        if (blk < nvalid) cp_async16(stage + stage_off(blk, c & 7), g + (size_t)c * 16);
    }
}

// Block samples from the prefetch buffer when they were prefetched, else from
// global memory (edge blocks, unaligned planes, first tile of an item).
__device__ __forceinline__ void fetch_block(const PlaneArg& P, const uint8_t* base, int pitch, int vec_flag,
                                            const uint8_t* buf, int lane, int by, int bx, uint32_t (&pix)[8][2]) {
    if (buf && (P.flags & vec_flag) && interior(P, by, bx)) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint2 v = *reinterpret_cast<const uint2*>(buf + pix_off(lane, r));
            pix[r][0] = v.x;
            pix[r][1] = v.y;
        }
    } else {
        load_block(base, pitch, P.width, P.height, by, bx, (P.flags & vec_flag) != 0, pix);
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

__device__ __forceinline__ unsigned warp_sum(unsigned v) { return __reduce_add_sync(0xffffffffu, v); }

// statistics sink updates: atomics when the sink is shared, plain
// read-modify-write when it belongs to the calling warp
template <unsigned MODE>
__device__ __forceinline__ void st_add(unsigned long long* p, unsigned long long v) {
    if (MODE & kStatsPrivate) *p += v;
    else atomicAdd(p, v);
}
template <unsigned MODE>
__device__ __forceinline__ void st_min(unsigned long long* p, unsigned long long v) {
    if (MODE & kStatsPrivate) *p = *p < v ? *p : v;
    else atomicMin(p, v);
}
template <unsigned MODE>
__device__ __forceinline__ void st_max(unsigned long long* p, unsigned long long v) {
    if (MODE & kStatsPrivate) *p = *p > v ? *p : v;
    else atomicMax(p, v);
}

// Shared memory a warp needs in a given mode (batched kernel): its item's
// tables and descriptor, double-buffered samples and coefficient stages.
constexpr int kDescBytes = 128;
static_assert(sizeof(PlaneArg) <= kDescBytes, "descriptor slot too small");
constexpr int kStatBytes = kStatsWords * 8;   // warp-private statistics accumulator
__host__ __device__ constexpr int warp_smem_bytes(unsigned mode) {
    return (int)sizeof(QuantSet) + kDescBytes + ((mode & kStats) ? kStatBytes : 0) +
           (((mode & kLoadPix) || (mode & kSse)) ? 2 * kPixBytes : 0) +
           ((mode & kLoadCoef) ? 2 * kStageBytes : ((mode & kStoreCoef) ? kStageBytes : 0));
}

// --------------------------------------------------------------------------
// one warp tile
// --------------------------------------------------------------------------

// Processes warp tile `tile_in_plane` of plane P.
//  stage      kStageBytes of this warp's shared memory (coefficients)
//  pixbuf     this tile's prefetched samples (forward) or SSE reference
//             (inverse), or nullptr
//  coef_ready the stage already holds this tile's coefficients
// Statistics go to the 80 words at `st` (shared or global); the return value
// is the tile's SSE (the same in every lane; 0 without kSse).
template <unsigned MODE>
__device__ __forceinline__ unsigned process_tile(const PlaneArg& P, const QuantSet& T, int tile_in_plane, int lane,
                                                 uint8_t* stage, const uint8_t* pixbuf, bool coef_ready,
                                                 unsigned long long* st) {
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
            fetch_block(P, P.src, P.src_pitch, kVecSrc, pixbuf, lane, by, bx, pix);
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
                st_add<MODE>(&st[kStSum], vals[0]);
                st_add<MODE>(&st[kStSum2], vals[1]);
                st_min<MODE>(&st[kStMin], vals[2]);
                st_max<MODE>(&st[kStMax], vals[3]);
                st_add<MODE>(&st[kStAbsDx], vals[4]);
                st_add<MODE>(&st[kStAbsDy], vals[5]);
                st_add<MODE>(&st[kStDx2], vals[6]);
                st_add<MODE>(&st[kStDy2], vals[7]);
                st_add<MODE>(&st[kStBlocks], (unsigned long long)nvalid);
                st_add<MODE>(&st[kStSamples], (unsigned long long)nvalid * 64ull);
            }
        }

        // level shift: x = (p - 128) << P
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[r][c] = (sample(pix, r, c) - 128) * (1 << kP);

        fwd2d<fwd_in_float(MODE)>(x);

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
                    if (lane == 0) st_add<MODE>(&st[kStBand + u * 8 + v], tot);
                }
            }
            const unsigned thr[4] = {1u << 10, 1u << 14, 1u << 18, 1u << 22};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned n = warp_sum((active && ac < thr[k]) ? 1u : 0u);
                if (lane == 0) st_add<MODE>(&st[kStLowAc + k], n);
            }
        }

        // Quantiser q = sgn(Y) ((|Y| M + 2^31) >> 32).  Away from the four
        // tie entries the high word of Y M + 2^31 is exact (tie_entry).  At
        // the tie entries the fused kernels use the high word of the signed
        // Y * M + 2^31 - [Y < 0] (for Y < 0, floor((Y M + 2^31 - 1) / 2^32) =
        // -floor((|Y| M + 2^31) / 2^32), so both signs round half away from
        // zero exactly as the definition); the forward-only kernels use |Y|,
        // an unsigned multiply and the sign.
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int y = x[u][v];
                if (!tie_entry(u, v)) {
                    const long long p = (long long)y * (long long)(int)T.M[u * 8 + v] + 0x80000000ll;
                    x[u][v] = (int)(p >> 32);
                } else if (MODE & kInverse) {
                    const unsigned c = 0x80000000u ^ (unsigned)(y >> 31);
                    const long long p = (long long)y * (long long)(int)T.M[u * 8 + v] + (long long)c;
                    x[u][v] = (int)(p >> 32);
                } else {
                    const uint32_t a = (uint32_t)abs(y);
                    const uint32_t q = (uint32_t)(((unsigned long long)a * T.M[u * 8 + v] + 0x80000000ull) >> 32);
                    x[u][v] = y < 0 ? -(int)q : (int)q;
                }
            }
        }

        if (MODE & kStoreCoef) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint4 w;
                w.x = ((uint32_t)x[u][0] & 0xFFFFu) | ((uint32_t)x[u][1] << 16);
                w.y = ((uint32_t)x[u][2] & 0xFFFFu) | ((uint32_t)x[u][3] << 16);
                w.z = ((uint32_t)x[u][4] & 0xFFFFu) | ((uint32_t)x[u][5] << 16);
                w.w = ((uint32_t)x[u][6] & 0xFFFFu) | ((uint32_t)x[u][7] << 16);
                *reinterpret_cast<uint4*>(stage + stage_off(lane, u)) = w;
            }
            __syncwarp();
            uint4* g = reinterpret_cast<uint4*>(P.coef + (size_t)b0 * 64);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = k * 32 + lane;
                const int blk = c >> 3;
                if (blk < nvalid) g[c] = *reinterpret_cast<const uint4*>(stage + stage_off(blk, c & 7));
            }
            __syncwarp();
        }
    }

    if (MODE & kLoadCoef) {
        if (!coef_ready) {
            const uint4* g = reinterpret_cast<const uint4*>(P.coef + (size_t)b0 * 64);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = k * 32 + lane;
                const int blk = c >> 3;
                if (blk < nvalid) *reinterpret_cast<uint4*>(stage + stage_off(blk, c & 7)) = __ldg(g + c);
            }
            __syncwarp();
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint4 w = *reinterpret_cast<const uint4*>(stage + stage_off(lane, u));
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                x[u][2 * k] = (int)(int16_t)(ws[k] & 0xFFFFu);
                x[u][2 * k + 1] = (int)ws[k] >> 16;
            }
        }
        if (!active) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) x[u][v] = 0;
        }
    }

    if (MODE & kInverse) {
        // Dequantiser G = clamp(q Q, -4096, 4096) W.  When q comes from this
        // library's quantiser (this kernel's, or the forward kernel's of the
        // same two-pass graph), |q Q| <= |X| + Q/2 + 1 < 1200 (the Cordic
        // coefficient |X| is within 14 of an orthonormal DCT value, itself at
        // most 1024), so the clamp never acts and G = q (Q W) exactly.
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                if (MODE & (kLoadPix | kOwnCodes)) {
                    x[u][v] = x[u][v] * T.QW[u * 8 + v];
                } else {
                    int t = x[u][v] * T.Q[u * 8 + v];
                    t = max(-kDequantClamp, min(kDequantClamp, t));
                    x[u][v] = t * T.W[u * 8 + v];
                }
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
                    const int v = clamp_u8(x[r][4 * h + k] >> (kR + 3));
                    wd |= (uint32_t)v << (8 * k);
                }
                out[r][h] = wd;
            }
        }
        if ((MODE & kStoreRecon) && active)
            store_block(P.dst, P.dst_pitch, P.width, P.height, by, bx, (P.flags & kVecDst) != 0, out);

        if (MODE & kSse) {
            if (!(MODE & kLoadPix) && active) fetch_block(P, P.ref, P.ref_pitch, kVecRef, pixbuf, lane, by, bx, pix);
            unsigned e = 0;
            if (active) {
                const int nr = min(8, P.height - by * 8), nc = min(8, P.width - bx * 8);
                if (nr == 8 && nc == 8) {
                    // |r - p| per byte (vabsdiffu4), then the four squares and their
                    // sum in one dp4a
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const unsigned ad = __vabsdiffu4(out[r][h], pix[r][h]);
                            e = __dp4a(ad, ad, e);
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
// persistent kernel over all tiles of up to kMaxPlanes planes (direct calls)
// --------------------------------------------------------------------------

struct CtaAcc {
    unsigned long long sse[kMaxPlanes];
    unsigned long long st[kMaxPlanes][kStatsWords];
};

template <unsigned MODE>
__global__ void __launch_bounds__(256, DCTGB_MINB) k_codec(const __grid_constant__ DirectArgs args) {
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
    uint8_t* stage = stage_all + warp * kStageBytes;
    const int warps_per_cta = blockDim.x >> 5;
    const int total_warps = gridDim.x * warps_per_cta;

    for (int tile = blockIdx.x * warps_per_cta + warp; tile < args.ntiles; tile += total_warps) {
        int pi = 0;
#pragma unroll
        for (int k = 1; k < kMaxPlanes; ++k)
            if (k < args.nplanes && tile >= args.p[k].tile_begin) pi = k;
        const PlaneArg& P = args.p[pi];
        const unsigned e = process_tile<MODE>(P, tabs[P.table], tile - P.tile_begin, lane, stage, nullptr, false,
                                              acc->st[pi]);
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
    return 2 * sizeof(QuantSet) + sizeof(CtaAcc) + (size_t)(threads / 32) * kStageBytes;
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
