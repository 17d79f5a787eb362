// Codec tile with two lanes per 8x8 block: the fused pass, the forward pass
// alone and the inverse pass alone.
//
// The one-lane-per-block tile (kernels.cuh) keeps all 64 samples of a block
// in one thread, which makes the row/column transpose free but needs about
// 128 registers, so only 16 warps fit on an SM; the path is bound by integer
// issue, and 16 warps leave about a quarter of the issue slots idle on
// dependency and pipe-throttle stalls.  Here lanes 2k and 2k+1 share block k
// of a 16-block half tile: lane h owns rows 4h..4h+3 for the row passes and
// columns 4h..4h+3 for the column passes, 32 values in registers, and the two
// transposes go through a padded per-warp shared-memory slot (8 stores and 8
// loads of 16 bytes per lane each, no bank conflicts).  To stay within 64
// registers with few spills, the samples wait for the SSE in a per-lane
// shared-memory slot, and the coefficients go straight from registers to
// global memory (8 bytes per lane and row: the lane pair fills the row's 16
// bytes).  The arithmetic is the same integer graph in the same order as the
// one-lane tile, so every output is bit-identical to it.
//
// Transpose slot of block k (kXSlot bytes): row r, column quad q (columns
// 4q..4q+3, four int32) at k*kXSlot + (r>>2)*kXRowHalf + (r&3)*32 + q*16.
// With kXSlot/16 = 2 and kXRowHalf/16 = 1 (mod 8), the 16-byte bank group of
// an access is (lane + const) mod 8 both when lane h writes its rows and when
// it reads its column quad, so each quarter-warp phase hits 8 distinct
// groups.
#pragma once
#include "kernels.cuh"

#ifndef DCTGB_PAIR_MINB
#define DCTGB_PAIR_MINB 4   // resident CTAs of 256 threads per SM (launch bounds: <= 64 registers)
#endif

namespace dctgb {

constexpr int kPairBlocks = kTileBlocks / 2;      // blocks per half tile
constexpr int kXSlot = 288;                       // transpose bytes per block
constexpr int kXRowHalf = 144;                    // offset of rows 4..7 in a slot
constexpr int kXBytes = kPairBlocks * kXSlot;     // per warp
constexpr int kParkBytes = 32 * 32;               // each lane's 32 samples, kept for the SSE

// Shared memory per warp of the two-lane batched kernel: tables, descriptor,
// transpose buffer, sample slots.
__host__ __device__ constexpr int pair_warp_smem_bytes() {
    return (int)sizeof(QuantSet) + kDescBytes + kXBytes + kParkBytes;
}

// The two-lane tile implements the fused modes (samples in, inverse out),
// the forward pass alone (samples in, coefficients out) and the inverse pass
// alone (coefficients in, reconstruction and/or SSE out); the statistics
// modes keep the one-lane tile.
__host__ __device__ constexpr bool pair_mode_supported(unsigned mode) {
    return !(mode & (kStats | kStatsPrivate)) &&
           (((mode & kLoadPix) && !(mode & kLoadCoef) && ((mode & kInverse) || mode == (kLoadPix | kStoreCoef))) ||
            ((mode & kLoadCoef) && (mode & kInverse) && !(mode & (kLoadPix | kStoreCoef))));
}

// Loads rows 4h..4h+3 of block (by, bx) as two little-endian words each,
// with edge replication outside the plane.
__device__ __forceinline__ void load_rows4(const uint8_t* __restrict__ src, int pitch, int w, int hgt,
                                           int by, int bx, int h, bool vec, uint32_t (&pix)[4][2]) {
    const int x0 = bx * 8, y0 = by * 8 + 4 * h;
    if (vec && x0 + 8 <= w && by * 8 + 8 <= hgt) {
        const uint8_t* p = src + (size_t)y0 * pitch + x0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(p + (size_t)j * pitch));
            pix[j][0] = v.x;
            pix[j][1] = v.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int yy = min(y0 + j, hgt - 1);
            const uint8_t* row = src + (size_t)yy * pitch;
            uint32_t wd[2] = {0u, 0u};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int xx = min(x0 + c, w - 1);
                wd[c >> 2] |= (uint32_t)__ldg(row + xx) << (8 * (c & 3));
            }
            pix[j][0] = wd[0];
            pix[j][1] = wd[1];
        }
    }
}

// Stores the in-plane part of rows 4h..4h+3 of block (by, bx).
__device__ __forceinline__ void store_rows4(uint8_t* __restrict__ dst, int pitch, int w, int hgt,
                                            int by, int bx, int h, bool vec, const uint32_t (&pix)[4][2]) {
    const int x0 = bx * 8, y0 = by * 8 + 4 * h;
    if (vec && x0 + 8 <= w && by * 8 + 8 <= hgt) {
        uint8_t* p = dst + (size_t)y0 * pitch + x0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<uint2*>(p + (size_t)j * pitch) = make_uint2(pix[j][0], pix[j][1]);
    } else {
        const int nr = min(4, hgt - y0), nc = min(8, w - x0);
        for (int j = 0; j < nr; ++j) {
            uint8_t* row = dst + (size_t)(y0 + j) * pitch + x0;
            for (int c = 0; c < nc; ++c) row[c] = (uint8_t)(pix[j][c >> 2] >> (8 * (c & 3)));
        }
    }
}

__device__ __forceinline__ int sample4(const uint32_t (&pix)[4][2], int j, int c) {
    return (int)((pix[j][c >> 2] >> (8 * (c & 3))) & 0xFFu);
}

__device__ __forceinline__ void sts128(uint8_t* p, int a, int b, int c, int d) {
    *reinterpret_cast<int4*>(p) = make_int4(a, b, c, d);
}
__device__ __forceinline__ int4 lds128(const uint8_t* p) { return *reinterpret_cast<const int4*>(p); }

// A lane's four sample rows in its 32-byte slot; the halves swap on every
// fourth lane so a quarter warp's 16-byte accesses hit distinct bank groups.
__device__ __forceinline__ void park_rows(uint8_t* slot, int sw, const uint32_t (&pix)[4][2]) {
    *reinterpret_cast<uint4*>(slot + 16 * sw) = make_uint4(pix[0][0], pix[0][1], pix[1][0], pix[1][1]);
    *reinterpret_cast<uint4*>(slot + 16 * (sw ^ 1)) = make_uint4(pix[2][0], pix[2][1], pix[3][0], pix[3][1]);
}
__device__ __forceinline__ void unpark_rows(const uint8_t* slot, int sw, uint32_t (&pix)[4][2]) {
    const uint4 a = *reinterpret_cast<const uint4*>(slot + 16 * sw);
    const uint4 b = *reinterpret_cast<const uint4*>(slot + 16 * (sw ^ 1));
    pix[0][0] = a.x; pix[0][1] = a.y; pix[1][0] = a.z; pix[1][1] = a.w;
    pix[2][0] = b.x; pix[2][1] = b.y; pix[3][0] = b.z; pix[3][1] = b.w;
}

// Processes warp tile `tile_in_plane` of plane P (two half tiles of 16
// blocks).  xb is this warp's kXBytes transpose buffer followed by its
// kParkBytes sample slots.  Returns the tile's SSE (the same in every lane;
// 0 without kSse).
template <unsigned MODE>
__device__ __forceinline__ unsigned process_tile_pair(const PlaneArg& P, const QuantSet& T, int tile_in_plane,
                                                      int lane, uint8_t* xb) {
    static_assert(pair_mode_supported(MODE), "no two-lane form of this mode");
    const int k = lane >> 1, h = lane & 1;
    uint8_t* const xw = xb + k * kXSlot + h * kXRowHalf;   // rows 4h..4h+3, both quads
    uint8_t* const xr = xb + k * kXSlot + h * 16;           // rows 0..7, quad h
    // descale rounding term and +128 level, added once to the DC input
    // (column 0 belongs to lane h = 0)
    const int dc_bias = h ? 0 : (1 << (kR + 2)) + (128 << (kR + 3));
    const int32_t* Mh = reinterpret_cast<const int32_t*>(T.M) + 4 * h;
    const int32_t* QWh = T.QW + 4 * h;
    const int32_t* Qh = T.Q + 4 * h;
    const int32_t* Wh = T.W + 4 * h;
    uint8_t* const park = xb + kXBytes + lane * 32;
    const int psw = (lane >> 2) & 1;
    unsigned e = 0;
    // block coordinates: one division per tile, then steps of 16 blocks
    const int bt = tile_in_plane * kTileBlocks;
    const int by_t = bt / P.nbx;
    const int bx_t = bt - by_t * P.nbx;

#pragma unroll 1
    for (int hf = 0; hf < 2; ++hf) {
        const int b0 = bt + hf * kPairBlocks;
        const int nvalid = min(kPairBlocks, P.nblk - b0);
        if (nvalid <= 0) break;                      // warp-uniform
        const bool active = k < nvalid;
        int by = by_t, bx = bx_t + hf * kPairBlocks + k;
        if (bx >= P.nbx) {
            bx -= P.nbx;
            ++by;
            if (bx >= P.nbx) {                       // planes narrower than 32 blocks
                by += bx / P.nbx;
                bx -= (bx / P.nbx) * P.nbx;
            }
        }

        int v[4][8];
        int c[4][8];
        uint32_t pix[4][2];
        if (MODE & kLoadPix) {
            // level shift and row pass on rows 4h..4h+3
            if (active) {
                load_rows4(P.src, P.src_pitch, P.width, P.height, by, bx, h, (P.flags & kVecSrc) != 0, pix);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) pix[j][0] = pix[j][1] = 0x80808080u;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int col = 0; col < 8; ++col) v[j][col] = (sample4(pix, j, col) - 128) * (1 << kP);
#pragma unroll
            for (int j = 0; j < 4; ++j) loeffler8_fwd<false>(v[j]);

            // the samples wait for the SSE in this lane's slot (the two 16-byte
            // halves swap on every fourth lane: no bank conflicts)
            if (MODE & kSse) park_rows(park, psw, pix);

            // transpose: rows 4h..4h+3 out, columns 4h..4h+3 in
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                sts128(xw + j * 32, v[j][0], v[j][1], v[j][2], v[j][3]);
                sts128(xw + j * 32 + 16, v[j][4], v[j][5], v[j][6], v[j][7]);
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int4 t = lds128(xr + (r >> 2) * kXRowHalf + (r & 3) * 32);
                c[0][r] = t.x;
                c[1][r] = t.y;
                c[2][r] = t.z;
                c[3][r] = t.w;
            }

            // column pass: c[i][u] = Y[u][4h + i]
#pragma unroll
            for (int i = 0; i < 4; ++i) loeffler8_fwd<false>(c[i]);

            // quantiser: high word of Y M + 2^31, with - [Y < 0] at the tie
            // entries (u, v in {0, 4}: i = 0 and u = 0 or 4 in both lanes)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int4 m = *reinterpret_cast<const int4*>(Mh + u * 8);
                const int mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int y = c[i][u];
                    long long p = (long long)y * (long long)mv[i] + 0x80000000ll;
                    if (tie_entry(u, i)) p += (long long)(y >> 31);
                    c[i][u] = (int)(p >> 32);
                }
            }

            // coefficients: row u of the block is 16 bytes, lane h writes its half
            if ((MODE & kStoreCoef) && active) {
                uint2* g = reinterpret_cast<uint2*>(P.coef + (size_t)(b0 + k) * 64 + 4 * h);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    g[2 * u] = make_uint2(((uint32_t)c[0][u] & 0xFFFFu) | ((uint32_t)c[1][u] << 16),
                                          ((uint32_t)c[2][u] & 0xFFFFu) | ((uint32_t)c[3][u] << 16));
            }
            // dequantiser G = q (Q W): the clamp of the definition never acts
            // on this kernel's own codes (|q Q| < 1200)
            if (MODE & kInverse) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int4 qw = *reinterpret_cast<const int4*>(QWh + u * 8);
                    c[0][u] *= qw.x;
                    c[1][u] *= qw.y;
                    c[2][u] *= qw.z;
                    c[3][u] *= qw.w;
                }
            }
        } else {
            // coefficients in: lane h reads the 8-byte half of each row u; the
            // SSE reference rows wait in its slot
            if (active) {
                const uint2* g = reinterpret_cast<const uint2*>(P.coef + (size_t)(b0 + k) * 64 + 4 * h);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint2 w = __ldg(g + 2 * u);
                    c[0][u] = (int)(int16_t)(w.x & 0xFFFFu);
                    c[1][u] = (int)w.x >> 16;
                    c[2][u] = (int)(int16_t)(w.y & 0xFFFFu);
                    c[3][u] = (int)w.y >> 16;
                }
                if (MODE & kSse) {
                    load_rows4(P.ref, P.ref_pitch, P.width, P.height, by, bx, h, (P.flags & kVecRef) != 0, pix);
                    park_rows(park, psw, pix);
                }
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) c[0][u] = c[1][u] = c[2][u] = c[3][u] = 0;
            }
            if constexpr ((MODE & kOwnCodes) != 0) {
                // this library's own codes (two-pass graph): G = q (Q W), the
                // clamp never acts (|q Q| < 1200)
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int4 qw = *reinterpret_cast<const int4*>(QWh + u * 8);
                    c[0][u] *= qw.x;
                    c[1][u] *= qw.y;
                    c[2][u] *= qw.z;
                    c[3][u] *= qw.w;
                }
            } else {
                // dequantiser G = clamp(q Q, -4096, 4096) W for arbitrary codes
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int4 q4 = *reinterpret_cast<const int4*>(Qh + u * 8);
                    const int4 w4 = *reinterpret_cast<const int4*>(Wh + u * 8);
                    c[0][u] = max(-kDequantClamp, min(kDequantClamp, c[0][u] * q4.x)) * w4.x;
                    c[1][u] = max(-kDequantClamp, min(kDequantClamp, c[1][u] * q4.y)) * w4.y;
                    c[2][u] = max(-kDequantClamp, min(kDequantClamp, c[2][u] * q4.z)) * w4.z;
                    c[3][u] = max(-kDequantClamp, min(kDequantClamp, c[3][u] * q4.w)) * w4.w;
                }
            }
        }
        if constexpr ((MODE & kInverse) != 0) {
            c[0][0] += dc_bias;

            // inverse column pass, transpose back, inverse row pass
#pragma unroll
            for (int i = 0; i < 4; ++i) loeffler8_inv(c[i]);
            __syncwarp();                                // transpose reads done
#pragma unroll
            for (int r = 0; r < 8; ++r)
                sts128(xr + (r >> 2) * kXRowHalf + (r & 3) * 32, c[0][r], c[1][r], c[2][r], c[3][r]);
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int4 a = lds128(xw + j * 32);
                const int4 b = lds128(xw + j * 32 + 16);
                v[j][0] = a.x; v[j][1] = a.y; v[j][2] = a.z; v[j][3] = a.w;
                v[j][4] = b.x; v[j][5] = b.y; v[j][6] = b.z; v[j][7] = b.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) loeffler8_inv(v[j]);

            // descale, clamp, pack
            uint32_t out[4][2];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    uint32_t wd = 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int s = clamp_u8(v[j][4 * q + t] >> (kR + 3));
                        wd |= (uint32_t)s << (8 * t);
                    }
                    out[j][q] = wd;
                }
            }
            if ((MODE & kStoreRecon) && active)
                store_rows4(P.dst, P.dst_pitch, P.width, P.height, by, bx, h, (P.flags & kVecDst) != 0, out);

            if ((MODE & kSse) && active) {
                unpark_rows(park, psw, pix);
                const int nr = min(4, P.height - (by * 8 + 4 * h)), nc = min(8, P.width - bx * 8);
                if (nr == 4 && nc == 8) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const unsigned ad = __vabsdiffu4(out[j][q], pix[j][q]);
                            e = __dp4a(ad, ad, e);
                        }
                } else {
                    for (int j = 0; j < nr; ++j)
                        for (int cc = 0; cc < nc; ++cc) {
                            const int d = sample4(out, j, cc) - sample4(pix, j, cc);
                            e += d * d;
                        }
                }
            }
        }
    }
    return (MODE & kSse) ? warp_sum(e) : 0u;
}

// Direct (non-batched) fused calls with two lanes per block: grid-stride over
// the warp tiles of up to kMaxPlanes planes, tables in shared memory, SSE
// summed per CTA and added to each plane's word once (zero on entry).
constexpr int kPairCodecHeader = 2 * (int)sizeof(QuantSet) + kMaxPlanes * 8;
static_assert(kPairCodecHeader % 16 == 0, "per-warp buffers must stay 16-byte aligned");

__host__ __device__ constexpr int pair_codec_smem_bytes(int threads) {
    return kPairCodecHeader + (threads / 32) * (kXBytes + kParkBytes);
}

template <unsigned MODE>
__global__ void __launch_bounds__(256, DCTGB_PAIR_MINB) k_codec_pair(const __grid_constant__ DirectArgs args) {
    extern __shared__ __align__(16) uint8_t smem[];
    QuantSet* tabs = reinterpret_cast<QuantSet*>(smem);
    unsigned long long* csse = reinterpret_cast<unsigned long long*>(smem + 2 * sizeof(QuantSet));
    {
        const uint32_t* s = reinterpret_cast<const uint32_t*>(args.tabs);
        uint32_t* d = reinterpret_cast<uint32_t*>(tabs);
        for (int i = threadIdx.x; i < (int)(2 * sizeof(QuantSet) / 4); i += blockDim.x) d[i] = s[i];
        if (threadIdx.x < kMaxPlanes) csse[threadIdx.x] = 0ull;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int warps_per_cta = blockDim.x >> 5;
    uint8_t* xb = smem + kPairCodecHeader + warp * (kXBytes + kParkBytes);
    for (int tile = blockIdx.x * warps_per_cta + warp; tile < args.ntiles; tile += gridDim.x * warps_per_cta) {
        int pi = 0;
#pragma unroll
        for (int k = 1; k < kMaxPlanes; ++k)
            if (k < args.nplanes && tile >= args.p[k].tile_begin) pi = k;
        const PlaneArg& P = args.p[pi];
        const unsigned e = process_tile_pair<MODE>(P, tabs[P.table], tile - P.tile_begin, lane, xb);
        if ((MODE & kSse) && lane == 0 && e) atomicAdd(&csse[pi], (unsigned long long)e);
    }
    __syncthreads();
    if ((MODE & kSse) && threadIdx.x < args.nplanes && csse[threadIdx.x])
        atomicAdd(args.p[threadIdx.x].sse, csse[threadIdx.x]);
}

// Host launcher of k_codec_pair: one persistent grid of resident CTAs.  A
// call with fewer tiles than warps in `num_sms` CTAs of `threads` gets
// smaller CTAs (down to two warps), so a small plane spreads over more SMs
// instead of sharing a few SMs' schedulers (a tile takes one warp many
// microseconds, so that sharing sets the latency of the whole call).
template <unsigned MODE>
inline cudaError_t launch_codec_pair(const DirectArgs& a, int num_sms, int threads, cudaStream_t s) {
    while (threads > 64 && (long long)a.ntiles < (long long)num_sms * (threads / 32)) threads /= 2;
    const size_t smem = pair_codec_smem_bytes(threads);
    cudaError_t e = cudaFuncSetAttribute(k_codec_pair<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_codec_pair<MODE>, threads, smem);
    if (e != cudaSuccess) return e;
    k_codec_pair<MODE><<<persistent_grid(a.ntiles, threads, num_sms, occ), threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dctgb
