// RGB input straight into the forward path (no counterpart in the paper,
// which codes grey images): RGB -> YCbCr 4:2:0 (full-range BT.601 as in
// JFIF, 16-bit fixed-point coefficients, per-pixel chroma averaged over 2x2
// with rounding) fused with the level shift, the 2-D Cordic-Loeffler DCT
// (Sec. 2.5.2) and the quantiser (Sec. 3.2).  The Y, Cb and Cr planes never
// reach global memory: 3 bytes per pixel are read and the coefficients
// written (3 bytes per pixel), against 9 for the conversion kernel followed
// by dct_compress.
//
// Work unit: a strip of 16 macroblocks of one macroblock row (16 x 256
// pixels) gives 2 x 32 luma blocks and 16 blocks of each chroma plane.  A
// CTA of 96 threads converts the strip into shared memory (phase 1), then
// each thread runs the one-lane forward tile on one of the 96 blocks and
// stages its codes; the CTA writes each plane's run of consecutive blocks
// with 16-byte stores (phase 2).
//
// Padding follows the planes the two-kernel route builds: a luma sample
// outside the image repeats the nearest pixel; a chroma sample outside the
// ceil(W/2) x ceil(H/2) chroma plane repeats the nearest chroma sample,
// which is the rounded average of the 2x2 pixels of that sample (an odd last
// pixel row or column repeated).
#include <cstring>

#include "host_common.h"

namespace dctgb {

constexpr int kRgbMbPerUnit = 16;                  // macroblocks per work unit
constexpr int kRgbUnitW = 16 * kRgbMbPerUnit;       // 256 pixels
constexpr int kRgbThreads = 96;                     // one thread per block: 64 Y + 16 Cb + 16 Cr
constexpr int kRgbYBytes = 16 * kRgbUnitW;          // 16 rows x 256 luma samples
constexpr int kRgbCBytes = 8 * (kRgbUnitW / 2);     // 8 rows x 128 chroma samples
constexpr int kRgbRawRow = 3 * kRgbUnitW + 32;       // one strip row of RGB bytes, from its aligned 16-byte chunk
constexpr int kRgbSmem = 2 * (int)sizeof(QuantSet) + kRgbYBytes + 2 * kRgbCBytes + kRgbThreads * 128 +
                         16 * kRgbRawRow + 16 * 4;

struct RgbArgs {
    const uint8_t* rgb;
    int16_t* coef;                 // Y codes, then Cb, then Cr (dct_compress layout)
    QuantSet tabs[2];              // luma, chroma
    int32_t width, height, pitch;  // pixels, bytes between RGB rows
    int32_t cw, ch;                // chroma plane size
    int32_t nbx_y, nby_y;          // luma block grid
    int32_t nbx_c, nby_c;          // chroma block grid (= macroblock grid)
    int32_t units_x, units;        // work units per macroblock row, in total
    int64_t cb_offset, cr_offset;  // element offsets of the Cb and Cr codes
};

__device__ __forceinline__ void rgb_convert(const uint8_t* p, int& y, int& cb, int& cr) {
    const int r = p[0], g = p[1], b = p[2];
    y = (19595 * r + 38470 * g + 7471 * b + 32768) >> 16;
    cb = max(0, min(255, (-11058 * r - 21710 * g + 32768 * b + (128 << 16) + 32768) >> 16));
    cr = max(0, min(255, (32768 * r - 27439 * g - 5329 * b + (128 << 16) + 32768) >> 16));
}

// Forward-path quantiser of the one-lane tile: the high word of Y M + 2^31
// away from the four tie entries, |Y| with an unsigned multiply and the sign
// there (tie_entry).
__device__ __forceinline__ void quantize_fwd(int (&x)[8][8], const QuantSet& T) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int y = x[u][v];
            if (!tie_entry(u, v)) {
                const long long p = (long long)y * (long long)(int)T.M[u * 8 + v] + 0x80000000ll;
                x[u][v] = (int)(p >> 32);
            } else {
                const uint32_t a = (uint32_t)abs(y);
                const uint32_t q = (uint32_t)(((unsigned long long)a * T.M[u * 8 + v] + 0x80000000ull) >> 32);
                x[u][v] = y < 0 ? -(int)q : (int)q;
            }
        }
    }
}

__global__ void __launch_bounds__(kRgbThreads, 6) k_compress_rgb(const __grid_constant__ RgbArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    QuantSet* tabs = reinterpret_cast<QuantSet*>(smem);
    uint8_t* ys = smem + 2 * sizeof(QuantSet);            // [16][256]
    uint8_t* cbs = ys + kRgbYBytes;                       // [8][128]
    uint8_t* crs = cbs + kRgbCBytes;                      // [8][128]
    uint8_t* stage = crs + kRgbCBytes;                    // [96][128]
    uint8_t* raw = stage + kRgbThreads * 128;             // [16][kRgbRawRow] RGB bytes of the strip
    int* lead16 = reinterpret_cast<int*>(raw + 16 * kRgbRawRow);   // [16] offset of each row in its chunk
    {
        const uint32_t* s = reinterpret_cast<const uint32_t*>(a.tabs);
        uint32_t* d = reinterpret_cast<uint32_t*>(tabs);
        for (int i = threadIdx.x; i < (int)(2 * sizeof(QuantSet) / 4); i += blockDim.x) d[i] = s[i];
    }
    const int t = threadIdx.x;
    for (int unit = blockIdx.x; unit < a.units; unit += gridDim.x) {
        const int my = unit / a.units_x;
        const int mx0 = (unit - my * a.units_x) * kRgbMbPerUnit;
        __syncthreads();          // the previous unit's stage is written out; tables are in place

        // phase 0: the strip's 16 pixel rows (the last image row repeated
        // below the image), columns x0 .. x1 - 1, into shared memory with
        // 16-byte cp.async copies of the aligned chunks inside each row's
        // bytes; the partial chunks at either end are read byte by byte, so
        // nothing outside the caller's rows is touched.  Every pixel phase
        // 1 needs lies in these rows and columns.
        const int x0 = 16 * mx0, x1 = min(x0 + kRgbUnitW, a.width);
        const int nbytes = 3 * (x1 - x0);
        if (t < 16)
            lead16[t] = (int)((uintptr_t)(a.rgb + (size_t)min(16 * my + t, a.height - 1) * a.pitch + 3 * x0) & 15u);
        constexpr int kChunks = kRgbRawRow / 16;
        for (int c = t; c < 16 * kChunks; c += kRgbThreads) {
            const int r = c / kChunks, k = c - r * kChunks;
            const uint8_t* row = a.rgb + (size_t)min(16 * my + r, a.height - 1) * a.pitch + 3 * x0;
            const int lead = (int)((uintptr_t)row & 15u);
            const int b0 = 16 * k;
            if (b0 >= lead + nbytes) continue;
            const uint8_t* src = row - lead + b0;           // 16-byte aligned
            uint8_t* dst = raw + r * kRgbRawRow + b0;
            if (b0 >= lead && b0 + 16 <= lead + nbytes) {
                cp_async16(dst, src);
            } else {
                for (int j = max(b0, lead); j < min(b0 + 16, lead + nbytes); ++j) dst[j - b0] = __ldg(src + (j - b0));
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();

        // phase 1: every 2x2 quad of the strip -> 4 luma samples and one
        // chroma sample of each plane (8 x 128 quads), from shared memory
        for (int q = t; q < 8 * (kRgbUnitW / 2); q += kRgbThreads) {
            const int qi = q / (kRgbUnitW / 2), qj = q - qi * (kRgbUnitW / 2);
            int sb = 0, sr = 0;
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const uint8_t* rr = raw + (2 * qi + dy) * kRgbRawRow + lead16[2 * qi + dy];
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int xx = min(x0 + 2 * qj + dx, a.width - 1) - x0;
                    int Y, Cb, Cr;
                    rgb_convert(rr + 3 * xx, Y, Cb, Cr);
                    ys[(2 * qi + dy) * kRgbUnitW + 2 * qj + dx] = (uint8_t)Y;
                    sb += Cb;
                    sr += Cr;
                }
            }
            // chroma sample (cy, cx); outside the chroma plane the nearest
            // chroma sample, whose pixels lie elsewhere in this strip
            const int cy = 8 * my + qi, cx = 8 * mx0 + qj;
            if (cy >= a.ch || cx >= a.cw) {
                const int cyc = min(cy, a.ch - 1), cxc = min(cx, a.cw - 1);
                sb = sr = 0;
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int ry = min(2 * cyc + dy, a.height - 1) - 16 * my;
                    const uint8_t* rr = raw + ry * kRgbRawRow + lead16[ry];
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int xx = min(2 * cxc + dx, a.width - 1) - x0;
                        int Y, Cb, Cr;
                        rgb_convert(rr + 3 * xx, Y, Cb, Cr);
                        sb += Cb;
                        sr += Cr;
                    }
                }
            }
            cbs[qi * (kRgbUnitW / 2) + qj] = (uint8_t)((sb + 2) >> 2);
            crs[qi * (kRgbUnitW / 2) + qj] = (uint8_t)((sr + 2) >> 2);
        }
        __syncthreads();

        // phase 2: thread t owns luma block (2 my + t / 32, 2 mx0 + t % 32)
        // for t < 64, else chroma block (my, mx0 + (t - 64) % 16) of Cb or Cr
        const bool luma = t < 64;
        const int k = luma ? t & 31 : (t - 64) & 15;
        const uint8_t* src = luma ? ys + (t >> 5) * 8 * kRgbUnitW + 8 * k : (t < 80 ? cbs : crs) + 8 * k;
        const int spitch = luma ? kRgbUnitW : kRgbUnitW / 2;
        const bool valid = luma ? (2 * my + (t >> 5) < a.nby_y && 2 * mx0 + k < a.nbx_y) : (mx0 + k < a.nbx_c);
        if (valid) {
            int x[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint2 w = *reinterpret_cast<const uint2*>(src + r * spitch);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    x[r][c] = ((int)(((c < 4 ? w.x : w.y) >> (8 * (c & 3))) & 0xFFu) - 128) * (1 << kP);
            }
            fwd2d<false>(x);
            quantize_fwd(x, tabs[luma ? 0 : 1]);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint4 w;
                w.x = ((uint32_t)x[u][0] & 0xFFFFu) | ((uint32_t)x[u][1] << 16);
                w.y = ((uint32_t)x[u][2] & 0xFFFFu) | ((uint32_t)x[u][3] << 16);
                w.z = ((uint32_t)x[u][4] & 0xFFFFu) | ((uint32_t)x[u][5] << 16);
                w.w = ((uint32_t)x[u][6] & 0xFFFFu) | ((uint32_t)x[u][7] << 16);
                *reinterpret_cast<uint4*>(stage + t * 128 + ((u ^ (t & 7)) << 4)) = w;
            }
        }
        __syncthreads();

        // write-out: four runs of consecutive blocks (two luma block rows,
        // one row of each chroma plane), 16 bytes per thread and step
        const int ny_blk = min(32, a.nbx_y - 2 * mx0);
        const int nc_blk = min(kRgbMbPerUnit, a.nbx_c - mx0);
        for (int run = 0; run < 4; ++run) {
            int first, nblk;
            int64_t base;
            if (run < 2) {
                if (2 * my + run >= a.nby_y) continue;
                first = run * 32;
                nblk = ny_blk;
                base = ((int64_t)(2 * my + run) * a.nbx_y + 2 * mx0) * 64;
            } else {
                first = run == 2 ? 64 : 80;
                nblk = nc_blk;
                base = (run == 2 ? a.cb_offset : a.cr_offset) + ((int64_t)my * a.nbx_c + mx0) * 64;
            }
            uint4* g = reinterpret_cast<uint4*>(a.coef + base);
            for (int c = t; c < nblk * 8; c += kRgbThreads) {
                const int blk = first + (c >> 3), row = c & 7;
                g[c] = *reinterpret_cast<const uint4*>(stage + blk * 128 + ((row ^ (blk & 7)) << 4));
            }
        }
    }
}

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_compress_rgb(dct_plan_t plan, const uint8_t* rgb, int32_t width, int32_t height,
                                       int32_t rgb_pitch, int quality, const uint16_t* qtab_host, int qtab_entries,
                                       int16_t* coeffs, dct_stream_t stream) {
    if (!plan) return fail(DCT_ERR_INVALID_ARG, "null plan");
    if (!rgb || !coeffs) return fail(DCT_ERR_INVALID_ARG, "null rgb or coeffs");
    if (width < 1 || height < 1 || width > plan->desc.max_width || height > plan->desc.max_height)
        return fail(DCT_ERR_INVALID_ARG, "width/height outside 1..the plan's limits");
    if ((int64_t)rgb_pitch < 3 * (int64_t)width) return fail(DCT_ERR_INVALID_ARG, "rgb_pitch < 3 * width");
    if (((uintptr_t)coeffs) & 15u) return fail(DCT_ERR_INVALID_ARG, "coeffs must be 16-byte aligned");
    RgbArgs a;
    memset(&a, 0, sizeof a);
    dct_status st = build_tables(quality, qtab_host, qtab_entries, 0, a.tabs[0]);
    if (st == DCT_OK) st = build_tables(quality, qtab_host, qtab_entries, 1, a.tabs[1]);
    if (st != DCT_OK) return st;
    a.rgb = rgb;
    a.coef = coeffs;
    a.width = width;
    a.height = height;
    a.pitch = rgb_pitch;
    a.cw = (width + 1) / 2;
    a.ch = (height + 1) / 2;
    a.nbx_y = (width + 7) / 8;
    a.nby_y = (height + 7) / 8;
    a.nbx_c = (a.cw + 7) / 8;
    a.nby_c = (a.ch + 7) / 8;
    a.units_x = (a.nbx_c + kRgbMbPerUnit - 1) / kRgbMbPerUnit;
    const int64_t units = (int64_t)a.units_x * a.nby_c;
    if (units > (1 << 30)) return fail(DCT_ERR_INVALID_ARG, "frame too large");
    a.units = (int32_t)units;
    a.cb_offset = (int64_t)a.nbx_y * a.nby_y * 64;
    a.cr_offset = a.cb_offset + (int64_t)a.nbx_c * a.nby_c * 64;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaFuncSetAttribute(k_compress_rgb, cudaFuncAttributeMaxDynamicSharedMemorySize, kRgbSmem);
    int occ = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_compress_rgb, kRgbThreads, kRgbSmem);
    if (e != cudaSuccess) return cuda_fail(e, "rgb kernel attributes");
    const int64_t cap = (int64_t)plan->num_sms * (occ > 0 ? occ : 1);
    const int grid = (int)(units < cap ? units : cap);
    k_compress_rgb<<<grid, kRgbThreads, kRgbSmem, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "rgb kernel launch");
}
