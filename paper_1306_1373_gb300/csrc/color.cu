// RGB (interleaved uint8) to YCbCr 4:2:0 planes on the GPU (no counterpart in
// the paper, which works on grey images): full-range BT.601 as in JFIF with
// 16-bit fixed-point coefficients, per-pixel chroma averaged over 2x2 with
// rounding; an odd last row or column repeats its edge pixel.  One thread
// owns one 2x2 quad; a warp covers 64 consecutive pixels of two rows.
#include "host_common.h"

namespace dctgb {

struct ColorArgs {
    const uint8_t* rgb;
    uint8_t *y, *cb, *cr;
    int32_t width, height, rgb_pitch, y_pitch, cb_pitch, cr_pitch;
    int32_t cw, ch;   // chroma size
};

__device__ __forceinline__ void convert(const uint8_t* p, int& y, int& cb, int& cr) {
    const int r = p[0], g = p[1], b = p[2];
    y = (19595 * r + 38470 * g + 7471 * b + 32768) >> 16;
    cb = max(0, min(255, (-11058 * r - 21710 * g + 32768 * b + (128 << 16) + 32768) >> 16));
    cr = max(0, min(255, (32768 * r - 27439 * g - 5329 * b + (128 << 16) + 32768) >> 16));
}

__global__ void __launch_bounds__(256) k_rgb_to_yuv420(const __grid_constant__ ColorArgs a) {
    const long long nquads = (long long)a.cw * a.ch;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nquads;
         q += (long long)gridDim.x * blockDim.x) {
        const int qy = (int)(q / a.cw), qx = (int)(q - (long long)qy * a.cw);
        int sb = 0, sr = 0;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int yy = min(2 * qy + dy, a.height - 1);
            const bool real_row = 2 * qy + dy < a.height;
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int xx = min(2 * qx + dx, a.width - 1);
                int Y, Cb, Cr;
                convert(a.rgb + (size_t)yy * a.rgb_pitch + 3 * xx, Y, Cb, Cr);
                sb += Cb;
                sr += Cr;
                if (real_row && 2 * qx + dx < a.width) a.y[(size_t)yy * a.y_pitch + xx] = (uint8_t)Y;
            }
        }
        a.cb[(size_t)qy * a.cb_pitch + qx] = (uint8_t)((sb + 2) >> 2);
        a.cr[(size_t)qy * a.cr_pitch + qx] = (uint8_t)((sr + 2) >> 2);
    }
}

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_rgb_to_yuv420(const uint8_t* rgb, int32_t width, int32_t height, int32_t rgb_pitch,
                                        const dct_plane* y, const dct_plane* cb, const dct_plane* cr,
                                        dct_stream_t stream) {
    if (!rgb || !y || !cb || !cr || !y->data || !cb->data || !cr->data)
        return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (width < 1 || height < 1 || width > (1 << 16) || height > (1 << 16))
        return fail(DCT_ERR_INVALID_ARG, "width/height must be 1..65536");
    if (rgb_pitch < 3 * width) return fail(DCT_ERR_INVALID_ARG, "rgb_pitch < 3 * width");
    const int cw = (width + 1) / 2, ch = (height + 1) / 2;
    if (y->width != width || y->height != height || y->pitch < width)
        return fail(DCT_ERR_INVALID_ARG, "Y plane must be width x height");
    if (cb->width != cw || cb->height != ch || cr->width != cw || cr->height != ch || cb->pitch < cw || cr->pitch < cw)
        return fail(DCT_ERR_INVALID_ARG, "chroma planes must be ceil(width/2) x ceil(height/2)");
    ColorArgs a{rgb, y->data, cb->data, cr->data, width, height, rgb_pitch, y->pitch, cb->pitch, cr->pitch, cw, ch};
    const long long nq = (long long)cw * ch;
    long long grid = (nq + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_rgb_to_yuv420<<<(int)grid, 256, 0, (cudaStream_t)stream>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "color launch");
}
