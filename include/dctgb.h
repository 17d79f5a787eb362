/*
 * dctgb.h - C ABI of the GB300 (sm_103a) Cordic-based Loeffler DCT image codec.
 *
 * The library implements the compression path of "CUDA based performance
 * evaluation of the computational efficiency of the DCT image compression
 * technique on both the CPU and GPU": a per-8x8-block Cordic-based Loeffler
 * forward DCT (Sec. 2.5.2, Fig. 1), a quantiser, the inverse DCT (Sec. 3.2
 * runs DCT, quantiser and IDCT as separate kernels) and the PSNR of the
 * reconstruction (Sec. 4.1, Eq. 23 and Eq. 24).  Numeric choices the paper
 * leaves open (fixed-point widths, CORDIC iteration count, rounding, table
 * scaling, padding) are those of include/dctgb_spec.json; dct_spec_query()
 * reports the values compiled into the library.
 *
 * Conventions shared by every entry point:
 *  - All image, coefficient and result pointers are DEVICE pointers unless
 *    the parameter name ends in _host.  The caller owns them; the library
 *    never frees or keeps them past the call (dct_batch_prepare keeps them
 *    until the next prepare or dct_plan_destroy, see there).
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream).  No call synchronises unless
 *    it writes a _host output that depends on GPU results (documented).
 *  - Arguments are checked on the host before anything is enqueued; a bad
 *    argument returns DCT_ERR_INVALID_ARG and enqueues nothing.  Launch
 *    errors return DCT_ERR_CUDA.  Device code never traps or asserts.
 *  - dct_last_error() returns a thread-local message for the last failure.
 *  - Samples are uint8.  A plane is width x height samples with `pitch`
 *    bytes between row starts (pitch >= width).  Planes whose width or
 *    height is not a multiple of 8 are padded by edge replication inside the
 *    transform; only real samples are written or counted.
 *  - Coefficients are int16, block-major: plane p's block (by, bx) holds 64
 *    values in natural order u*8+v (u vertical frequency, v horizontal) at
 *    element offset coeff_offset(p) + (by * nbx + bx) * 64, where
 *    nbx = ceil(width/8), nby = ceil(height/8) and coeff_offset(p) is the sum
 *    of nbx*nby*64 over the planes before p in the same call.
 */
#ifndef DCTGB_H
#define DCTGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DCT_OK = 0,
    DCT_ERR_INVALID_ARG = 1,   /* bad pointer, size, quality or table value */
    DCT_ERR_UNSUPPORTED = 2,   /* valid request the library does not serve */
    DCT_ERR_ALLOC = 3,         /* a device or host allocation failed */
    DCT_ERR_CUDA = 4,          /* a CUDA call or launch failed */
    DCT_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    DCT_ERR_STATE = 6          /* the plan is not in the state the call needs */
} dct_status;

typedef struct dct_plan_s* dct_plan_t;
typedef void* dct_stream_t;    /* cudaStream_t */

/* One uint8 sample plane.  `data` is a device pointer; it is read-only for
 * inputs and written for outputs. */
typedef struct {
    uint8_t* data;
    int32_t width;
    int32_t height;
    int32_t pitch;             /* bytes between row starts, >= width */
} dct_plane;

enum { DCT_LAYOUT_GRAY8 = 0, DCT_LAYOUT_YUV420 = 1 };

/* Quality 1..100 selects the IJG-scaled T.81 Annex K tables: the luminance
 * table for plane 0 and, under DCT_LAYOUT_YUV420, the chrominance table for
 * planes 1 and 2.  Quality 0 means "use qtab_host", which holds 64 entries
 * (one table for every plane) or 2*64 entries (luma table, then chroma table
 * for planes >= 1 under DCT_LAYOUT_YUV420), natural order, each in 1..255. */

typedef struct {
    int32_t max_width;         /* largest plane width accepted, >= 1 */
    int32_t max_height;        /* largest plane height accepted, >= 1 */
    int32_t layout;            /* DCT_LAYOUT_GRAY8 or DCT_LAYOUT_YUV420 */
    int32_t max_batch;         /* largest item count for the batch calls, >= 0 */
    uint32_t flags;            /* reserved, must be 0 */
} dct_plan_desc;

/* Numeric spec compiled into the library (mirrors include/dctgb_spec.json). */
typedef struct {
    int32_t P;                 /* level-shift fraction bits: x = (p - 128) << P */
    int32_t N;                 /* CORDIC micro-rotations per rotation (shifts 1..N) */
    int32_t R;                 /* dequantiser weight fraction bits */
    int32_t quant_shift;       /* quantiser multiplier fraction bits (32) */
    int32_t dequant_clamp;     /* |q*Q| clamp before weighting (4096) */
    int32_t psnr_max;          /* default MAX of Eq. 23 (255) */
    uint32_t sigma_odd_upper;  /* bit i set <=> s_i = +1 for rot(d3,d0,3pi/16) */
    uint32_t sigma_odd_lower;  /* same for rot(d2,d1,pi/16) */
    uint32_t sigma_even;       /* same for the -pi/8 part of rot(e2,e3,3pi/8) */
    int32_t stats_words;       /* uint64 words per plane written by dct_compress stats */
} dct_spec_info;

/* Fills *out with the compiled spec.  Host only; never fails for out != NULL. */
dct_status dct_spec_query(dct_spec_info* out);

/* Host only: the quantiser/dequantiser tables the device uses for one plane
 * (Sec. 3.2 quantiser; IJG scaling of T.81 Annex K).  quality/qtab_host as
 * above; chroma selects the chrominance table (quality > 0) or the second
 * half of qtab_host.  Writes Q_host[64] (1..255), M_host[64] =
 * rint(2^32 / (8 * 2^P * g_u g_v Q)), W_host[64] = rint(2^R / (g_u g_v)).
 * Any output pointer may be NULL. */
dct_status dct_tables(int quality, const uint16_t* qtab_host, int qtab_entries, int chroma,
                      uint16_t* Q_host, uint32_t* M_host, int32_t* W_host);

/* Creates a plan: validates the limits and allocates the plan's own device
 * workspace (batch work list, tables, statistics scratch).  `stream` orders
 * the workspace initialisation.  The plan is not thread-safe: one host
 * thread at a time; calls on different streams must not overlap on the GPU
 * when they share the plan's workspace (the batch and rate-control calls). */
dct_status dct_plan_create(dct_plan_t* out, const dct_plan_desc* desc, dct_stream_t stream);

/* Frees the plan's workspace and graphs (synchronises the device first). */
dct_status dct_plan_destroy(dct_plan_t plan);

/* Forward path (Sec. 2.5.2 transform, Sec. 3.2 quantiser): for each plane,
 * level shift, 2-D Cordic-Loeffler DCT, quantise, store int16 coefficients.
 *  planes[nplanes]  1..4 input planes (device data), each within the plan limits.
 *  coeffs           device int16 output, sum over planes of nbx*nby*64 values,
 *                   16-byte aligned.
 *  stats_out        optional (NULL = skip) device uint64 array of
 *                   dct_spec_info.stats_words words per plane, overwritten:
 *                   words 0..63 band energies sum_blocks ((|Y_uv| >> (P+1))^2),
 *                   then pixel statistics (see dct_stats_layout in the
 *                   Python binding): sum p, sum p^2, min p, max p,
 *                   sum |dx|, sum |dy|, sum dx^2, sum dy^2 (within blocks),
 *                   four counts of blocks whose AC band-energy sum is below
 *                   2^10, 2^14, 2^18, 2^22, number of blocks, samples. */
dct_status dct_compress(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                        const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                        uint64_t* stats_out, dct_stream_t stream);

/* Inverse path (Sec. 3.2 dequantiser and IDCT): dequantise, 2-D transposed
 * Cordic-Loeffler graph, descale and clamp to uint8.
 *  coeffs           device int16 input laid out as dct_compress writes it
 *                   for planes of the sizes of out_planes, 16-byte aligned.
 *  out_planes       nplanes output planes (device data written).
 *  ref_planes       optional originals (same sizes) for a fused SSE; NULL = none.
 *  sse_out          device uint64[nplanes], overwritten with
 *                   sum (ref - out)^2 per plane (Eq. 24 numerator); required
 *                   iff ref_planes != NULL. */
dct_status dct_reconstruct(dct_plan_t plan, const int16_t* coeffs, const dct_plane* out_planes,
                           int nplanes, int quality, const uint16_t* qtab_host, int qtab_entries,
                           const dct_plane* ref_planes, uint64_t* sse_out, dct_stream_t stream);

/* One pass over the pixels doing the forward path, the inverse path and the
 * SSE (the whole Sec. 3.2 pipeline and Eq. 24) with the coefficients kept in
 * registers.  coeffs (may be NULL) receives what dct_compress would write;
 * recon_planes (may be NULL) receives what dct_reconstruct would write;
 * sse_out (device uint64[nplanes], required) is overwritten with the SSE. */
dct_status dct_codec_fused(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                           const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                           const dct_plane* recon_planes, uint64_t* sse_out, dct_stream_t stream);

/* Exact-DCT pipeline: the "DCT" rows of Tables 3 and 4 (the orthonormal 2-D
 * DCT of Eq. 6, quantiser, dequantiser, inverse), for comparing its PSNR with
 * the Cordic-based path.  Computed in float32 with a fixed operation order
 * (each product and sum rounded on its own, k ascending; q = sgn(X)
 * floor(|X| / Q + 0.5); pixel = clamp(floor((y + 128) + 0.5), 0, 255)) so
 * the codes are reproducible.  Arguments as dct_codec_fused; coeffs holds the
 * exact pipeline's int16 codes. */
dct_status dct_exact_fused(dct_plan_t plan, const dct_plane* planes, int nplanes, int quality,
                           const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                           const dct_plane* recon_planes, uint64_t* sse_out, dct_stream_t stream);

/* RGB to YCbCr 4:2:0 (no counterpart in the paper, which works on grey
 * images): full-range BT.601 as in JFIF with 16-bit fixed-point coefficients
 * (Y = (19595 R + 38470 G + 7471 B + 32768) >> 16, Cb and Cr likewise with
 * offset 128 and clamping), chroma averaged over 2x2 as (a+b+c+d+2) >> 2 with
 * the edge pixel repeated for odd sizes.
 *  rgb        device, interleaved R,G,B bytes, rgb_pitch bytes between rows
 *  y          width x height output plane (device data written)
 *  cb, cr     ceil(width/2) x ceil(height/2) output planes */
dct_status dct_rgb_to_yuv420(const uint8_t* rgb, int32_t width, int32_t height, int32_t rgb_pitch,
                             const dct_plane* y, const dct_plane* cb, const dct_plane* cr, dct_stream_t stream);

/* RGB input straight into the forward path (no counterpart in the paper,
 * which codes grey images): the RGB -> YCbCr 4:2:0 conversion of
 * dct_rgb_to_yuv420 fused with dct_compress of the three planes, so the
 * planes never reach device memory (3 bytes per pixel in, the codes out).
 * The codes equal those of dct_rgb_to_yuv420 followed by dct_compress on the
 * planes [Y (width x height), Cb, Cr (ceil(width/2) x ceil(height/2))] with
 * the luminance table for Y and the chrominance table for Cb and Cr.
 *  rgb            device, interleaved R,G,B bytes; row r starts at
 *                 rgb + r * rgb_pitch (rgb_pitch >= 3 * width)
 *  width, height  within the plan's limits
 *  quality/qtab   as dct_compress under DCT_LAYOUT_YUV420 (64 entries: one
 *                 table for all three planes; 128: luma, then chroma)
 *  coeffs         device int16, 16-byte aligned: Y codes, then Cb, then Cr,
 *                 laid out as dct_compress writes them for those planes. */
dct_status dct_compress_rgb(dct_plan_t plan, const uint8_t* rgb, int32_t width, int32_t height, int32_t rgb_pitch,
                            int quality, const uint16_t* qtab_host, int qtab_entries, int16_t* coeffs,
                            dct_stream_t stream);

/* Rate of quantised coefficients (no counterpart in the paper, which never
 * measures the compressed size): counts of the JPEG-style symbols of each
 * plane.  Per plane DCT_ENTROPY_WORDS uint64 words (device, overwritten):
 * 0..15 DC categories of the block-major DC differences (first block
 * predicted by 0), 16..271 AC run/size symbols in zig-zag order (ZRL 0xF0
 * per 16 zeros before a value, EOB 0x00 for trailing zeros), 272 amplitude
 * bits, 273 blocks.  coeffs is laid out as dct_compress writes it for
 * planes of the given sizes (only width and height are read).
 * Synchronises `stream` before launching (host block counts are uploaded). */
#define DCT_ENTROPY_WORDS 274
dct_status dct_entropy_stats(dct_plan_t plan, const int16_t* coeffs, const dct_plane* planes, int nplanes,
                             uint64_t* stats_out, dct_stream_t stream);

/* Host only: bits of one plane from its DCT_ENTROPY_WORDS words: amplitude
 * bits + sum over the DC and the AC counts of n log2(N / n) (the length of an
 * ideal static code for the plane's own symbol statistics). */
double dct_entropy_bits(const uint64_t* stats_host);

/* Host only: an achievable bit count of one plane from the same words:
 * amplitude bits + the cost of an optimal prefix code for the DC counts and
 * one for the AC counts, no codeword longer than 16 bits (the limit of
 * JPEG's Huffman tables; package-merge), a lone symbol coded in one bit.
 * 0 for a NULL pointer. */
uint64_t dct_huffman_bits(const uint64_t* stats_host);

/* SSE and PSNR of two sets of planes of equal sizes (Eq. 23, Eq. 24).
 *  sse_out    device uint64[nplanes], overwritten.
 *  psnr_host  optional host double[nplanes + 1]: per-plane PSNR and the
 *             sample-weighted PSNR over all planes, with MAX = max_value
 *             (0 = the spec default 255); +inf when the SSE is 0.  When it is
 *             given the call synchronises `stream`. */
dct_status dct_psnr(dct_plan_t plan, const dct_plane* a, const dct_plane* b, int nplanes,
                    uint64_t* sse_out, double* psnr_host, double max_value, dct_stream_t stream);

/* Host only: PSNR = 10 log10(max_value^2 * n / sse) (Eq. 23 with Eq. 24);
 * +inf for sse == 0; max_value 0 means 255. */
double dct_psnr_from_sse(uint64_t sse, int64_t n_samples, double max_value);

/* Host only: PSNR (Eq. 23 with Eq. 24) of n planes from their SSEs and
 * sample counts, and the sample-weighted PSNR over all of them (one MSE
 * over the union of their samples, the combined figure of a 4:2:0 frame).
 * psnr_host receives n + 1 values; +inf where an SSE is 0; max_value 0
 * means 255.  Sample counts must be >= 1. */
dct_status dct_psnr_from_sse_list(const uint64_t* sse_host, const int64_t* samples_host, int n, double max_value,
                                  double* psnr_host);

/* ---------------------------------------------------------------------
 * Batched path: many images of uneven sizes and qualities in one
 * persistent launch replayed from a CUDA graph.
 * --------------------------------------------------------------------- */

enum {
    DCT_OP_COMPRESS = 1u,      /* write coefficients */
    DCT_OP_RECONSTRUCT = 2u,   /* write the reconstruction */
    DCT_OP_SSE = 4u,           /* accumulate the SSE against the source */
    DCT_OP_TWO_PASS = 8u       /* with COMPRESS|RECONSTRUCT: a forward kernel that
                                  writes the coefficients, then an inverse kernel
                                  that reads them back (Sec. 3.2's separate
                                  kernels), instead of one fused pass */
};

typedef struct {
    dct_plane src;             /* input plane (device) */
    int16_t* coeffs;           /* output coefficients or NULL (needs OP_COMPRESS) */
    uint8_t* recon;            /* output plane data or NULL (needs OP_RECONSTRUCT) */
    int32_t recon_pitch;       /* bytes between reconstruction rows */
    int32_t quality;           /* 1..100, or 0 = use qtab_host of the item */
    int32_t chroma;            /* 1 = chrominance table (quality > 0) */
    const uint16_t* qtab_host; /* 64 entries when quality == 0, else NULL */
} dct_batch_item;

/* Launch shape of the persistent kernel, chosen by dct_autotune.  A new
 * plan starts with {256, 8, 32, 2}. */
typedef struct {
    int32_t threads_per_cta;   /* 64..256, multiple of 32 */
    int32_t ctas_per_sm;       /* 1..32 CTAs per SM in the grid (more than fit
                                * at once: shorter tile ranges); 0: as many
                                * as fit at once */
    int32_t tile_blocks;       /* 8x8 blocks per warp tile: 32 */
    int32_t lanes_per_block;   /* 0 or 1: one lane per 8x8 block; 2: two lanes
                                * per block (fused COMPRESS/RECONSTRUCT/SSE
                                * operations only; other operations use one) */
} dct_launch_shape;

/* Uploads a work list of n items (1..max_batch) to the plan's workspace,
 * builds the per-item tables and captures [clear SSE, persistent kernel(s)]
 * into a CUDA graph on a plan-owned stream.  ops is a mask of DCT_OP_*:
 *   COMPRESS alone                forward pass, coefficients written;
 *   RECONSTRUCT without COMPRESS  inverse pass from the items' coefficients;
 *   COMPRESS|RECONSTRUCT          one fused pass writing both;
 *   ... | TWO_PASS                forward kernel, then inverse kernel;
 *   SSE                           adds the SSE against src (alone: a fused
 *                                 pass that stores nothing).
 * With DCT_OP_SSE, sse_out (device uint64[n]) receives each item's SSE.
 * The call synchronises `stream` (the upload uses plan-owned pinned
 * staging buffers).  The device pointers
 * of the items are kept by the plan and used by every dct_batch_launch until
 * the next dct_batch_prepare.  shape may be NULL (the plan's tuned or
 * default shape). */
dct_status dct_batch_prepare(dct_plan_t plan, const dct_batch_item* items, int n, uint32_t ops,
                             uint64_t* sse_out, const dct_launch_shape* shape, dct_stream_t stream);

/* Replays the prepared graph on `stream`.  DCT_ERR_STATE if nothing is
 * prepared.  Replays of one plan must not overlap on the GPU: they share the
 * plan's tile counters (the two-lane kernels claim their tiles from them) and
 * their first launch re-clears the SSE words; streams that run batches
 * concurrently each need a plan of their own. */
dct_status dct_batch_launch(dct_plan_t plan, dct_stream_t stream);

/* Times candidate launch shapes for the prepared batch (CUDA events on
 * `stream`, which is synchronised), keeps the fastest as the plan's shape,
 * re-captures the graph with it and writes it to *best (may be NULL).
 * ms_host (may be NULL) receives the best time in milliseconds.  The
 * candidates are 64/128/256 threads per CTA x 1..16 CTAs per SM, with one
 * and (fused operations) two lanes per block.  Every timed replay follows a
 * write over twice the L2 size into a temporary device buffer, so the
 * choice holds for inputs that are not already cached; if that buffer
 * cannot be allocated the replays run warm.  Replays the batch's kernels,
 * so its outputs are overwritten. */
dct_status dct_autotune(dct_plan_t plan, dct_launch_shape* best, float* ms_host, dct_stream_t stream);

/* ---------------------------------------------------------------------
 * Learned rate control.  The paper has no rate controller; these calls
 * choose the quality factor of the plain pipeline above for a target PSNR
 * (Eq. 23): a small network predicts it from statistics the forward pass
 * gathers, the pipeline verifies it, and an 8-step bisection over the
 * qualities 1..100 is the fallback.
 * --------------------------------------------------------------------- */

#define DCT_MLP_INPUTS 80
#define DCT_MLP_HIDDEN 64
#define DCT_MLP_PARAMS 9409   /* 64*80 + 64 + 64*64 + 64 + 64 + 1 */

/* Network 80 -> 64 -> 64 -> 1: a1 = W1 xn + b1, h1 = act(gelu(a1)),
 * a2 = W2 h1 + b2, h2 = act(gelu(a2)), y = sigmoid(W3 h2 + b3), with
 * xn = (x - feat_mean) / feat_std, gelu(a) = a Phi(a) and act() rounding to
 * bfloat16 (act_bf16 = 1) or the identity.  y predicts (Q* - 1) / 99; the
 * quality is clamp(rint(1 + 99 y), 1, 100).  All arrays are device float32
 * owned by the caller. */
typedef struct {
    float* params;        /* DCT_MLP_PARAMS: W1[64][80], b1[64], W2[64][64], b2[64], W3[64], b3;
                             16-byte aligned */
    float* adam_m;        /* DCT_MLP_PARAMS, Adam first moments (training only) */
    float* adam_v;        /* DCT_MLP_PARAMS, Adam second moments (training only) */
    float* feat_mean;     /* DCT_MLP_INPUTS */
    float* feat_std;      /* DCT_MLP_INPUTS */
    int32_t step;         /* Adam steps taken (dct_mlp_adam increments it) */
    int32_t act_bf16;     /* 1: bfloat16 hidden activations, 0: float32 */
} dct_mlp;

/* 80 features per frame from dct_compress-style statistics words (device
 * uint64, DCT stats_words per frame), the frame size and its target PSNR
 * (device arrays of n entries): log band energies, pixel and gradient
 * statistics, low-energy block fractions, log2 sizes, the target and a bias
 * term (see oracle/features.py for the exact formulas). */
dct_status dct_features(const uint64_t* stats, const int32_t* width, const int32_t* height, const float* target,
                        int n, float* feats_out, dct_stream_t stream);

/* Sets feat_mean / feat_std to the mean and standard deviation (floored at
 * 1e-6) of each feature over n rows of feats (device, n x 80). */
dct_status dct_mlp_set_norm(dct_mlp* net, const float* feats, int n, dct_stream_t stream);

/* Forward pass for n rows: y_out (device float[n], may be NULL) and
 * quality_out (device int32[n], may be NULL). */
dct_status dct_mlp_forward(const dct_mlp* net, const float* feats, int n, float* y_out, int32_t* quality_out,
                           dct_stream_t stream);

/* Training targets of n quality labels (device int32, 1..100): labels_out
 * (device float[n]) = (Q - 1) / 99, the value the network's output y
 * predicts. */
dct_status dct_mlp_labels(const int32_t* quality, int n, float* labels_out, dct_stream_t stream);

/* Bytes of device workspace dct_mlp_loss_grad needs for a minibatch of
 * `batch` rows (the workspace must be 16-byte aligned). */
size_t dct_mlp_workspace_bytes(int batch);

/* Mean squared error over the minibatch rows index[0..batch) of (feats,
 * labels) and its gradient (device float[DCT_MLP_PARAMS], overwritten).
 * loss_out: device float[1].  Sums over the minibatch run in a fixed order,
 * so the result is deterministic.  workspace: dct_mlp_workspace_bytes(batch). */
dct_status dct_mlp_loss_grad(const dct_mlp* net, const float* feats, const float* labels, const int32_t* index,
                             int batch, float* grad_out, float* loss_out, void* workspace, dct_stream_t stream);

/* One Adam update of net->params from grad (Kingma and Ba, bias-corrected);
 * increments net->step (host field). */
dct_status dct_mlp_adam(dct_mlp* net, const float* grad, float lr, float beta1, float beta2, float eps,
                        dct_stream_t stream);

/* One epoch of minibatch training: for each consecutive `batch` rows of
 * order[0..n) (device int32, a permutation chosen by the caller) a
 * loss_grad + adam step (beta1 0.9, beta2 0.999, eps 1e-8), the Adam update
 * fused into the gradient kernel with the same arithmetic (two launches per
 * minibatch).  batch in 1..2^20, lr > 0.  loss_out: device
 * float[ceil(n / batch)].  workspace: dct_mlp_workspace_bytes(batch) +
 * DCT_MLP_PARAMS floats. */
dct_status dct_mlp_train_epoch(dct_mlp* net, const float* feats, const float* labels, const int32_t* order, int n,
                               int batch, float lr, float* loss_out, void* workspace, dct_stream_t stream);

/* Result summary of dct_rate_control. */
typedef struct {
    int32_t frames;        /* frames processed */
    int32_t fell_back;     /* frames that went through the bisection */
    int32_t unreachable;   /* frames whose final PSNR is outside the 0.25 dB band: the
                            * bisection evaluated the qualities on both sides of the
                            * band (or ended at 1 or 100), so no quality lands in it
                            * while PSNR rises with quality */
    int32_t within_tol;    /* frames whose final PSNR is within 0.25 dB of the target */
    int32_t passes;        /* full-pipeline passes over frames (sum over frames) */
    float gpu_ms;          /* device time of the call (CUDA events on `stream`) */
} dct_rc_summary;

/* Quality per frame for a target PSNR.  planes holds nframes * planes_per_frame
 * device planes, frame-major; planes_per_frame is 1 (grey) or 3 (4:2:0: the
 * chrominance table for planes 1 and 2).  A frame's PSNR is Eq. 23 over all
 * of its samples with MAX 255.  With net == NULL every frame is bisected
 * (8 passes: lo = 1, hi = 100, mid = (lo + hi) / 2, hi = mid if
 * PSNR(mid) >= target else lo = mid + 1, giving Q* = hi; when PSNR(Q*) is
 * more than 0.25 dB from the target but the last rejected quality, Q* - 1,
 * is within 0.25 dB, the result is Q* - 1).  With a network,
 * the statistics pass, features and network give a quality, one pass
 * verifies it, and frames whose PSNR misses the target by more than 0.25 dB
 * (either way) fall back to the bisection.  Decisions compare the integer
 * SSE with thresholds computed on the host in float64.  Host outputs
 * (nframes entries each, any may be NULL): quality_host, sse_host (SSE at
 * the chosen quality), fell_back_host.  Synchronises `stream`.  Uses the
 * plan's workspace: nframes * planes_per_frame <= max_batch. */
dct_status dct_rate_control(dct_plan_t plan, const dct_plane* planes, int planes_per_frame, int nframes,
                            const float* target_host, const dct_mlp* net, int32_t* quality_host,
                            uint64_t* sse_host, uint8_t* fell_back_host, dct_rc_summary* summary,
                            dct_stream_t stream);

/* Features (device float[nframes * 80]) of each frame's plane 0 for the given
 * targets: the statistics pass of dct_rate_control on its own, for training
 * and inspection.  Same plane layout as dct_rate_control. */
dct_status dct_rate_features(dct_plan_t plan, const dct_plane* planes, int planes_per_frame, int nframes,
                             const float* target_host, float* feats_out, dct_stream_t stream);

/* Runs one batch like dct_batch_prepare + dct_batch_launch, same item
 * fields and ops, same results, without allocating anything: no
 * cudaMalloc, cudaFree, pinned buffers or plan.  The paper has no
 * counterpart; this exists for callers that cannot allocate device memory
 * while they run: processes whose device memory another allocator reserved
 * up front, latency-critical loops that cannot absorb the implicit device
 * synchronisation of cudaMalloc / cudaFree, and deployments with a fixed
 * memory budget that forbid allocation after start-up.
 *  - The work list goes to a fixed array inside the library image
 *    (about 70 KB on every device that loads the library, held until the
 *    process exits).  n is limited to 1..64 items; larger n returns
 *    DCT_ERR_INVALID_ARG.  Each item obeys the limits of a plan: at most
 *    65536 x 65536 and below 2^31 samples.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress).
 *  - Every call on a device shares the array and overwrites it.  Calls that
 *    overlap on the GPU (different streams, or host threads racing) race on
 *    it: serialise them.  sse_out is cleared by the call itself.
 *  - The descriptors are copied from the caller's stack with
 *    cudaMemcpyAsync on `stream`.  That memory is pageable, so the driver
 *    may first wait for the work already queued on `stream`; the call
 *    returns once the descriptors are staged.  For the same reason the call
 *    returns DCT_ERR_UNSUPPORTED, enqueuing nothing, while `stream` is being
 *    captured into a graph.
 *  - Launch shape: a new plan's default (two lanes per block where the
 *    operation has a two-lane kernel, fixed tile ranges per warp). */
dct_status dct_batch_run_noalloc(const dct_batch_item* items, int n, uint32_t ops, uint64_t* sse_out,
                                 dct_stream_t stream);

/* Integer issue-rate probe (no counterpart in the paper; measurement helper
 * for the roofline of the codec kernels, which are bound by integer
 * instruction issue).  Runs `iters` iterations of 32 CORDIC micro-rotations
 * (a, b) <- (a + (b >> i), b - (a >> i)), i in 2..6, per thread on 8
 * independent chains, over every SM, in one of four instruction forms:
 * kind 0 shift + add for both halves (the inverse kernels' form, and the
 * forward kernels' for i = 1); kind 1 one half as mad.hi.s32, the other as
 * shift + add; kind 2 both halves as mad.hi.s32; kind 3 both halves as
 * float32 fused multiply-adds with directed rounding (the forward kernels'
 * form for i >= 2, exact on their biased operands).  Counts 4 integer
 * operations (2 floor shifts, 2 adds) per micro-rotation.  Host outputs (any may be NULL): operations per clock per
 * SM (from clock64 spans, independent of the clock the GPU ran at),
 * Tops/s and the kernel time in ms.  Allocates two small device buffers;
 * synchronises `stream`.  iters in 1..2^24. */
dct_status dct_int_peak(int kind, int iters, double* ops_per_clk_sm_host, double* tops_host, float* ms_host,
                        dct_stream_t stream);

/* Test hook for the failure paths (no counterpart in the paper): arms the
 * library so that the nth allocation attempt from now (device or pinned
 * memory, stream or event creation of a plan's workspaces: the batch work
 * list, the rate-control state, the autotuner's events and flush buffer)
 * fails as if the device were out of memory, without calling CUDA; the
 * call that meets it returns DCT_ERR_ALLOC having enqueued nothing, and
 * the hook disarms (the autotuner's flush buffer is optional: without it
 * the candidates are timed warm).  nth = 0 disarms it.  attempts_host (may be NULL)
 * receives the number of attempts counted since the library loaded.  Host
 * only; never touches the GPU. */
dct_status dct_debug_fail_alloc(int nth, int64_t* attempts_host);

/* Thread-local description of the last error on this thread. */
const char* dct_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DCTGB_H */
