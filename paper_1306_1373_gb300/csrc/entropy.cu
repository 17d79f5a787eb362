// Rate of the quantised coefficients (no counterpart in the paper, which never
// measures the compressed size): counts of the JPEG-style symbols of each
// plane, from which an ideal static code's length follows on the host.
//   DC  category of q00 - q00(previous block in block-major order), 0..15
//   AC  zig-zag run/size symbols; ZRL (0xF0) for every 16 zeros before a
//       non-zero value; EOB (0x00) when trailing zeros remain
//   amplitude bits: the category of every coded value
// One lane reads one block's 64 stored int16 coefficients; symbol counts
// go to per-CTA shared histograms (one per plane) flushed once per CTA.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_common.h"

namespace dctgb {

constexpr int kEntWords = DCT_ENTROPY_WORDS;   // 16 DC + 256 AC + amplitude bits + blocks
constexpr int kMaxCodeLen = 16;                 // longest codeword of the prefix codes (as JPEG's Huffman tables)

// Natural index u*8+v of zig-zag position k (T.81 Figure A.6): diagonals
// s = u + v in turn, odd s with u rising, even s with u falling.  Called with
// unrolled constant k, it folds to an immediate, so the coefficients stay in
// registers.
__host__ __device__ constexpr int zigzag_index(int k) {
    int n = 0;
    for (int s = 0; s < 15; ++s) {
        const int lo = s > 7 ? s - 7 : 0, hi = s < 7 ? s : 7;
        if (k < n + hi - lo + 1) {
            const int u = (s & 1) ? lo + (k - n) : hi - (k - n);
            return u * 8 + (s - u);
        }
        n += hi - lo + 1;
    }
    return 63;
}
static_assert(zigzag_index(2) == 8 && zigzag_index(3) == 16 && zigzag_index(63) == 63, "zig-zag order");

struct EntropyArgs {
    const int16_t* coef[kMaxPlanes];
    unsigned long long* out[kMaxPlanes];
    int32_t nblk[kMaxPlanes];
    int32_t tile_begin[kMaxPlanes + 1];
    int32_t nplanes;
};

__device__ __forceinline__ int category(int v) { return 32 - __clz(abs(v)); }

__global__ void __launch_bounds__(256) k_entropy(const __grid_constant__ EntropyArgs a) {
    __shared__ unsigned int hist[kMaxPlanes][272];
    __shared__ unsigned long long amp[kMaxPlanes];
    for (int i = threadIdx.x; i < kMaxPlanes * 272; i += blockDim.x) (&hist[0][0])[i] = 0u;
    if (threadIdx.x < kMaxPlanes) amp[threadIdx.x] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int ntiles = a.tile_begin[a.nplanes];
    for (int tile = blockIdx.x * warps + (threadIdx.x >> 5); tile < ntiles; tile += gridDim.x * warps) {
        int pi = 0;
        while (pi + 1 < a.nplanes && tile >= a.tile_begin[pi + 1]) ++pi;
        const int b = (tile - a.tile_begin[pi]) * kTileBlocks + lane;
        unsigned bits = 0;
        if (b < a.nblk[pi]) {
            const int16_t* blk = a.coef[pi] + (size_t)b * 64;
            int q[64];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint4 w = __ldg(reinterpret_cast<const uint4*>(blk) + r);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    q[r * 8 + 2 * k] = (int)(int16_t)(ws[k] & 0xFFFFu);
                    q[r * 8 + 2 * k + 1] = (int)ws[k] >> 16;
                }
            }
            const int prev = b > 0 ? (int)__ldg(blk - 64) : 0;
            const int dc = category(q[0] - prev);
            atomicAdd(&hist[pi][dc], 1u);
            bits += dc;
            int run = 0;
#pragma unroll
            for (int k = 1; k < 64; ++k) {
                const int v = q[zigzag_index(k)];
                if (v == 0) {
                    ++run;
                } else {
                    while (run >= 16) {
                        atomicAdd(&hist[pi][16 + 0xF0], 1u);
                        run -= 16;
                    }
                    const int s = category(v);
                    atomicAdd(&hist[pi][16 + ((run << 4) | s)], 1u);
                    bits += s;
                    run = 0;
                }
            }
            if (run) atomicAdd(&hist[pi][16 + 0x00], 1u);
        }
        const unsigned tot = __reduce_add_sync(0xffffffffu, bits);
        if (lane == 0 && tot) atomicAdd(&amp[pi], (unsigned long long)tot);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.nplanes * 272; i += blockDim.x) {
        const int pl = i / 272, w = i - pl * 272;
        if (hist[pl][w]) atomicAdd(a.out[pl] + w, (unsigned long long)hist[pl][w]);
    }
    if (threadIdx.x < a.nplanes && amp[threadIdx.x]) atomicAdd(a.out[threadIdx.x] + 272, amp[threadIdx.x]);
}

}  // namespace dctgb

using namespace dctgb;

extern "C" dct_status dct_entropy_stats(dct_plan_t plan, const int16_t* coeffs, const dct_plane* planes, int nplanes,
                                        uint64_t* stats_out, dct_stream_t stream) {
    if (!plan || !coeffs || !planes || !stats_out) return fail(DCT_ERR_INVALID_ARG, "null pointer");
    if (nplanes < 1 || nplanes > kMaxPlanes) return fail(DCT_ERR_INVALID_ARG, "nplanes must be 1..4");
    if (((uintptr_t)coeffs) & 15u) return fail(DCT_ERR_INVALID_ARG, "coeffs must be 16-byte aligned");
    if (((uintptr_t)stats_out) & 7u) return fail(DCT_ERR_INVALID_ARG, "stats_out must be 8-byte aligned");
    EntropyArgs a;
    memset(&a, 0, sizeof a);
    size_t off = 0;
    int tiles = 0;
    for (int i = 0; i < nplanes; ++i) {
        const dct_plane& p = planes[i];
        if (p.width < 1 || p.height < 1 || p.width > plan->desc.max_width || p.height > plan->desc.max_height)
            return fail(DCT_ERR_INVALID_ARG, "plane size outside the plan limits");
        const int nblk = ((p.width + 7) / 8) * ((p.height + 7) / 8);
        a.coef[i] = coeffs + off;
        a.out[i] = reinterpret_cast<unsigned long long*>(stats_out) + (size_t)i * kEntWords;
        a.nblk[i] = nblk;
        a.tile_begin[i] = tiles;
        tiles += (nblk + kTileBlocks - 1) / kTileBlocks;
        off += (size_t)nblk * 64;
    }
    a.tile_begin[nplanes] = tiles;
    a.nplanes = nplanes;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(stats_out, 0, sizeof(uint64_t) * kEntWords * nplanes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    // the block counts are known on the host; write them with the clear
    std::vector<uint64_t> nb(nplanes);
    for (int i = 0; i < nplanes; ++i) {
        nb[i] = (uint64_t)a.nblk[i];
        e = cudaMemcpyAsync(stats_out + (size_t)i * kEntWords + 273, &nb[i], 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "block count upload");
    }
    e = cudaStreamSynchronize(s);   // the host block counts above live on this stack frame
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int grid = (tiles + 7) / 8;
    if (grid > plan->num_sms * 4) grid = plan->num_sms * 4;
    if (grid < 1) grid = 1;
    k_entropy<<<grid, 256, 0, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? DCT_OK : cuda_fail(e, "entropy launch");
}

extern "C" double dct_entropy_bits(const uint64_t* stats_host) {
    if (!stats_host) return NAN;
    double bits = (double)stats_host[272];
    for (int part = 0; part < 2; ++part) {
        const int lo = part ? 16 : 0, hi = part ? 272 : 16;
        double n = 0.0;
        for (int i = lo; i < hi; ++i) n += (double)stats_host[i];
        for (int i = lo; i < hi; ++i)
            if (stats_host[i]) bits += (double)stats_host[i] * std::log2(n / (double)stats_host[i]);
    }
    return bits;
}

namespace dctgb {

// Codeword lengths of an optimal prefix code over the symbols with non-zero
// counts, none longer than max_len bits: package-merge (Larmore and
// Hirschberg).  Every level lists the leaves (sorted by count, then symbol)
// merged with the adjacent pairs of the previous level's list, leaves first
// on equal weights; a symbol's length is the number of times its leaf occurs
// among the first 2m - 2 items of the last level (m live symbols).  A lone
// symbol gets one bit.
static void limited_code_lengths(const uint64_t* counts, int n, int max_len, int* len) {
    struct Node {
        uint64_t w;
        int sym;      // leaf symbol, or -1 for a package
        int a, b;     // children of a package
    };
    std::vector<Node> nodes;
    std::vector<int> leaves;
    for (int i = 0; i < n; ++i) {
        len[i] = 0;
        if (counts[i]) {
            nodes.push_back(Node{counts[i], i, -1, -1});
            leaves.push_back((int)nodes.size() - 1);
        }
    }
    const int m = (int)leaves.size();
    if (m == 0) return;
    if (m == 1) {
        len[nodes[leaves[0]].sym] = 1;
        return;
    }
    std::sort(leaves.begin(), leaves.end(), [&](int x, int y) {
        return nodes[x].w != nodes[y].w ? nodes[x].w < nodes[y].w : nodes[x].sym < nodes[y].sym;
    });
    std::vector<int> cur = leaves, next, packages;
    for (int level = 1; level < max_len; ++level) {
        packages.clear();
        for (size_t k = 0; k + 1 < cur.size(); k += 2) {
            nodes.push_back(Node{nodes[cur[k]].w + nodes[cur[k + 1]].w, -1, cur[k], cur[k + 1]});
            packages.push_back((int)nodes.size() - 1);
        }
        next.clear();
        size_t x = 0, y = 0;
        while (x < leaves.size() || y < packages.size()) {
            if (y == packages.size() || (x < leaves.size() && nodes[leaves[x]].w <= nodes[packages[y]].w))
                next.push_back(leaves[x++]);
            else
                next.push_back(packages[y++]);
        }
        cur.swap(next);
    }
    std::vector<int> stack;
    for (int k = 0; k < 2 * m - 2; ++k) {
        stack.push_back(cur[k]);
        while (!stack.empty()) {
            const Node& nd = nodes[stack.back()];
            stack.pop_back();
            if (nd.sym >= 0) {
                ++len[nd.sym];
            } else {
                stack.push_back(nd.a);
                stack.push_back(nd.b);
            }
        }
    }
}

}  // namespace dctgb

extern "C" uint64_t dct_huffman_bits(const uint64_t* stats_host) {
    using namespace dctgb;
    if (!stats_host) return 0;
    uint64_t bits = stats_host[272];
    int len[256];
    for (int part = 0; part < 2; ++part) {
        const int lo = part ? 16 : 0, n = part ? 256 : 16;
        limited_code_lengths(stats_host + lo, n, kMaxCodeLen, len);
        for (int i = 0; i < n; ++i) bits += stats_host[lo + i] * (uint64_t)len[i];
    }
    return bits;
}
