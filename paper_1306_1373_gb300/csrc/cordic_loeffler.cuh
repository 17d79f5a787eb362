// Device flow graphs of the Cordic-based Loeffler 8-point DCT (Sec. 2.5.2,
// Fig. 1) and its transpose, in int32 registers.
//
// Forward graph (standard Loeffler structure, four stages in series):
//   stage 1  s_n = x_n + x_{7-n}, d_n = x_n - x_{7-n}
//   stage 2  even e0 = s0+s3, e3 = s0-s3, e1 = s1+s2, e2 = s1-s2;
//            odd  (a4,a7) = rot(d3,d0,3pi/16), (a5,a6) = rot(d2,d1,pi/16)
//   stage 3  Y0 = e0+e1, Y4 = e0-e1, (Y2,Y6) = rot(e2,e3,3pi/8);
//            b4 = a4+a6, b6 = a4-a6, b7 = a7+a5, b5 = a7-a5
//   stage 4  Y1 = b7+b4, Y7 = b7-b4, Y3 = b5, Y5 = b6
// Every rot() is a CORDIC block of kN shift-add micro-rotations
// (a, b) <- (a + s (b >> i), b - s (a >> i)), i = 1..kN, arithmetic shifts;
// 3pi/8 is the exact quarter turn (a, b) -> (b, -a) followed by a CORDIC
// rotation of -pi/8.  The sqrt(2) factors of stage 4 and the CORDIC gain are
// not computed: the quantiser and dequantiser tables absorb them.
//
// The inverse graph is the transpose: steps in reverse order, butterflies
// unchanged, each micro-rotation with -s in ascending i, and the quarter
// turn's transpose (a, b) -> (-b, a).
#pragma once
#include "dctgb_spec.h"


namespace dctgb {

// acc + (v >> I) with an arithmetic (floor) shift: a shift and an add, both
// at the full integer issue rate on this GPU (dct_int_peak kind 0 measures
// 127 of 128 operations per clock per SM).  A single mad.hi.s32 computes
// the same value (the high word of v * 2^(32-I)), but it issues at about a
// quarter of that rate: using it for one half of each micro-rotation
// (dct_int_peak kind 1) measured 80 operations per clock per SM, and made
// the fused codec step 29% slower with byte-identical outputs.
template <int I>
__device__ __forceinline__ int add_shr(int acc, int v) {
    return acc + (v >> I);
}

template <int I>
__device__ __forceinline__ int sub_shr(int acc, int v) {
    return acc - (v >> I);
}

// Micro-rotations I..kN with the directions of MASK (bit i set: s_i = +1):
// (a, b) <- (a + s_i (b >> i), b - s_i (a >> i)) from the pre-step values.
template <unsigned MASK, int I>
__device__ __forceinline__ void cordic_fwd_from(int& a, int& b) {
    if constexpr (I <= kN) {
        int na, nb;
        if constexpr ((MASK >> I) & 1u) {
            na = add_shr<I>(a, b);
            nb = sub_shr<I>(b, a);
        } else {
            na = sub_shr<I>(a, b);
            nb = add_shr<I>(b, a);
        }
        a = na;
        b = nb;
        cordic_fwd_from<MASK, I + 1>(a, b);
    }
}

// Transposed micro-rotations: the same shifts with -s_i, ascending i.
template <unsigned MASK, int I>
__device__ __forceinline__ void cordic_tr_from(int& a, int& b) {
    if constexpr (I <= kN) {
        int na, nb;
        if constexpr ((MASK >> I) & 1u) {
            na = sub_shr<I>(a, b);
            nb = add_shr<I>(b, a);
        } else {
            na = add_shr<I>(a, b);
            nb = sub_shr<I>(b, a);
        }
        a = na;
        b = nb;
        cordic_tr_from<MASK, I + 1>(a, b);
    }
}

template <unsigned MASK>
__device__ __forceinline__ void cordic_fwd(int& a, int& b) { cordic_fwd_from<MASK, 1>(a, b); }

template <unsigned MASK>
__device__ __forceinline__ void cordic_tr(int& a, int& b) { cordic_tr_from<MASK, 1>(a, b); }

// Forward 8-point graph on v[0..7] (in place: v[k] <- Y_k).
__device__ __forceinline__ void loeffler8_fwd(int (&v)[8]) {
    const int s0 = v[0] + v[7], d0 = v[0] - v[7];
    const int s1 = v[1] + v[6], d1 = v[1] - v[6];
    const int s2 = v[2] + v[5], d2 = v[2] - v[5];
    const int s3 = v[3] + v[4], d3 = v[3] - v[4];
    const int e0 = s0 + s3, e3 = s0 - s3;
    const int e1 = s1 + s2, e2 = s1 - s2;
    int a4 = d3, a7 = d0;
    cordic_fwd<kSigOddUpper>(a4, a7);
    int a5 = d2, a6 = d1;
    cordic_fwd<kSigOddLower>(a5, a6);
    int y2 = e3, y6 = -e2;             // quarter turn of (e2, e3)
    cordic_fwd<kSigEven>(y2, y6);
    const int b4 = a4 + a6, b6 = a4 - a6;
    const int b7 = a7 + a5, b5 = a7 - a5;
    v[0] = e0 + e1;
    v[4] = e0 - e1;
    v[2] = y2;
    v[6] = y6;
    v[1] = b7 + b4;
    v[7] = b7 - b4;
    v[3] = b5;
    v[5] = b6;
}

// Transposed (inverse) 8-point graph on v[0..7] (in place: v[n] <- x_n).
__device__ __forceinline__ void loeffler8_inv(int (&v)[8]) {
    const int b7 = v[1] + v[7], b4 = v[1] - v[7];
    const int b5 = v[3], b6 = v[5];
    int a4 = b4 + b6, a6 = b4 - b6;
    int a7 = b7 + b5, a5 = b7 - b5;
    const int e0 = v[0] + v[4], e1 = v[0] - v[4];
    int p = v[2], q = v[6];
    cordic_tr<kSigEven>(p, q);
    const int e2 = -q, e3 = p;         // transposed quarter turn
    cordic_tr<kSigOddUpper>(a4, a7);   // -> (d3, d0)
    cordic_tr<kSigOddLower>(a5, a6);   // -> (d2, d1)
    const int s0 = e0 + e3, s3 = e0 - e3;
    const int s1 = e1 + e2, s2 = e1 - e2;
    v[0] = s0 + a7;
    v[7] = s0 - a7;
    v[1] = s1 + a6;
    v[6] = s1 - a6;
    v[2] = s2 + a5;
    v[5] = s2 - a5;
    v[3] = s3 + a4;
    v[4] = s3 - a4;
}

// 2-D forward: rows (points along the column index j), then columns.
__device__ __forceinline__ void fwd2d(int (&x)[8][8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) loeffler8_fwd(x[i]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = x[i][j];
        loeffler8_fwd(c);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i][j] = c[i];
    }
}

// 2-D inverse: columns first, then rows (the transpose of fwd2d).
__device__ __forceinline__ void inv2d(int (&x)[8][8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = x[i][j];
        loeffler8_inv(c);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i][j] = c[i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) loeffler8_inv(x[i]);
}

}  // namespace dctgb
