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

// ---- Forward micro-rotations 2..kN in float32 --------------------------
// Every float32 of magnitude in [2^23, 2^24) is an integer, and a fused
// multiply-add rounds its exact result once.  Hold a and b as the floats
// A = alpha + a and B = beta + b, with compile-time biases alpha, beta in
// that range (either sign) and beta * 2^-i, alpha * 2^-i integers; then
//   fma round-down(B,  2^-i, A) = (alpha + beta 2^-i) + a + floor(b / 2^i)
//   fma round-up  (A, -2^-i, B) = (beta - alpha 2^-i) + b - floor(a / 2^i)
// exactly, as long as the results stay in the range: one FFMA per half
// micro-rotation in place of a shift (integer ALU pipe only) and an add.
// The biases follow the micro-rotations themselves (without floors), so
// the schedule below is fixed per rotation block and checked at compile
// time against the forward graph's node bound.  Step 1 (a 26.6 degree turn
// of the bias vector) stays in integers: no bias pair survives it inside
// the range.  The inverse graph's nodes reach 2^30 and keep the integer
// form throughout.
constexpr long long kFwdNodeBound = 1LL << 20;   // |node| of the forward graph
                                                 // at kP = 4 (interval
                                                 // propagation: 719380)
constexpr bool kFltForward = kN <= 6;             // biases need 2^(2+..+kN) | alpha

struct FltBias {
    long long a, b;
};

// Bias pair before micro-rotation i (2 <= i <= kN + 1) of a block with
// directions MASK that starts step 2 with (a0, b0).
__host__ __device__ constexpr FltBias flt_bias(unsigned mask, long long a0, long long b0, int i) {
    long long a = a0, b = b0;
    for (int j = 2; j < i; ++j) {
        const long long da = b / (1LL << j), db = a / (1LL << j);
        if ((mask >> j) & 1u) {
            a += da;
            b -= db;
        } else {
            a -= da;
            b += db;
        }
    }
    return {a, b};
}

constexpr bool flt_in_range(long long x) {
    const long long m = x < 0 ? -x : x;
    return m - kFwdNodeBound >= (1LL << 23) && m + kFwdNodeBound < (1LL << 24);
}

constexpr bool flt_schedule_ok(unsigned mask, long long a0, long long b0) {
    for (int i = 2; i <= kN + 1; ++i) {
        const FltBias p = flt_bias(mask, a0, b0, i);
        if (!flt_in_range(p.a) || !flt_in_range(p.b)) return false;
        if (i <= kN && (p.a % (1LL << i) != 0 || p.b % (1LL << i) != 0)) return false;
    }
    return true;
}

// Starting biases (multiples of 2^20), chosen by exhaustive search for the
// widest margin; one table serves kN = 3..6.
constexpr long long kFltUnit = 1LL << 20;
constexpr long long kFltOddUpperA = -13 * kFltUnit, kFltOddUpperB = 10 * kFltUnit;
constexpr long long kFltOddLowerA = -14 * kFltUnit, kFltOddLowerB = -10 * kFltUnit;
constexpr long long kFltEvenA = -13 * kFltUnit, kFltEvenB = 10 * kFltUnit;
static_assert(!kFltForward || (flt_schedule_ok(kSigOddUpper, kFltOddUpperA, kFltOddUpperB) &&
                               flt_schedule_ok(kSigOddLower, kFltOddLowerA, kFltOddLowerB) &&
                               flt_schedule_ok(kSigEven, kFltEvenA, kFltEvenB)),
              "float micro-rotation bias schedule leaves the exact-integer range");

// Bit image of the float alpha + v: for alpha + v in [2^23, 2^24) the bits
// are 0x4A800000 + alpha + v; in (-2^24, -2^23] (sign and magnitude) they
// are 0xCA800000 - alpha - v.
template <long long ALPHA>
__device__ __forceinline__ float flt_enc(int v) {
    if constexpr (ALPHA > 0)
        return __int_as_float((int)(0x4A800000u + (unsigned)ALPHA + (unsigned)v));
    else
        return __int_as_float((int)(0xCA800000u + (unsigned)(-ALPHA) - (unsigned)v));
}

template <long long ALPHA>
__device__ __forceinline__ int flt_dec(float f) {
    const unsigned bits = (unsigned)__float_as_int(f);
    if constexpr (ALPHA > 0)
        return (int)(bits - (0x4A800000u + (unsigned)ALPHA));
    else
        return (int)(0xCA800000u + (unsigned)(-ALPHA) - bits);
}

template <unsigned MASK, int I>
__device__ __forceinline__ void cordic_fwd_flt_from(float& a, float& b) {
    if constexpr (I <= kN) {
        constexpr float sc = 1.0f / float(1 << I);   // exact power of two
        float na, nb;
        if constexpr ((MASK >> I) & 1u) {
            na = __fmaf_rd(b, sc, a);     // a + floor(b / 2^I)
            nb = __fmaf_ru(a, -sc, b);    // b - floor(a / 2^I)
        } else {
            na = __fmaf_ru(b, -sc, a);    // a - floor(b / 2^I)
            nb = __fmaf_rd(a, sc, b);     // b + floor(a / 2^I)
        }
        a = na;
        b = nb;
        cordic_fwd_flt_from<MASK, I + 1>(a, b);
    }
}

template <unsigned MASK, long long A0, long long B0>
__device__ __forceinline__ void cordic_fwd_flt(int& a, int& b) {
    int a1, b1;
    if constexpr ((MASK >> 1) & 1u) {
        a1 = add_shr<1>(a, b);
        b1 = sub_shr<1>(b, a);
    } else {
        a1 = sub_shr<1>(a, b);
        b1 = add_shr<1>(b, a);
    }
    float fa = flt_enc<A0>(a1), fb = flt_enc<B0>(b1);
    cordic_fwd_flt_from<MASK, 2>(fa, fb);
    constexpr FltBias e = flt_bias(MASK, A0, B0, kN + 1);
    a = flt_dec<e.a>(fa);
    b = flt_dec<e.b>(fb);
}

template <unsigned MASK, long long A0 = 0, long long B0 = 0>
__device__ __forceinline__ void cordic_fwd(int& a, int& b) {
    if constexpr (kFltForward && (A0 != 0 || B0 != 0))
        cordic_fwd_flt<MASK, A0, B0>(a, b);
    else
        cordic_fwd_from<MASK, 1>(a, b);
}

template <unsigned MASK>
__device__ __forceinline__ void cordic_tr(int& a, int& b) { cordic_tr_from<MASK, 1>(a, b); }

// Forward 8-point graph on v[0..7] (in place: v[k] <- Y_k); FLT selects
// the float form of micro-rotations 2..kN (same results, bit for bit).
template <bool FLT>
__device__ __forceinline__ void loeffler8_fwd(int (&v)[8]) {
    constexpr bool F = FLT && kFltForward;
    constexpr long long UA = F ? kFltOddUpperA : 0, UB = F ? kFltOddUpperB : 0;
    constexpr long long LA = F ? kFltOddLowerA : 0, LB = F ? kFltOddLowerB : 0;
    constexpr long long EA = F ? kFltEvenA : 0, EB = F ? kFltEvenB : 0;
    const int s0 = v[0] + v[7], d0 = v[0] - v[7];
    const int s1 = v[1] + v[6], d1 = v[1] - v[6];
    const int s2 = v[2] + v[5], d2 = v[2] - v[5];
    const int s3 = v[3] + v[4], d3 = v[3] - v[4];
    const int e0 = s0 + s3, e3 = s0 - s3;
    const int e1 = s1 + s2, e2 = s1 - s2;
    int a4 = d3, a7 = d0;
    cordic_fwd<kSigOddUpper, UA, UB>(a4, a7);
    int a5 = d2, a6 = d1;
    cordic_fwd<kSigOddLower, LA, LB>(a5, a6);
    int y2 = e3, y6 = -e2;             // quarter turn of (e2, e3)
    cordic_fwd<kSigEven, EA, EB>(y2, y6);
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
template <bool FLT>
__device__ __forceinline__ void fwd2d(int (&x)[8][8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) loeffler8_fwd<FLT>(x[i]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = x[i][j];
        loeffler8_fwd<FLT>(c);
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
