// Numeric spec of the fixed-point Cordic-based Loeffler codec, compiled into
// the library.  The paper (Sec. 2.5.2) fixes the structure of the flow graph
// but none of these numbers; include/dctgb_spec.json records the same
// choices and dct_spec_query() reports these so a test can compare them.
#pragma once
#include <cstdint>

namespace dctgb {

// CORDIC micro-rotations per rotation.  The spec file's value (6) is the
// default; the build can compile the same library at another count
// (-DDCTGB_CORDIC_N=4 or 5) to trade accuracy for integer operations.
#ifndef DCTGB_CORDIC_N
#define DCTGB_CORDIC_N 6
#endif

constexpr int kP = 4;              // x = (p - 128) << kP
constexpr int kN = DCTGB_CORDIC_N; // CORDIC micro-rotations, shifts 1..kN
static_assert(kN >= 3 && kN <= 12, "CORDIC iteration count outside the supported range");
constexpr int kR = 11;             // dequantiser weights carry 2^kR
constexpr int kQuantShift = 32;    // quantiser multipliers carry 2^32
constexpr int kDequantClamp = 4096;
constexpr int kPsnrMax = 255;
constexpr int kStatsWords = 80;    // uint64 statistics words per plane
constexpr int kBandShift = kP + 1; // band energy term: (|Y| >> kBandShift)^2

// ---- CORDIC direction tables, derived at compile time ---------------------
// atan(2^-i) from its Maclaurin series (|x| <= 1/2, 60 terms converge far
// below double precision) and the greedy rule: z = angle; for i = 1..N,
// s_i = +1 if z >= 0 else -1, z -= s_i * atan(2^-i).  Bit i of a mask is set
// when s_i = +1.
constexpr double cx_atan_pow2(int i) {
    double x = 1.0;
    for (int k = 0; k < i; ++k) x *= 0.5;
    const double x2 = x * x;
    double term = x, sum = 0.0;
    for (int k = 0; k < 60; ++k) {
        sum += ((k & 1) ? -term : term) / double(2 * k + 1);
        term *= x2;
    }
    return sum;
}

constexpr unsigned cx_sigma_mask(double angle, int n) {
    double z = angle;
    unsigned mask = 0u;
    for (int i = 1; i <= n; ++i) {
        const bool pos = z >= 0.0;
        if (pos) mask |= 1u << i;
        z -= (pos ? 1.0 : -1.0) * cx_atan_pow2(i);
    }
    return mask;
}

constexpr double kPi = 3.14159265358979323846264338327950288;
// (a4, a7) = rot(d3, d0, 3pi/16)
constexpr unsigned kSigOddUpper = cx_sigma_mask(3.0 * kPi / 16.0, kN);
// (a5, a6) = rot(d2, d1, pi/16)
constexpr unsigned kSigOddLower = cx_sigma_mask(kPi / 16.0, kN);
// (Y2, Y6) = rot(e2, e3, 3pi/8) = quarter turn, then rot(-pi/8)
constexpr unsigned kSigEven = cx_sigma_mask(-kPi / 8.0, kN);

}  // namespace dctgb
