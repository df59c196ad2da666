// Double-precision log, sin/cos-of-turns and atan2 built only from correctly rounded IEEE operations
// (+, -, *, /, sqrt, floor) in a fixed order.  Used by the bit-reproducible walk variant, whose translation
// unit is compiled with --fmad=false so that no multiply-add is contracted.  Any implementation performing
// the same operations in the same order obtains the same bits, which is what makes the walk's integer
// outputs (scatter counts, histogram bins) reproducible exactly.
//
//  log   : x = m 2^e, m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(s) with s = (m-1)/(m+1), the odd series of
//          atanh to z^12 (z = s^2), summed innermost first; e ln 2 added with ln 2 split into a 32-bit head
//          (exact products) and its tail.
//  turns : sin/cos(2 pi u): r = 4u - nearest integer (exact), theta = r pi/2 in [-pi/4, pi/4], Taylor
//          series of sin and cos in nested form through theta^21, quadrant from the integer.
//  atan2 : octant reduction to a in [0, 1], two half-angle reductions a -> a / (1 + sqrt(1 + a^2)) to
//          |a| <= tan(pi/16), Gregory series to a^29, times 4.
#pragma once

#include <stdint.h>

namespace ms {
namespace det {

constexpr double kLn2Head = 0x1.62e42fee00000p-1;
constexpr double kLn2Tail = 0x1.a39ef35793c76p-33;
constexpr double kRootHalf = 0x1.6a09e667f3bcdp-1;
constexpr double kHalfPi = 0x1.921fb54442d18p+0;
constexpr double kPi = 0x1.921fb54442d18p+1;
constexpr double kTwoPi = 0x1.921fb54442d18p+2;

__device__ __forceinline__ double log(double x)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7ffu) - 1022;
    double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) | 0x3fe0000000000000ull));
    if (m < kRootHalf) {
        m = m + m;
        e = e - 1;
    }
    const double s = (m - 1.0) / (m + 1.0);
    const double z = s * s;
    double acc = 1.0 / 25.0;
#pragma unroll
    for (int k = 11; k >= 0; --k) acc = acc * z + 1.0 / (double)(2 * k + 1);
    const double r = (s + s) * acc;
    const double ed = (double)e;
    return ed * kLn2Head + (ed * kLn2Tail + r);
}

__device__ __forceinline__ void sincos_turns(double u, double* sin_out, double* cos_out)
{
    const double y = 4.0 * u;
    const double nearest = floor(y + 0.5);
    const double r = y - nearest;
    const int quadrant = ((int)nearest) & 3;
    const double th = r * kHalfPi;
    const double t = th * th;
    double ps = 1.0, pc = 1.0;
#pragma unroll
    for (int k = 10; k >= 1; --k) {
        ps = 1.0 - t / (double)((2 * k) * (2 * k + 1)) * ps;
        pc = 1.0 - t / (double)((2 * k - 1) * (2 * k)) * pc;
    }
    const double sn = th * ps, cs = pc;
    if (quadrant == 0) { *sin_out = sn; *cos_out = cs; }
    else if (quadrant == 1) { *sin_out = cs; *cos_out = -sn; }
    else if (quadrant == 2) { *sin_out = -sn; *cos_out = -cs; }
    else { *sin_out = -cs; *cos_out = sn; }
}

__device__ __forceinline__ double atan_unit(double a)
{
    const double a1 = a / (1.0 + sqrt(1.0 + a * a));
    const double a2 = a1 / (1.0 + sqrt(1.0 + a1 * a1));
    const double t = a2 * a2;
    double acc = 0.0;
#pragma unroll
    for (int k = 14; k >= 0; --k) acc = acc * t + ((k & 1) ? -1.0 : 1.0) / (double)(2 * k + 1);
    return 4.0 * (a2 * acc);
}

__device__ __forceinline__ double atan2(double y, double x)
{
    const double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0) return 0.0;
    const bool swap = ay > ax;
    double th = atan_unit(swap ? ax / ay : ay / ax);
    if (swap) th = kHalfPi - th;
    if (x < 0.0) th = kPi - th;
    if (y < 0.0) th = -th;
    return th;
}

}  // namespace det
}  // namespace ms
