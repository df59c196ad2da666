/*
 * Oracle: deterministic FP64 log, sin/cos and atan2 — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The walk's integer outputs (scatter counts, histogram bins) are decided by floating point. To make
 * them reproducible bit for bit on another machine, the functions the walk needs are written here from
 * textbook series using only +, -, *, / and sqrt (each correctly rounded by IEEE 754) in a fixed order,
 * compiled without contraction (-ffp-contract=off).  Any other implementation that performs the same
 * operations in the same order gets the same bits.  Accuracy against the C library is pinned in the
 * tests (a few ulp).
 *
 *  log:  x = m * 2^e with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh(s), s = (m-1)/(m+1), summed as the
 *        odd power series of atanh; e*ln2 added with ln2 split in a 32-bit head and a tail.
 *  sin/cos of 2*pi*u ("turns"): the reduction to [-1/8, 1/8] turn is exact in binary (4u minus the
 *        nearest integer), then the Taylor series of sin and cos in nested form, then the quadrant.
 *  atan2: octant reduction to a in [0,1], two half-angle steps a -> a/(1+sqrt(1+a^2)) so that
 *        |a| <= tan(pi/16), then the Gregory series, times 4.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define OM_LN2_HI   0x1.62e42fee00000p-1
#define OM_LN2_LO   0x1.a39ef35793c76p-33
#define OM_SQRT1_2  0x1.6a09e667f3bcdp-1
#define OM_PI_2     0x1.921fb54442d18p+0
#define OM_PI       0x1.921fb54442d18p+1

double om_log(double x)
{
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7ffu) - 1022;
    uint64_t mbits = (bits & 0x000fffffffffffffull) | 0x3fe0000000000000ull;
    double m;
    memcpy(&m, &mbits, sizeof m);
    if (m < OM_SQRT1_2) {
        m = m + m;
        e = e - 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    /* sum_{k=0}^{12} z^k / (2k+1), innermost term first */
    double p = 1.0 / 25.0;
    for (int k = 11; k >= 0; --k)
        p = p * z + 1.0 / (double)(2 * k + 1);
    double r = (s + s) * p;
    double ed = (double)e;
    return ed * OM_LN2_HI + (ed * OM_LN2_LO + r);
}

void om_sincos_turns(double u, double* s_out, double* c_out)
{
    double y = 4.0 * u;
    double qf = floor(y + 0.5);
    double r = y - qf;
    int q = ((int)qf) & 3;
    double th = r * OM_PI_2;
    double t = th * th;
    /* sin(th) = th * (1 - t/(2*3) * (1 - t/(4*5) * (...))),  cos(th) = 1 - t/(1*2) * (1 - t/(3*4) * (...)) */
    double ps = 1.0, pc = 1.0;
    for (int k = 10; k >= 1; --k) {
        ps = 1.0 - t / (double)((2 * k) * (2 * k + 1)) * ps;
        pc = 1.0 - t / (double)((2 * k - 1) * (2 * k)) * pc;
    }
    double sn = th * ps;
    double cs = pc;
    switch (q) {
    case 0: *s_out = sn;  *c_out = cs;  break;
    case 1: *s_out = cs;  *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
    }
}

static double om_atan01(double a)
{
    double a1 = a / (1.0 + sqrt(1.0 + a * a));
    double a2 = a1 / (1.0 + sqrt(1.0 + a1 * a1));
    double t = a2 * a2;
    double p = 0.0;
    for (int k = 14; k >= 0; --k)
        p = p * t + ((k & 1) ? -1.0 : 1.0) / (double)(2 * k + 1);
    return 4.0 * (a2 * p);
}

double om_atan2(double y, double x)
{
    double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0)
        return 0.0;
    int swap = ay > ax;
    double a = swap ? ax / ay : ay / ax;
    double th = om_atan01(a);
    if (swap)
        th = OM_PI_2 - th;
    if (x < 0.0)
        th = OM_PI - th;
    if (y < 0.0)
        th = -th;
    return th;
}
