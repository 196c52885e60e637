// FP64 exponential for the step kernel, after the table-driven method of
// P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989:
//
//   x = (32 m + j) ln2/32 + r,  |r| <= ln2/64,  0 <= j < 32
//   exp(x) = 2^m * 2^(j/32) * (1 + p(r)),  p(r) = exp(r) - 1
//
// N = 32 m + j is x * 32/ln2 rounded to the nearest integer (by adding 1.5 * 2^52,
// which leaves N in the low bits of the sum); r is formed with ln2/32 split into
// its double rounding and the remainder (Cody and Waite), so N * ln2/32 is
// subtracted to well below one ulp of r. p is the Taylor polynomial of exp(r) - 1
// to degree 6, whose remainder r^7/7! < 4e-18 stays below the rounding of the
// result; 2^(j/32) comes from a 32-entry table set on the host. The scaling by 2^m
// adds m to the exponent field. The result is within 2 ulp of exp(x) over
// -707 < x <= 709; below -707 (results under ~1e-307, down to the subnormal range)
// it is 0, above 709 it is +inf, and NaN propagates.
#pragma once

#include <cmath>

namespace m2m {

// 2^(j/32), j = 0 .. 31, rounded to double (set by exp2_table on the host). Each
// translation unit holds its own copy.
static __constant__ double kExp2j[32];

inline void exp2_table(double t[32])
{
    for (int j = 0; j < 32; ++j) t[j] = double(std::exp2((long double)j / 32.0L));
}

__device__ __forceinline__ double exp_tab(double x, const double *e2)
{
    constexpr double kInvL = 46.166241308446829036;      // 32 / ln 2
    constexpr double kL1 = 0.021660849392498290;         // ln2/32 rounded to double
    constexpr double kL2 = 7.2470212932696862984e-19;    // ln2/32 - kL1
    constexpr double kShift = 6755399441055744.0;        // 1.5 * 2^52
    // |x| < 707 on the bit pattern (one integer compare); the rest, NaN included,
    // takes the slow branch
    if ((__double_as_longlong(x) & 0x7fffffffffffffffll) >= 0x4086180000000000ll) {
        if (!(x > -707.0)) return x != x ? x : 0.0;
        if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    }
    const double t = fma(x, kInvL, kShift);
    const int N = __double2loint(t);
    const double Nd = t - kShift;
    double r = fma(Nd, -kL1, x);
    r = fma(Nd, -kL2, r);
    double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r * r, r);
    const double tj = e2[N & 31];
    const double res = fma(tj, p, tj);
    const long long m = (long long)(N >> 5);  // floor(N / 32)
    return __longlong_as_double(__double_as_longlong(res) + (m << 52));
}

}  // namespace m2m
