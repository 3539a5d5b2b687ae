// expneg.cuh -- e^{-x} for the lapse factor F = A e^{-delta} of Eqs. (eq:phi), (eq:pi).
// Two entry points: a_exp_neg(A, x) for x in natural units, a_exp_neg_scaled(A, X) for
// X = x * 256/ln2.
//
// Method: Tang's table-driven exponential (P. T. P. Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989), written from
// the published method: with y = -x,
//   y = (256 m + j) ln2/256 + r,  0 <= j < 256,  |r| <= ln2/512,
//   e^y = 2^m * 2^{j/256} * e^r,  e^r - 1 = r + r^2/2 + r^3/6 + r^4/24 + O(r^5),
// where the O(r^5) remainder is below 4e-17 for |r| <= ln2/512.  The reduction uses the
// round-to-integer shift constant 1.5*2^52 and a two-term (Cody-Waite) ln2/256 with FMAs, the
// table holds 2^{j/256} rounded to double, and 2^m is applied by integer addition to the
// exponent field of the table entry.  The caller's factor A is applied in the same FMA:
//   A e^{-x} = fma(A t, p, A t),  t = 2^m 2^{j/256},  p = e^r - 1,
// ten FP64 instructions in all (the library's double exp costs about twenty FP64 issue slots on
// this part).  Accuracy: within 2 ulp of the exact value for x in [0, 700]; the result is 0 for
// x > 700 (e^{-700} ~ 1e-304) and NaN for NaN input.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace adscl {

// Additions and plain multiplications issued as FMAs.  On this part DADD and DMUL issue at about
// 0.84 of the DFMA rate, while fma(x, 1, y) = x + y and fma(x, y, -0) = x * y exactly (the product
// by 1 is exact; adding -0 leaves every product, +0 included, unchanged under round-to-nearest)
// run at the DFMA rate.  The 1 and the -0 live in constant memory, where the compiler cannot see
// their values and fold the FMAs back into DADD / DMUL.
static __constant__ double c_fp_one = 1.0;
static __constant__ double c_fp_negzero = -0.0;
__device__ __forceinline__ double add_f(double x, double y) { return fma(x, c_fp_one, y); }
__device__ __forceinline__ double mul_f(double x, double y) { return fma(x, y, c_fp_negzero); }
// -x by flipping the sign bit on the integer pipe (IEEE negation, NaN payloads included), for the
// parity ghosts that only a few threads write: no FP64 instruction that every lane would issue
__device__ __forceinline__ double neg_bits(double x)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

constexpr int kExpTableSize = 256;

// two-term split of ln2/256: L1 = RN(ln2/256), L2 = RN(ln2/256 - L1)
constexpr double kLn2o256Hi = 0.0027076061740622863;
constexpr double kLn2o256Lo = 9.058776616587108e-20;
constexpr double kInvLn2x256 = 369.3299304675746;  // 256 / ln 2
constexpr double kShift = 6755399441055744.0;      // 1.5 * 2^52
constexpr int kExpNMin = -258531;                   // n below this: x > 700, result 0

// A * e^{-x} with the table `tab` (2^{j/256}, j < 256), normally in shared memory
__device__ __forceinline__ double a_exp_neg(double A, double x, const double *tab)
{
    const double y = -x;
    const double nf = fma(y, kInvLn2x256, kShift);
    const int n = __double2loint(nf);  // round(y * 256/ln2), exact integer in the low bits
    const double nd = add_f(nf, -kShift);
    double r = fma(-nd, kLn2o256Hi, y);
    r = fma(-nd, kLn2o256Lo, r);
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r, p, 1.0);
    p = mul_f(r, p);                   // e^r - 1
    const int j = n & (kExpTableSize - 1);
    const int m = n >> 8;              // floor(n / 256)
    const long long tb = __double_as_longlong(tab[j]) + ((long long)m << 52);
    double t = __longlong_as_double(tb);
    if (n < kExpNMin) t = 0.0;
    const double at = A * t;
    return fma(at, p, at);
}

// A e^{-x} from its argument given in units of ln2/256, X = x * 256/ln2 (the solver accumulates
// delta in these units, so the reduction needs no split of ln2/256): with n = round(-X), the
// remainder z = -X - n is exact (|z| <= 1/2, Sterbenz), and
//   e^{-x} = 2^{n/256} e^{z L},  e^{z L} - 1 = z (c1 + z (c2 + z (c3 + z c4))),  ck = L^k / k!,
// L = ln2/256; the degree-4 remainder is below 4e-17 for |z L| <= L/2.  Nine FP64 instructions.
// Accuracy: within 2 ulp of e^{-X L} for X in [0, 258531] (x up to 700); 0 for X in
// (258531, 2^51); NaN for NaN.
constexpr double kKappa = kInvLn2x256;     // 256 / ln 2
constexpr double kInvKappa = kLn2o256Hi;   // RN(ln 2 / 256)
constexpr double kExpC2 = 3.6655655969101062e-06;   // RN(L^2 / 2)
constexpr double kExpC3 = 3.3083026805413713e-09;   // RN(L^3 / 6)
constexpr double kExpC4 = 2.239395190875157e-12;    // RN(L^4 / 24)

__device__ __forceinline__ double a_exp_neg_scaled(double A, double X, const double *tab)
{
    const double nf = add_f(-X, kShift);   // kShift + round(-X): the integer n in the low bits
    const int n = __double2loint(nf);
    const double nd = add_f(nf, -kShift);  // n, exactly
    const double z = add_f(-X, -nd);       // exact
    double p = fma(z, kExpC4, kExpC3);
    p = fma(z, p, kExpC2);
    p = fma(z, p, kInvKappa);
    p = mul_f(z, p);                       // e^{z L} - 1
    const int j = n & (kExpTableSize - 1);
    const int m = n >> 8;
    const long long tb = __double_as_longlong(tab[j]) + ((long long)m << 52);
    double t = __longlong_as_double(tb);
    if (n < kExpNMin) t = 0.0;
    const double at = A * t;
    return fma(at, p, at);
}

}  // namespace adscl
