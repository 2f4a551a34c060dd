// expcr.cuh -- correctly rounded binary64 exp and pow for the FP64 step.
//
// psi = exp(-1/n) (Sec. IV B of the paper) must be rounded identically on
// every platform for FP64 results to be reproducible bit for bit, so the
// library evaluates exp(x) to ~2^-100 relative accuracy and rounds once.
//
// Method (standard published techniques, written for this library):
//   * argument reduction x = k ln2 + r, |r| <= ln2/2, with ln2 split in three
//     parts L1 + L2 + L3 (Cody & Waite 1980): L1 and L2 carry 32 significant
//     bits so k*L1 and k*L2 are exact for |k| < 2^21, and x - k*L1 is exact by
//     Sterbenz's lemma;
//   * r kept as a double-double (Dekker 1971 TwoSum/TwoProduct, the product
//     error taken with an FMA);
//   * s = r / 2^10, expm1(s) by its Taylor series to degree 9 in
//     double-double (truncation below 2^-110 relative), then ten doublings
//     p <- 2p + p^2 (expm1(2s) = 2 expm1(s) + expm1(s)^2), which keep the
//     relative error of p near the double-double level;
//   * y = 1 + p; the result 2^k y is rounded once: for normal results the
//     high word of the normalised pair is RN(y) and scaling by 2^k is exact;
//     for subnormal results the rounding to the 2^-1074 grid is done on the
//     pair explicitly (ties to even).
//   * a result whose pair lies within 2^-97 relative of a rounding boundary
//     cannot be certified; it is counted in *ambiguous (probability about
//     2^-45 per call) and the nearest-pair rounding is returned.
#pragma once
#include <cuda_runtime.h>

namespace sclbm {

struct ddv { double hi, lo; };

__device__ __forceinline__ ddv dd_two_sum(double a, double b) {
    double s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ddv dd_fast_two_sum(double a, double b) {  // |a| >= |b|
    double s = __dadd_rn(a, b);
    double e = __dsub_rn(b, __dsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ddv dd_add(ddv a, ddv b) {
    ddv s = dd_two_sum(a.hi, b.hi);
    ddv t = dd_two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ddv dd_mul(ddv a, ddv b) {
    double p = __dmul_rn(a.hi, b.hi);
    double e = __fma_rn(a.hi, b.hi, -p);
    e = __fma_rn(a.hi, b.lo, e);
    e = __fma_rn(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}

// 2^k exp(r) for a double-double argument x = x.hi + x.lo (|x.lo| <= ulp(x.hi)/2),
// rounded once; tol_rel is the relative half-width of the interval in which
// the exact result is known to lie (the pair's own error plus the argument's),
// used to certify the rounding.  *ambiguous is incremented (atomically, if
// non-null) when the rounding cannot be certified.
__device__ inline double exp_dd_cr(ddv x, double tol_rel, unsigned long long *ambiguous) {
    if (x.hi != x.hi) return x.hi;
    if (x.hi > 709.8) return __longlong_as_double(0x7ff0000000000000ULL);
    if (x.hi < -745.2) return 0.0;
    if (x.hi == 0.0 && x.lo == 0.0) return 1.0;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    const double L1 = 0x1.62e42fee00000p-1;
    const double L2 = 0x1.a39ef35600000p-33;
    const double L3 = 0x1.93c7673007e5fp-65;
    double kd = rint(__dmul_rn(x.hi, INV_LN2));
    double r1 = __dsub_rn(x.hi, __dmul_rn(kd, L1));       // exact
    ddv r = dd_two_sum(r1, -__dmul_rn(kd, L2));            // kd*L2 exact
    r.lo = __dadd_rn(r.lo, __dsub_rn(x.lo, __dmul_rn(kd, L3)));
    r = dd_fast_two_sum(r.hi, r.lo);
    // s = r / 2^10 (exact)
    ddv s = {__dmul_rn(r.hi, 0x1p-10), __dmul_rn(r.lo, 0x1p-10)};
    // Horner for 1/9! + s(...)... down to 1/2, then q*s+1, then *s
    const double C_HI[8] = {0x1.0000000000000p-1, 0x1.5555555555555p-3,
                            0x1.5555555555555p-5, 0x1.1111111111111p-7,
                            0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
                            0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19};
    const double C_LO[8] = {0.0, 0x1.5555555555555p-57, 0x1.5555555555555p-59,
                            0x1.1111111111111p-63, -0x1.f49f49f49f49fp-65,
                            0x1.a01a01a01a01ap-73, 0x1.a01a01a01a01ap-76,
                            -0x1.c154f8ddc6c00p-73};
    ddv q = {C_HI[7], C_LO[7]};
#pragma unroll
    for (int k = 6; k >= 0; --k) q = dd_add(dd_mul(q, s), ddv{C_HI[k], C_LO[k]});
    q = dd_add(dd_mul(q, s), ddv{1.0, 0.0});
    ddv p = dd_mul(q, s);                                  // expm1(s)
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        ddv p2 = dd_mul(p, p);
        p = dd_add(ddv{__dmul_rn(p.hi, 2.0), __dmul_rn(p.lo, 2.0)}, p2);
    }
    ddv y = dd_add(ddv{1.0, 0.0}, p);                      // exp(r), normalised
    int k = (int)kd;
    const double tol = __dmul_rn(y.hi, tol_rel);
    if (k > -1022) {
        // certify: distance of y.lo to the half-ulp midpoints around y.hi
        double up = __dsub_rn(__longlong_as_double(__double_as_longlong(y.hi) + 1), y.hi);
        double dn = __dsub_rn(y.hi, __longlong_as_double(__double_as_longlong(y.hi) - 1));
        double dist = y.lo >= 0.0 ? __dsub_rn(__dmul_rn(up, 0.5), y.lo)
                                  : __dadd_rn(__dmul_rn(dn, 0.5), y.lo);
        if (dist < tol && ambiguous) atomicAdd(ambiguous, 1ULL);
        return scalbn(y.hi, k);                            // exact scaling (or inf)
    }
    // subnormal or underflowing result: round (y.hi + y.lo) * 2^(k+1074) to
    // an integer, ties to even.
    int e = k + 1074;
    if (e <= -2) return 0.0;
    double H = scalbn(y.hi, e), Lw = scalbn(y.lo, e);
    double N = rint(H);
    double d = __dsub_rn(H, N);
    if (d == 0.5) {
        if (Lw > 0.0) N = __dadd_rn(N, 1.0);
    } else if (d == -0.5) {
        if (Lw < 0.0) N = __dsub_rn(N, 1.0);
    }
    if ((fabs(d) == 0.5 && fabs(Lw) < scalbn(tol, e)) && ambiguous) atomicAdd(ambiguous, 1ULL);
    return scalbn(N, -1074);
}

// exp(x) correctly rounded (see header comment).
__device__ inline double exp_cr(double x, unsigned long long *ambiguous) {
    return exp_dd_cr(ddv{x, 0.0}, 0x1p-97, ambiguous);
}

// ln(r) for a positive finite double r, as a double-double with relative
// error below about 2^-102:
//   r = m 2^k with m in [sqrt(1/2), sqrt(2)); ln r = k ln2 + 2 atanh(s),
//   s = (m - 1)/(m + 1) (|s| <= 0.1716; m - 1 is exact by Sterbenz's lemma,
//   the quotient formed in double-double), and
//   atanh(s) = s (1 + s^2/3 + s^4/5 + ...) summed to s^40 (truncation
//   below 2^-106 relative) by Horner in double-double; ln2 in the three
//   parts of exp_dd_cr (k L1, k L2 exact).
__device__ inline ddv log_dd(double r) {
    int k0 = 0;
    if (r < 0x1p-1022) {   // subnormal: scale into the normal range (exact)
        r = __dmul_rn(r, 0x1p54);
        k0 = -54;
    }
    long long bits = __double_as_longlong(r);
    int k = (int)((bits >> 52) & 0x7ff) - 1023 + k0;
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    if (m > 1.4142135623730951) {
        m = __dmul_rn(m, 0.5);   // exact
        k += 1;
    }
    const double a = __dsub_rn(m, 1.0);                    // exact
    const ddv b = dd_two_sum(m, 1.0);
    // s = a / b in double-double
    const double q1 = __ddiv_rn(a, b.hi);
    const ddv qb = dd_mul(ddv{q1, 0.0}, b);
    const ddv rem = dd_add(ddv{a, 0.0}, ddv{-qb.hi, -qb.lo});
    const double q2 = __ddiv_rn(rem.hi, b.hi);
    const ddv s = dd_fast_two_sum(q1, q2);
    const ddv s2 = dd_mul(s, s);
    // Horner: t = 1/41, t = 1/(2j+1) + s2 t, j = 19 .. 0
    ddv t = ddv{__ddiv_rn(1.0, 41.0), 0.0};
    {
        const double h = t.hi;
        t.lo = __ddiv_rn(__fma_rn(-h, 41.0, 1.0), 41.0);
    }
#pragma unroll 1
    for (int j = 19; j >= 0; --j) {
        const double d = (double)(2 * j + 1);
        const double h = __ddiv_rn(1.0, d);
        const ddv inv = ddv{h, __ddiv_rn(__fma_rn(-h, d, 1.0), d)};
        t = dd_add(inv, dd_mul(s2, t));
    }
    ddv at = dd_mul(s, t);                                  // atanh(s)
    at = ddv{__dmul_rn(at.hi, 2.0), __dmul_rn(at.lo, 2.0)}; // ln m
    const double L1 = 0x1.62e42fee00000p-1;
    const double L2 = 0x1.a39ef35600000p-33;
    const double L3 = 0x1.93c7673007e5fp-65;
    const double kd = (double)k;
    ddv kl = dd_two_sum(__dmul_rn(kd, L1), __dmul_rn(kd, L2));   // both products exact
    kl.lo = __dadd_rn(kl.lo, __dmul_rn(kd, L3));
    return dd_add(kl, at);
}

// r^e correctly rounded for a positive finite double r and e > 0 (the
// pseudopotential psi_eps = (n/(eps+n))^(1/eps), eq. psieps): exp of the
// double-double e ln r.  The argument carries an absolute error of about
// |e ln r| 2^-100, widened into the certification interval.
__device__ inline double pow_cr(double r, double e, unsigned long long *ambiguous) {
    if (r == 1.0) return 1.0;
    const ddv l = log_dd(r);
    const ddv y = dd_mul(l, ddv{e, 0.0});
    const double ay = fabs(y.hi);
    const double tol = 0x1p-97 + __dmul_rn(ay, 0x1p-98);
    return exp_dd_cr(y, tol, ambiguous);
}

}  // namespace sclbm
