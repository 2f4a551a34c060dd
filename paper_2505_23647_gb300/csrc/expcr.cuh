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
// exp_cr first tries a quick phase (exp_quick: Tang's table-driven method to
// 2^-64 relative, accepted only when the rounding is certified with a 2^-60
// margin, Ziv's strategy); about 1 % of arguments fall through to the
// double-double evaluation above.  pow_cr likewise tries a table-driven
// logarithm and the same exp first (pow_quick).  Both phases return the
// correctly rounded value.
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

// 2^(j/64), j = 0..63, as double-double pairs (gen_exp_table.py, 80 digits)
__device__ const double EXP2_J64[64][2] = {
    {0x1.0000000000000p+0, 0x0.0p+0},   // 2^(0/64)
    {0x1.02c9a3e778061p+0, -0x1.19083535b085dp-56},   // 2^(1/64)
    {0x1.059b0d3158574p+0, 0x1.d73e2a475b465p-55},   // 2^(2/64)
    {0x1.0874518759bc8p+0, 0x1.186be4bb284ffp-57},   // 2^(3/64)
    {0x1.0b5586cf9890fp+0, 0x1.8a62e4adc610bp-54},   // 2^(4/64)
    {0x1.0e3ec32d3d1a2p+0, 0x1.03a1727c57b53p-59},   // 2^(5/64)
    {0x1.11301d0125b51p+0, -0x1.6c51039449b3ap-54},   // 2^(6/64)
    {0x1.1429aaea92de0p+0, -0x1.32fbf9af1369ep-54},   // 2^(7/64)
    {0x1.172b83c7d517bp+0, -0x1.19041b9d78a76p-55},   // 2^(8/64)
    {0x1.1a35beb6fcb75p+0, 0x1.e5b4c7b4968e4p-55},   // 2^(9/64)
    {0x1.1d4873168b9aap+0, 0x1.e016e00a2643cp-54},   // 2^(10/64)
    {0x1.2063b88628cd6p+0, 0x1.dc775814a8495p-55},   // 2^(11/64)
    {0x1.2387a6e756238p+0, 0x1.9b07eb6c70573p-54},   // 2^(12/64)
    {0x1.26b4565e27cddp+0, 0x1.2bd339940e9d9p-55},   // 2^(13/64)
    {0x1.29e9df51fdee1p+0, 0x1.612e8afad1255p-55},   // 2^(14/64)
    {0x1.2d285a6e4030bp+0, 0x1.0024754db41d5p-54},   // 2^(15/64)
    {0x1.306fe0a31b715p+0, 0x1.6f46ad23182e4p-55},   // 2^(16/64)
    {0x1.33c08b26416ffp+0, 0x1.32721843659a6p-54},   // 2^(17/64)
    {0x1.371a7373aa9cbp+0, -0x1.63aeabf42eae2p-54},   // 2^(18/64)
    {0x1.3a7db34e59ff7p+0, -0x1.5e436d661f5e3p-56},   // 2^(19/64)
    {0x1.3dea64c123422p+0, 0x1.ada0911f09ebcp-55},   // 2^(20/64)
    {0x1.4160a21f72e2ap+0, -0x1.ef3691c309278p-58},   // 2^(21/64)
    {0x1.44e086061892dp+0, 0x1.89b7a04ef80d0p-59},   // 2^(22/64)
    {0x1.486a2b5c13cd0p+0, 0x1.3c1a3b69062f0p-56},   // 2^(23/64)
    {0x1.4bfdad5362a27p+0, 0x1.d4397afec42e2p-56},   // 2^(24/64)
    {0x1.4f9b2769d2ca7p+0, -0x1.4b309d25957e3p-54},   // 2^(25/64)
    {0x1.5342b569d4f82p+0, -0x1.07abe1db13cadp-55},   // 2^(26/64)
    {0x1.56f4736b527dap+0, 0x1.9bb2c011d93adp-54},   // 2^(27/64)
    {0x1.5ab07dd485429p+0, 0x1.6324c054647adp-54},   // 2^(28/64)
    {0x1.5e76f15ad2148p+0, 0x1.ba6f93080e65ep-54},   // 2^(29/64)
    {0x1.6247eb03a5585p+0, -0x1.383c17e40b497p-54},   // 2^(30/64)
    {0x1.6623882552225p+0, -0x1.bb60987591c34p-54},   // 2^(31/64)
    {0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54},   // 2^(32/64)
    {0x1.6dfb23c651a2fp+0, -0x1.bbe3a683c88abp-57},   // 2^(33/64)
    {0x1.71f75e8ec5f74p+0, -0x1.16e4786887a99p-55},   // 2^(34/64)
    {0x1.75feb564267c9p+0, -0x1.0245957316dd3p-54},   // 2^(35/64)
    {0x1.7a11473eb0187p+0, -0x1.41577ee04992fp-55},   // 2^(36/64)
    {0x1.7e2f336cf4e62p+0, 0x1.05d02ba15797ep-56},   // 2^(37/64)
    {0x1.82589994cce13p+0, -0x1.d4c1dd41532d8p-54},   // 2^(38/64)
    {0x1.868d99b4492edp+0, -0x1.fc6f89bd4f6bap-54},   // 2^(39/64)
    {0x1.8ace5422aa0dbp+0, 0x1.6e9f156864b27p-54},   // 2^(40/64)
    {0x1.8f1ae99157736p+0, 0x1.5cc13a2e3976cp-55},   // 2^(41/64)
    {0x1.93737b0cdc5e5p+0, -0x1.75fc781b57ebcp-57},   // 2^(42/64)
    {0x1.97d829fde4e50p+0, -0x1.d185b7c1b85d1p-54},   // 2^(43/64)
    {0x1.9c49182a3f090p+0, 0x1.c7c46b071f2bep-56},   // 2^(44/64)
    {0x1.a0c667b5de565p+0, -0x1.359495d1cd533p-54},   // 2^(45/64)
    {0x1.a5503b23e255dp+0, -0x1.d2f6edb8d41e1p-54},   // 2^(46/64)
    {0x1.a9e6b5579fdbfp+0, 0x1.0fac90ef7fd31p-54},   // 2^(47/64)
    {0x1.ae89f995ad3adp+0, 0x1.7a1cd345dcc81p-54},   // 2^(48/64)
    {0x1.b33a2b84f15fbp+0, -0x1.2805e3084d708p-57},   // 2^(49/64)
    {0x1.b7f76f2fb5e47p+0, -0x1.5584f7e54ac3bp-56},   // 2^(50/64)
    {0x1.bcc1e904bc1d2p+0, 0x1.23dd07a2d9e84p-55},   // 2^(51/64)
    {0x1.c199bdd85529cp+0, 0x1.11065895048ddp-55},   // 2^(52/64)
    {0x1.c67f12e57d14bp+0, 0x1.2884dff483cadp-54},   // 2^(53/64)
    {0x1.cb720dcef9069p+0, 0x1.503cbd1e949dbp-56},   // 2^(54/64)
    {0x1.d072d4a07897cp+0, -0x1.cbc3743797a9cp-54},   // 2^(55/64)
    {0x1.d5818dcfba487p+0, 0x1.2ed02d75b3707p-55},   // 2^(56/64)
    {0x1.da9e603db3285p+0, 0x1.c2300696db532p-54},   // 2^(57/64)
    {0x1.dfc97337b9b5fp+0, -0x1.1a5cd4f184b5cp-54},   // 2^(58/64)
    {0x1.e502ee78b3ff6p+0, 0x1.39e8980a9cc8fp-55},   // 2^(59/64)
    {0x1.ea4afa2a490dap+0, -0x1.e9c23179c2893p-54},   // 2^(60/64)
    {0x1.efa1bee615a27p+0, 0x1.dc7f486a4b6b0p-54},   // 2^(61/64)
    {0x1.f50765b6e4540p+0, 0x1.9d3e12dd8a18bp-54},   // 2^(62/64)
    {0x1.fa7c1819e90d8p+0, 0x1.74853f3a5931ep-55},   // 2^(63/64)
};

// Quick phase of exp_cr (Ziv's two-phase strategy, Tang's table-driven
// method): x = (64 m + j) ln2/64 + r with |r| <= ln2/128 (ln2/64 split as
// C1 + C2, C1 with 32 significant bits so that k C1 is exact for |k| < 2^21
// and x - k C1 is exact by Sterbenz's lemma; the neglected remainder of the
// split contributes below 2^-74), exp(x) = 2^m 2^(j/64) exp(r), exp(r) - 1
// by its Taylor polynomial to degree 6 (truncation below 2^-65) around the
// double-double r.  The pair y = 2^(j/64)(1 + p) is within 2^-64 relative of
// exp(x); RN(exp x) = y.hi is returned only when y (1 +- 2^-60) lies inside
// the rounding interval of y.hi, otherwise false (about 1.5 % of arguments)
// and the double-double phase decides.  Both phases return the correctly
// rounded value, so the result does not depend on which one answered.  A
// double-double argument x.hi + x.lo enters the reduced argument whole;
// extra_rel widens the certification interval by the argument's own error.
__device__ __forceinline__ bool exp_quick_dd(ddv x, double extra_rel, double *out) {
    if (!(x.hi > -700.0 && x.hi < 700.0)) return false;   // also NaN
    const double INV = 0x1.71547652b82fep+6;   // 64/ln2
    const double C1 = 0x1.62e42fee00000p-7;
    const double C2 = 0x1.a39ef35793c76p-39;
    const double kd = rint(__dmul_rn(x.hi, INV));
    const double s = __fma_rn(-kd, C1, x.hi);              // exact
    const double p2 = __dmul_rn(kd, C2);
    const double e2 = __fma_rn(kd, C2, -p2);               // k C2 = p2 + e2
    ddv r = dd_two_sum(s, -p2);
    r.lo = __dadd_rn(__dsub_rn(r.lo, e2), x.lo);
    r = dd_fast_two_sum(r.hi, r.lo);
    const double rh = r.hi;
    double q = __fma_rn(rh, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7);   // 1/720, 1/120
    q = __fma_rn(q, rh, 0x1.5555555555555p-5);             // 1/24
    q = __fma_rn(q, rh, 0x1.5555555555555p-3);             // 1/6
    q = __fma_rn(q, rh, 0.5);
    q = __dmul_rn(__dmul_rn(rh, rh), q);                   // r^2/2 + ... + r^6/720
    const ddv p = dd_fast_two_sum(rh, __dadd_rn(r.lo, __fma_rn(rh, r.lo, q)));   // expm1(r)
    const int k = (int)kd, j = k & 63, m = k >> 6;
    const double th = EXP2_J64[j][0], tl = EXP2_J64[j][1];
    const double a = __dmul_rn(th, p.hi);
    const double ae = __fma_rn(th, p.hi, -a);              // th p.hi = a + ae
    ddv y = dd_two_sum(th, a);
    y.lo = __dadd_rn(y.lo, __dadd_rn(ae, __fma_rn(th, p.lo, __fma_rn(tl, p.hi, tl))));
    y = dd_fast_two_sum(y.hi, y.lo);
    // certify: distance of y.lo to the half-ulp midpoints around y.hi (> 0)
    const double up = __dsub_rn(__longlong_as_double(__double_as_longlong(y.hi) + 1), y.hi);
    const double dn = __dsub_rn(y.hi, __longlong_as_double(__double_as_longlong(y.hi) - 1));
    const double dist = y.lo >= 0.0 ? __dsub_rn(__dmul_rn(up, 0.5), y.lo)
                                    : __dadd_rn(__dmul_rn(dn, 0.5), y.lo);
    if (!(dist > __dmul_rn(y.hi, __dadd_rn(0x1p-60, extra_rel)))) return false;
    *out = __dmul_rn(y.hi, __longlong_as_double((long long)(m + 1023) << 52));   // exact
    return true;
}

__device__ __forceinline__ bool exp_quick(double x, double *out) {
    return exp_quick_dd(ddv{x, 0.0}, 0.0, out);
}

// exp(x) correctly rounded (see header comment): the quick phase, else the
// double-double evaluation.
__device__ inline double exp_cr(double x, unsigned long long *ambiguous) {
    double v;
    if (exp_quick(x, &v)) return v;
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
// 1/(2j+1), j = 0..20, as double-double pairs (hi = RN(1/d), lo =
// RN((1 - hi d)/d)); gen_exp_table.py
__device__ const double ATANH_INV[21][2] = {
    {0x1.0000000000000p+0, 0x0.0p+0},   // 1/1
    {0x1.5555555555555p-2, 0x1.5555555555555p-56},   // 1/3
    {0x1.999999999999ap-3, -0x1.999999999999ap-57},   // 1/5
    {0x1.2492492492492p-3, 0x1.2492492492492p-57},   // 1/7
    {0x1.c71c71c71c71cp-4, 0x1.c71c71c71c71cp-58},   // 1/9
    {0x1.745d1745d1746p-4, -0x1.745d1745d1746p-59},   // 1/11
    {0x1.3b13b13b13b14p-4, -0x1.3b13b13b13b14p-58},   // 1/13
    {0x1.1111111111111p-4, 0x1.1111111111111p-60},   // 1/15
    {0x1.e1e1e1e1e1e1ep-5, 0x1.e1e1e1e1e1e1ep-61},   // 1/17
    {0x1.af286bca1af28p-5, 0x1.af286bca1af28p-59},   // 1/19
    {0x1.8618618618618p-5, 0x1.8618618618618p-59},   // 1/21
    {0x1.642c8590b2164p-5, 0x1.642c8590b2164p-60},   // 1/23
    {0x1.47ae147ae147bp-5, -0x1.eb851eb851eb8p-61},   // 1/25
    {0x1.2f684bda12f68p-5, 0x1.2f684bda12f68p-59},   // 1/27
    {0x1.1a7b9611a7b96p-5, 0x1.1a7b9611a7b96p-61},   // 1/29
    {0x1.0842108421084p-5, 0x1.0842108421084p-60},   // 1/31
    {0x1.f07c1f07c1f08p-6, -0x1.f07c1f07c1f08p-61},   // 1/33
    {0x1.d41d41d41d41dp-6, 0x1.0750750750750p-60},   // 1/35
    {0x1.bacf914c1bad0p-6, -0x1.bacf914c1bad0p-60},   // 1/37
    {0x1.a41a41a41a41ap-6, 0x1.0690690690690p-60},   // 1/39
    {0x1.8f9c18f9c18fap-6, -0x1.f3831f3831f38p-61},   // 1/41
};

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
    ddv t = ddv{ATANH_INV[20][0], ATANH_INV[20][1]};
#pragma unroll
    for (int j = 19; j >= 0; --j) t = dd_add(ddv{ATANH_INV[j][0], ATANH_INV[j][1]}, dd_mul(s2, t));
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

// 1/F and ln F, F = 1 + j/128, j = 0..128, as double-double pairs
// (gen_exp_table.py)
__device__ const double LOG_F128[129][4] = {
    {0x1.0000000000000p+0, 0x0.0p+0, 0x0.0p+0, 0x0.0p+0},   // F = 1 + 0/128
    {0x1.fc07f01fc07f0p-1, 0x1.fc07f01fc07f0p-57, 0x1.fe02a6b106789p-8, -0x1.e44b7e3711ebfp-67},   // F = 1 + 1/128
    {0x1.f81f81f81f820p-1, -0x1.f81f81f81f820p-55, 0x1.fc0a8b0fc03e4p-7, -0x1.83092c59642a1p-62},   // F = 1 + 2/128
    {0x1.f44659e4a4271p-1, 0x1.5fc17734c36b8p-55, 0x1.7b91b07d5b11bp-6, -0x1.5b602ace3a510p-60},   // F = 1 + 3/128
    {0x1.f07c1f07c1f08p-1, -0x1.f07c1f07c1f08p-56, 0x1.f829b0e783300p-6, 0x1.33e3f04f1ef23p-60},   // F = 1 + 4/128
    {0x1.ecc07b301ecc0p-1, 0x1.ecc07b301ecc0p-55, 0x1.39e87b9febd60p-5, -0x1.5bfa937f551bbp-59},   // F = 1 + 5/128
    {0x1.e9131abf0b767p-1, 0x1.503d226357e17p-56, 0x1.77458f632dcfcp-5, 0x1.18d3ca87b9296p-59},   // F = 1 + 6/128
    {0x1.e573ac901e574p-1, -0x1.4dbf86a314dc0p-55, 0x1.b42dd711971bfp-5, -0x1.eb9759c130499p-60},   // F = 1 + 7/128
    {0x1.e1e1e1e1e1e1ep-1, 0x1.e1e1e1e1e1e1ep-57, 0x1.f0a30c01162a6p-5, 0x1.85f325c5bbacdp-59},   // F = 1 + 8/128
    {0x1.de5d6e3f8868ap-1, 0x1.1c077975b8fe2p-55, 0x1.16536eea37ae1p-4, -0x1.79da3e8c22cdap-60},   // F = 1 + 9/128
    {0x1.dae6076b981dbp-1, -0x1.9f89467e251a0p-57, 0x1.341d7961bd1d1p-4, -0x1.b599f227becbbp-58},   // F = 1 + 10/128
    {0x1.d77b654b82c34p-1, -0x1.ba03aef6ca970p-55, 0x1.51b073f06183fp-4, 0x1.a49e39a1a8be4p-58},   // F = 1 + 11/128
    {0x1.d41d41d41d41dp-1, 0x1.0750750750750p-55, 0x1.6f0d28ae56b4cp-4, -0x1.906d99184b992p-58},   // F = 1 + 12/128
    {0x1.d0cb58f6ec074p-1, 0x1.96b1edd80e866p-56, 0x1.8c345d6319b21p-4, -0x1.4a697ab3424a9p-61},   // F = 1 + 13/128
    {0x1.cd85689039b0bp-1, -0x1.76fc64f52edf9p-56, 0x1.a926d3a4ad563p-4, 0x1.942f48aa70ea9p-58},   // F = 1 + 14/128
    {0x1.ca4b3055ee191p-1, 0x1.ca4b3055ee191p-61, 0x1.c5e548f5bc743p-4, 0x1.5d617ef8161b1p-60},   // F = 1 + 15/128
    {0x1.c71c71c71c71cp-1, 0x1.c71c71c71c71cp-55, 0x1.e27076e2af2e6p-4, -0x1.61578001e0162p-60},   // F = 1 + 16/128
    {0x1.c3f8f01c3f8f0p-1, 0x1.c3f8f01c3f8f0p-57, 0x1.fec9131dbeabbp-4, -0x1.5746b9981b36cp-58},   // F = 1 + 17/128
    {0x1.c0e070381c0e0p-1, 0x1.c0e070381c0e0p-55, 0x1.0d77e7cd08e59p-3, 0x1.9a5dc5e9030acp-57},   // F = 1 + 18/128
    {0x1.bdd2b899406f7p-1, 0x1.2b899406f74aep-55, 0x1.1b72ad52f67a0p-3, 0x1.483023472cd74p-58},   // F = 1 + 19/128
    {0x1.bacf914c1bad0p-1, -0x1.bacf914c1bad0p-55, 0x1.29552f81ff523p-3, 0x1.301771c407dbfp-57},   // F = 1 + 20/128
    {0x1.b7d6c3dda338bp-1, 0x1.579fc90527845p-56, 0x1.371fc201e8f74p-3, 0x1.de6cb62af18a0p-58},   // F = 1 + 21/128
    {0x1.b4e81b4e81b4fp-1, -0x1.f92c5f92c5f93p-55, 0x1.44d2b6ccb7d1ep-3, 0x1.9f4f6543e1f88p-57},   // F = 1 + 22/128
    {0x1.b2036406c80d9p-1, 0x1.b2036406c80d9p-61, 0x1.526e5e3a1b438p-3, -0x1.746ff8a470d3ap-57},   // F = 1 + 23/128
    {0x1.af286bca1af28p-1, 0x1.af286bca1af28p-55, 0x1.5ff3070a793d4p-3, -0x1.bc60efafc6f6ep-58},   // F = 1 + 24/128
    {0x1.ac5701ac5701bp-1, -0x1.d47f29d47f29dp-56, 0x1.6d60fe719d21dp-3, -0x1.caae268ecd179p-57},   // F = 1 + 25/128
    {0x1.a98ef606a63bep-1, -0x1.f959c427e5671p-55, 0x1.7ab890210d909p-3, 0x1.be36b2d6a0608p-59},   // F = 1 + 26/128
    {0x1.a6d01a6d01a6dp-1, 0x1.a6d01a6d01a6dp-61, 0x1.87fa06520c911p-3, -0x1.bf7fdbfa08d9ap-57},   // F = 1 + 27/128
    {0x1.a41a41a41a41ap-1, 0x1.0690690690690p-55, 0x1.9525a9cf456b4p-3, 0x1.d904c1d4e2e26p-57},   // F = 1 + 28/128
    {0x1.a16d3f97a4b02p-1, -0x1.7a4b01a16d3f9p-55, 0x1.a23bc1fe2b563p-3, 0x1.93711b07a998cp-59},   // F = 1 + 29/128
    {0x1.9ec8e951033d9p-1, 0x1.d2a2067b23a54p-57, 0x1.af3c94e80bff3p-3, -0x1.398cff3641985p-58},   // F = 1 + 30/128
    {0x1.9c2d14ee4a102p-1, -0x1.8f4bac46d7bfap-55, 0x1.bc286742d8cd6p-3, 0x1.4fce744870f55p-58},   // F = 1 + 31/128
    {0x1.999999999999ap-1, -0x1.999999999999ap-55, 0x1.c8ff7c79a9a22p-3, -0x1.4f689f8434012p-57},   // F = 1 + 32/128
    {0x1.970e4f80cb872p-1, 0x1.f01970e4f80ccp-55, 0x1.d5c216b4fbb91p-3, 0x1.6e443597e4d40p-57},   // F = 1 + 33/128
    {0x1.948b0fcd6e9e0p-1, 0x1.948b0fcd6e9e0p-55, 0x1.e27076e2af2e6p-3, -0x1.61578001e0162p-59},   // F = 1 + 34/128
    {0x1.920fb49d0e229p-1, -0x1.533d406483ed2p-56, 0x1.ef0adcbdc5936p-3, 0x1.48637950dc20dp-57},   // F = 1 + 35/128
    {0x1.8f9c18f9c18fap-1, -0x1.f3831f3831f38p-56, 0x1.fb9186d5e3e2bp-3, -0x1.caaae64f21acbp-57},   // F = 1 + 36/128
    {0x1.8d3018d3018d3p-1, 0x1.8d3018d3018d3p-61, 0x1.0402594b4d041p-2, -0x1.28ec217a5022dp-57},   // F = 1 + 37/128
    {0x1.8acb90f6bf3aap-1, -0x1.721ed7e75346fp-55, 0x1.0a324e27390e3p-2, 0x1.7dcfde8061c03p-56},   // F = 1 + 38/128
    {0x1.886e5f0abb04ap-1, -0x1.ad38b7f3bc8d0p-55, 0x1.1058bf9ae4ad5p-2, 0x1.89fa0ab4cb31dp-58},   // F = 1 + 39/128
    {0x1.8618618618618p-1, 0x1.8618618618618p-55, 0x1.1675cababa60ep-2, 0x1.ce63eab883717p-61},   // F = 1 + 40/128
    {0x1.83c977ab2beddp-1, 0x1.4731fcf86d10bp-56, 0x1.1c898c16999fbp-2, -0x1.0e5c62aff1c44p-60},   // F = 1 + 41/128
    {0x1.8181818181818p-1, 0x1.8181818181818p-57, 0x1.22941fbcf7966p-2, -0x1.76f5eb09628afp-56},   // F = 1 + 42/128
    {0x1.7f405fd017f40p-1, 0x1.7f405fd017f40p-55, 0x1.2895a13de86a3p-2, 0x1.7ad24c13f040ep-56},   // F = 1 + 43/128
    {0x1.7d05f417d05f4p-1, 0x1.7d05f417d05f4p-57, 0x1.2e8e2bae11d31p-2, -0x1.8f4cdb95ebdf9p-56},   // F = 1 + 44/128
    {0x1.7ad2208e0ecc3p-1, 0x1.516324fe852dep-55, 0x1.347dd9a987d55p-2, -0x1.4dd4c580919f8p-57},   // F = 1 + 45/128
    {0x1.78a4c8178a4c8p-1, 0x1.78a4c8178a4c8p-57, 0x1.3a64c556945eap-2, -0x1.c68651945f97cp-57},   // F = 1 + 46/128
    {0x1.767dce434a9b1p-1, 0x1.767dce434a9b1p-61, 0x1.404308686a7e4p-2, -0x1.0bcfb6082ce6dp-56},   // F = 1 + 47/128
    {0x1.745d1745d1746p-1, -0x1.745d1745d1746p-56, 0x1.4618bc21c5ec2p-2, 0x1.f42decdeccf1dp-56},   // F = 1 + 48/128
    {0x1.724287f46debcp-1, 0x1.724287f46debcp-59, 0x1.4be5f957778a1p-2, -0x1.259b35b04813dp-57},   // F = 1 + 49/128
    {0x1.702e05c0b8170p-1, 0x1.702e05c0b8170p-56, 0x1.51aad872df82dp-2, 0x1.3927ac19f55e3p-59},   // F = 1 + 50/128
    {0x1.6e1f76b4337c7p-1, -0x1.a75461405b87ep-56, 0x1.5767717455a6cp-2, 0x1.526adb283660cp-56},   // F = 1 + 51/128
    {0x1.6c16c16c16c17p-1, -0x1.f49f49f49f49fp-56, 0x1.5d1bdbf5809cap-2, 0x1.4236383dc7fe1p-56},   // F = 1 + 52/128
    {0x1.6a13cd1537290p-1, 0x1.0f8ed9cfe95ecp-55, 0x1.62c82f2b9c795p-2, 0x1.7b7af915300e5p-57},   // F = 1 + 53/128
    {0x1.6816816816817p-1, -0x1.fa5fa5fa5fa60p-55, 0x1.686c81e9b14afp-2, -0x1.ddea0f7f58e3dp-57},   // F = 1 + 54/128
    {0x1.661ec6a5122f9p-1, 0x1.661ec6a5122f9p-61, 0x1.6e08eaa2ba1e4p-2, -0x1.cfb1b39ca3a0fp-56},   // F = 1 + 55/128
    {0x1.642c8590b2164p-1, 0x1.642c8590b2164p-56, 0x1.739d7f6bbd007p-2, -0x1.8c76ceb014b04p-56},   // F = 1 + 56/128
    {0x1.623fa77016240p-1, -0x1.623fa77016240p-55, 0x1.792a55fdd47a2p-2, 0x1.f057691fe9ed7p-56},   // F = 1 + 57/128
    {0x1.6058160581606p-1, -0x1.fa7e9fa7e9fa8p-55, 0x1.7eaf83b82afc3p-2, 0x1.92ce979ed2950p-56},   // F = 1 + 58/128
    {0x1.5e75bb8d015e7p-1, 0x1.6ee340579d6eep-55, 0x1.842d1da1e8b17p-2, 0x1.24ec519784676p-56},   // F = 1 + 59/128
    {0x1.5c9882b931057p-1, 0x1.310572620ae4cp-56, 0x1.89a3386c1425bp-2, -0x1.29639dfbbf0fbp-56},   // F = 1 + 60/128
    {0x1.5ac056b015ac0p-1, 0x1.5ac056b015ac0p-55, 0x1.8f11e873662c7p-2, 0x1.f85da755a61a3p-56},   // F = 1 + 61/128
    {0x1.58ed2308158edp-1, 0x1.1840ac7691841p-56, 0x1.947941c2116fbp-2, -0x1.16cc8bae0bbe4p-56},   // F = 1 + 62/128
    {0x1.571ed3c506b3ap-1, -0x1.7749b79f7f547p-55, 0x1.99d958117e08bp-2, -0x1.a2b6889dc3e72p-57},   // F = 1 + 63/128
    {0x1.5555555555555p-1, 0x1.5555555555555p-55, 0x1.9f323ecbf984cp-2, -0x1.a92e513217f5cp-59},   // F = 1 + 64/128
    {0x1.5390948f40febp-1, -0x1.c84a47a07f563p-56, 0x1.a484090e5bb0ap-2, 0x1.5fe535b875a75p-57},   // F = 1 + 65/128
    {0x1.51d07eae2f815p-1, 0x1.d07eae2f8151dp-57, 0x1.a9cec9a9a084ap-2, -0x1.cadec02b436afp-56},   // F = 1 + 66/128
    {0x1.5015015015015p-1, 0x1.5015015015015p-61, 0x1.af1293247786bp-2, 0x1.133844a15dc28p-58},   // F = 1 + 67/128
    {0x1.4e5e0a72f0539p-1, 0x1.e0a72f0539783p-55, 0x1.b44f77bcc8f63p-2, -0x1.cd04495459c78p-56},   // F = 1 + 68/128
    {0x1.4cab88725af6ep-1, 0x1.d3d137e0cfeb3p-55, 0x1.b9858969310fbp-2, 0x1.663ec53e23bc4p-56},   // F = 1 + 69/128
    {0x1.4afd6a052bf5bp-1, -0x1.fad40a57eb503p-55, 0x1.beb4d9da71b7cp-2, -0x1.0f3c590a887cap-59},   // F = 1 + 70/128
    {0x1.49539e3b2d067p-1, -0x1.5de8d81edfd6dp-57, 0x1.c3dd7a7cdad4dp-2, 0x1.cecf052dea69bp-56},   // F = 1 + 71/128
    {0x1.47ae147ae147bp-1, -0x1.eb851eb851eb8p-57, 0x1.c8ff7c79a9a22p-2, -0x1.4f689f8434012p-56},   // F = 1 + 72/128
    {0x1.460cbc7f5cf9ap-1, 0x1.c051832f1fd74p-57, 0x1.ce1af0b85f3ebp-2, 0x1.edf4af2ab4267p-56},   // F = 1 + 73/128
    {0x1.446f86562d9fbp-1, -0x1.1be1958b67ebcp-57, 0x1.d32fe7e00ebd5p-2, 0x1.877b232fafa37p-56},   // F = 1 + 74/128
    {0x1.42d6625d51f87p-1, -0x1.064e2febd299ep-57, 0x1.d83e7258a2f3ep-2, 0x1.41456e8bb2511p-56},   // F = 1 + 75/128
    {0x1.4141414141414p-1, 0x1.4141414141414p-57, 0x1.dd46a04c1c4a1p-2, -0x1.0467656d8b892p-56},   // F = 1 + 76/128
    {0x1.3fb013fb013fbp-1, 0x1.3fb013fb013fbp-61, 0x1.e24881a7c6c26p-2, 0x1.cbd8f45954a46p-58},   // F = 1 + 77/128
    {0x1.3e22cbce4a902p-1, 0x1.f1165e7254814p-55, 0x1.e744261d68788p-2, -0x1.c825c90c344b9p-58},   // F = 1 + 78/128
    {0x1.3c995a47babe7p-1, 0x1.1013c995a47bbp-55, 0x1.ec399d2468cc0p-2, 0x1.75cee53f35397p-58},   // F = 1 + 79/128
    {0x1.3b13b13b13b14p-1, -0x1.3b13b13b13b14p-55, 0x1.f128f5faf06edp-2, -0x1.328df13bb38c3p-56},   // F = 1 + 80/128
    {0x1.3991c2c187f63p-1, 0x1.b8f4f9e027324p-56, 0x1.f6123fa7028acp-2, 0x1.8515b0f2db341p-56},   // F = 1 + 81/128
    {0x1.3813813813814p-1, -0x1.fb1fb1fb1fb20p-55, 0x1.faf588f78f31fp-2, -0x1.328260d8abca0p-57},   // F = 1 + 82/128
    {0x1.3698df3de0748p-1, -0x1.ab1232f514a02p-55, 0x1.ffd2e0857f498p-2, 0x1.565f40d9321afp-56},   // F = 1 + 83/128
    {0x1.3521cfb2b78c1p-1, 0x1.a90e7d95bc60ap-56, 0x1.02552a5a5d0ffp-1, -0x1.cb1cb51408c00p-56},   // F = 1 + 84/128
    {0x1.33ae45b57bcb2p-1, -0x1.f3fb3146e92a1p-57, 0x1.04bdf9da926d2p-1, 0x1.97f304022c9dfp-55},   // F = 1 + 85/128
    {0x1.323e34a2b10bfp-1, 0x1.9b8396ba9de81p-55, 0x1.0723e5c1cdf40p-1, 0x1.395e58e2445bbp-55},   // F = 1 + 86/128
    {0x1.30d190130d190p-1, 0x1.30d190130d190p-57, 0x1.0986f4f573521p-1, -0x1.1b8095ac02f01p-55},   // F = 1 + 87/128
    {0x1.2f684bda12f68p-1, 0x1.2f684bda12f68p-55, 0x1.0be72e4252a83p-1, -0x1.259da11330801p-55},   // F = 1 + 88/128
    {0x1.2e025c04b8097p-1, 0x1.2e025c04b8097p-61, 0x1.0e44985d1cc8cp-1, -0x1.22a3442d2d384p-58},   // F = 1 + 89/128
    {0x1.2c9fb4d812ca0p-1, -0x1.2c9fb4d812ca0p-55, 0x1.109f39e2d4c97p-1, -0x1.0e09b27a4373ap-60},   // F = 1 + 90/128
    {0x1.2b404ad012b40p-1, 0x1.2b404ad012b40p-55, 0x1.12f719593efbcp-1, 0x1.4c048c671f435p-55},   // F = 1 + 91/128
    {0x1.29e4129e4129ep-1, 0x1.04a7904a7904ap-55, 0x1.154c3d2f4d5eap-1, -0x1.59c33171a6876p-55},   // F = 1 + 92/128
    {0x1.288b01288b013p-1, -0x1.dd3fb5dd3fb5ep-55, 0x1.179eabbd899a1p-1, -0x1.00e7c6417e0b4p-55},   // F = 1 + 93/128
    {0x1.27350b8812735p-1, 0x1.71024e6a17102p-58, 0x1.19ee6b467c96fp-1, -0x1.9d1a11443f10cp-56},   // F = 1 + 94/128
    {0x1.25e22708092f1p-1, 0x1.3840497889c20p-57, 0x1.1c3b81f713c25p-1, -0x1.0dac1c4c810e9p-55},   // F = 1 + 95/128
    {0x1.2492492492492p-1, 0x1.2492492492492p-55, 0x1.1e85f5e7040d0p-1, 0x1.ef62cd2f9f1e3p-56},   // F = 1 + 96/128
    {0x1.23456789abcdfp-1, 0x1.23456789abcdfp-61, 0x1.20cdcd192ab6ep-1, -0x1.b2bf0bc229014p-55},   // F = 1 + 97/128
    {0x1.21fb78121fb78p-1, 0x1.21fb78121fb78p-57, 0x1.23130d7bebf43p-1, -0x1.f48725e374d6ep-55},   // F = 1 + 98/128
    {0x1.20b470c67c0d9p-1, -0x1.e2adac8bd766ap-55, 0x1.2555bce98f7cbp-1, 0x1.e021d6d6881e7p-56},   // F = 1 + 99/128
    {0x1.1f7047dc11f70p-1, 0x1.1f7047dc11f70p-55, 0x1.2795e1289b11bp-1, -0x1.487c0c246978ep-57},   // F = 1 + 100/128
    {0x1.1e2ef3b3fb874p-1, 0x1.0c4c0478bbcedp-55, 0x1.29d37fec2b08bp-1, -0x1.bd1949a2d1982p-56},   // F = 1 + 101/128
    {0x1.1cf06ada2811dp-1, -0x1.f2a4bafdc61f3p-58, 0x1.2c0e9ed448e8cp-1, -0x1.1a158f3917586p-55},   // F = 1 + 102/128
    {0x1.1bb4a4046ed29p-1, 0x1.1bb4a4046ed29p-61, 0x1.2e47436e40268p-1, 0x1.0150861a4886bp-55},   // F = 1 + 103/128
    {0x1.1a7b9611a7b96p-1, 0x1.1a7b9611a7b96p-57, 0x1.307d7334f10bep-1, 0x1.fb590a1f566dap-57},   // F = 1 + 104/128
    {0x1.19453808ca29cp-1, 0x1.19453808ca29cp-59, 0x1.32b1339121d71p-1, 0x1.902ab5b3d916bp-56},   // F = 1 + 105/128
    {0x1.1811811811812p-1, -0x1.fb9fb9fb9fba0p-55, 0x1.34e289d9ce1d3p-1, 0x1.6eb92d885ce4fp-57},   // F = 1 + 106/128
    {0x1.16e0689427379p-1, -0x1.4b2a7c2fee920p-57, 0x1.37117b54747b6p-1, -0x1.d117edbdd9103p-56},   // F = 1 + 107/128
    {0x1.15b1e5f75270dp-1, 0x1.15b1e5f75270dp-59, 0x1.393e0d3562a1ap-1, -0x1.58eef67f2483ap-55},   // F = 1 + 108/128
    {0x1.1485f0e0acd3bp-1, 0x1.a31b011485f0ep-55, 0x1.3b68449fffc23p-1, -0x1.41c484f9e9b26p-55},   // F = 1 + 109/128
    {0x1.135c81135c811p-1, 0x1.ae4089ae4089bp-56, 0x1.3d9026a7156fbp-1, -0x1.6fef670bd4b62p-55},   // F = 1 + 110/128
    {0x1.12358e75d3033p-1, 0x1.a82ad85e42690p-55, 0x1.3fb5b84d16f42p-1, 0x1.6d3a754172aefp-55},   // F = 1 + 111/128
    {0x1.1111111111111p-1, 0x1.1111111111111p-57, 0x1.41d8fe84672aep-1, 0x1.9192f30bd1806p-55},   // F = 1 + 112/128
    {0x1.0fef010fef011p-1, -0x1.0fef010fef011p-61, 0x1.43f9fe2f9ce67p-1, 0x1.e9c9ee6d83b86p-55},   // F = 1 + 113/128
    {0x1.0ecf56be69c90p-1, -0x1.0ecf56be69c90p-56, 0x1.4618bc21c5ec2p-1, 0x1.f42decdeccf1dp-55},   // F = 1 + 114/128
    {0x1.0db20a88f4696p-1, -0x1.9cf8a021b6415p-55, 0x1.48353d1ea88dfp-1, 0x1.cf57a2ecc07f4p-55},   // F = 1 + 115/128
    {0x1.0c9714fbcda3bp-1, -0x1.f79b47582192ep-56, 0x1.4a4f85db03ebbp-1, 0x1.13dfa3d3761b6p-60},   // F = 1 + 116/128
    {0x1.0b7e6ec259dc8p-1, -0x1.b2ad73fbd2064p-55, 0x1.4c679afccee3ap-1, -0x1.3a5c4c8b39e41p-55},   // F = 1 + 117/128
    {0x1.0a6810a6810a7p-1, -0x1.fbd65fbd65fbdp-55, 0x1.4e7d811b75bb1p-1, -0x1.8d3d9ea6e9ea9p-55},   // F = 1 + 118/128
    {0x1.0953f39010954p-1, -0x1.8dfded5818dfep-58, 0x1.50913cc01686bp-1, 0x1.2f2ce96c2d5b1p-55},   // F = 1 + 119/128
    {0x1.0842108421084p-1, 0x1.0842108421084p-56, 0x1.52a2d265bc5abp-1, -0x1.1883750ea4d0ap-57},   // F = 1 + 120/128
    {0x1.073260a47f7c6p-1, 0x1.b3eb701073261p-55, 0x1.54b2467999498p-1, -0x1.5baaf5d2f09f4p-55},   // F = 1 + 121/128
    {0x1.0624dd2f1a9fcp-1, -0x1.89374bc6a7efap-57, 0x1.56bf9d5b3f399p-1, 0x1.0471885cd8ff3p-55},   // F = 1 + 122/128
    {0x1.05197f7d73404p-1, 0x1.465fdf5cd0105p-57, 0x1.58cadb5cd7989p-1, 0x1.849792ec98458p-56},   // F = 1 + 123/128
    {0x1.0410410410410p-1, 0x1.0410410410410p-55, 0x1.5ad404c359f2dp-1, -0x1.35955683f7196p-59},   // F = 1 + 124/128
    {0x1.03091b51f5e1ap-1, 0x1.3bb3194be3ab0p-55, 0x1.5cdb1dc6c1765p-1, -0x1.cc2470e8a3df4p-55},   // F = 1 + 125/128
    {0x1.0204081020408p-1, 0x1.0204081020408p-57, 0x1.5ee02a9241675p-1, 0x1.c358257f49082p-55},   // F = 1 + 126/128
    {0x1.0101010101010p-1, 0x1.0101010101010p-57, 0x1.60e32f44788d9p-1, -0x1.ac1bb52fa589bp-56},   // F = 1 + 127/128
    {0x1.0000000000000p-1, 0x0.0p+0, 0x1.62e42fefa39efp-1, 0x1.abc9e3b39803fp-56},   // F = 1 + 128/128
};

// Quick phase of pow_cr: ln r = k ln2 + ln F + ln(1 + f) for r = 2^k m,
// m in [1, 2), F = 1 + j/128 nearest to m (Tang's table-driven logarithm,
// ACM TOMS 16(4), 1990): d = m - F is exact (|d| <= 2^-8), f = d/F is formed
// in double-double from the tabulated 1/F, and ln(1 + f) = f + Q(f) with
// Q(f) = sum_{k=2..8} (-1)^(k+1) f^k/k evaluated by Horner on f.hi.
// Absolute error of the pair (ln(1 + f), the bound the certification uses):
//   * truncation after degree 8: |f|^9/9 <= 2^-75.2;
//   * f itself (fma rounding of d il + fe, table 1/F to 2^-106): 2^-113;
//   * Q on f.hi instead of f: the first-order term -f.hi f.lo is added
//     explicitly; what remains is f^2 |f.lo| <= 2^-16 2^-62 = 2^-78;
//   * Q's roundings: |Q| <= f^2/2 <= 2^-17; the Horner value q ~ -1/2 is
//     off by at most 2^-54 (its last fma; earlier steps enter times
//     |f| <= 2^-8), i.e. 2^-53 relative, f.hi^2 and the product add 2^-53
//     relative each: 3 2^-53 2^-17 = 3 2^-70;
//   * the two roundings of the low-part sums (values below 2^-17): 2 2^-70;
//   * k ln2 (split ln2 with exact k L1, k L2; k L3 rounded: 2^-107) and
//     ln F (tabulated double-double, 2^-107), the double-double additions
//     (relative 2^-104 of |l| <= 745): below 2^-94.
// Total below 5 2^-70 = 2^-67.68 (2^-68.9 is the largest seen over 40,000
// arguments against a 250-bit evaluation).  An absolute error of the
// exponent e ln r is a relative error of r^e, so the exp quick phase takes
// e 2^-67 (> e 2^-67.68) as extra certification width.
__device__ __forceinline__ bool pow_quick(double r, double e, double *out) {
    if (!(r >= 0x1p-1022 && r < 0x1p1023 && e > 0.0 && e < 0x1p20)) return false;
    const long long bits = __double_as_longlong(r);
    const int k = (int)((bits >> 52) & 0x7ff) - 1023;
    const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const int j = (int)rint(__dmul_rn(__dsub_rn(m, 1.0), 128.0));
    const double d = __dsub_rn(m, __dadd_rn(1.0, __dmul_rn((double)j, 0x1p-7)));   // exact
    const double ih = LOG_F128[j][0], il = LOG_F128[j][1];
    const double fh = __dmul_rn(d, ih);
    const double fe = __fma_rn(d, ih, -fh);                // d ih = fh + fe
    const ddv f = dd_fast_two_sum(fh, __fma_rn(d, il, fe));
    // -f^2/2 + f^3/3 - ... - f^8/8 on f.hi, plus the cross term -f.hi f.lo
    double q = __fma_rn(f.hi, -0.125, 0x1.2492492492492p-3);   // -1/8, 1/7
    q = __fma_rn(q, f.hi, -0x1.5555555555555p-3);            // -1/6
    q = __fma_rn(q, f.hi, 0x1.999999999999ap-3);             // 1/5
    q = __fma_rn(q, f.hi, -0.25);
    q = __fma_rn(q, f.hi, 0x1.5555555555555p-2);             // 1/3
    q = __fma_rn(q, f.hi, -0.5);
    q = __dmul_rn(__dmul_rn(f.hi, f.hi), q);
    const ddv p = dd_fast_two_sum(f.hi, __dadd_rn(f.lo, __fma_rn(-f.hi, f.lo, q)));   // ln(1 + f)
    const double L1 = 0x1.62e42fee00000p-1;
    const double L2 = 0x1.a39ef35600000p-33;
    const double L3 = 0x1.93c7673007e5fp-65;
    const double kd = (double)k;
    ddv l = dd_two_sum(__dmul_rn(kd, L1), __dmul_rn(kd, L2));   // both products exact
    l.lo = __dadd_rn(l.lo, __dmul_rn(kd, L3));
    l = dd_add(dd_add(l, ddv{LOG_F128[j][2], LOG_F128[j][3]}), p);
    const ddv y = dd_mul(l, ddv{e, 0.0});
    return exp_quick_dd(y, __dmul_rn(e, 0x1p-67), out);
}

// r^e correctly rounded for a positive finite double r and e > 0 (the
// pseudopotential psi_eps = (n/(eps+n))^(1/eps), eq. psieps): exp of the
// double-double e ln r.  The argument carries an absolute error of about
// |e ln r| 2^-100, widened into the certification interval.
__device__ inline double pow_cr(double r, double e, unsigned long long *ambiguous) {
    if (r == 1.0) return 1.0;
    double v;
    if (pow_quick(r, e, &v)) return v;
    const ddv l = log_dd(r);
    const ddv y = dd_mul(l, ddv{e, 0.0});
    const double ay = fabs(y.hi);
    const double tol = 0x1p-97 + __dmul_rn(ay, 0x1p-98);
    return exp_dd_cr(y, tol, ambiguous);
}

}  // namespace sclbm
