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
// double-double evaluation above.  Both return the correctly rounded value.
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
// rounded value, so the result does not depend on which one answered.
__device__ __forceinline__ bool exp_quick(double x, double *out) {
    if (!(x > -700.0 && x < 700.0)) return false;   // also NaN
    const double INV = 0x1.71547652b82fep+6;   // 64/ln2
    const double C1 = 0x1.62e42fee00000p-7;
    const double C2 = 0x1.a39ef35793c76p-39;
    const double kd = rint(__dmul_rn(x, INV));
    const double s = __fma_rn(-kd, C1, x);                 // exact
    const double p2 = __dmul_rn(kd, C2);
    const double e2 = __fma_rn(kd, C2, -p2);               // k C2 = p2 + e2
    ddv r = dd_two_sum(s, -p2);
    r.lo = __dsub_rn(r.lo, e2);
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
    if (!(dist > __dmul_rn(y.hi, 0x1p-60))) return false;
    *out = __dmul_rn(y.hi, __longlong_as_double((long long)(m + 1023) << 52));   // exact
    return true;
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
