// fusedcommon.cuh -- pieces shared by the fused single-pass D3Q19 kernels
// (fused3d.cu: cp.async staging, any lattice size; fused3d_tma.cu: TMA
// staging on the ghost-padded layout).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace sclbm {
namespace fc {

constexpr int TX = 32, TY = 8;

// canonical (e,-e) pairs of the seven E8 groups (1,0,0), (1,1,0), (1,1,1),
// (2,0,0), (2,1,0), (2,1,1), (2,2,0): e_x, e_y, e_z, group (the order of
// lb_expand_stencil; checked against it at context set-up)
__host__ __device__ constexpr int pair_c(int a, int k) {
    constexpr signed char t[46][4] = {
        {1, 0, 0, 0},   {0, 1, 0, 0},   {0, 0, 1, 0},   {1, 1, 0, 1},   {1, 0, 1, 1},
        {1, 0, -1, 1},  {1, -1, 0, 1},  {0, 1, 1, 1},   {0, 1, -1, 1},  {1, 1, 1, 2},
        {1, 1, -1, 2},  {1, -1, 1, 2},  {1, -1, -1, 2}, {2, 0, 0, 3},   {0, 2, 0, 3},
        {0, 0, 2, 3},   {2, 1, 0, 4},   {2, 0, 1, 4},   {2, 0, -1, 4},  {2, -1, 0, 4},
        {1, 2, 0, 4},   {1, 0, 2, 4},   {1, 0, -2, 4},  {1, -2, 0, 4},  {0, 2, 1, 4},
        {0, 2, -1, 4},  {0, 1, 2, 4},   {0, 1, -2, 4},  {2, 1, 1, 5},   {2, 1, -1, 5},
        {2, -1, 1, 5},  {2, -1, -1, 5}, {1, 2, 1, 5},   {1, 2, -1, 5},  {1, 1, 2, 5},
        {1, 1, -2, 5},  {1, -1, 2, 5},  {1, -1, -2, 5}, {1, -2, 1, 5},  {1, -2, -1, 5},
        {2, 2, 0, 6},   {2, 0, 2, 6},   {2, 0, -2, 6},  {2, -2, 0, 6},  {0, 2, 2, 6},
        {0, 2, -2, 6}};
    return t[a][k];
}
// one past the last pair of group g
__host__ __device__ constexpr int group_end(int g) {
    constexpr int t[7] = {3, 9, 13, 16, 28, 40, 46};
    return t[g];
}

struct Params {
    float W[7];      // group weights (0 for groups the stencil lacks)
    float W2[7];     // 2 W
    float M1, M2;    // z-offset sums of weights (plane-split force; M2 doubled)
    float omega;     // 1/tau
    float keep;      // 1 - 1/tau
    float mGp;       // -G'
    float rho0;      // population shift
    // collision constants per velocity class |xi|^2 = 0, 1, 2 (weight w,
    // cw = (1 - 1/(2 tau)) w): omega w, -3 cw, 4.5 omega w, 3 omega w, 9 cw, 3 cw
    float omw[3], m3cw[3], b45[3], d3[3], c9[3], c3[3];
    int nx, ny, nz;  // lattice
    int nxp, nyp;    // padded population plane
    int ox, oy;      // node (0,0) inside a padded plane
    int pplane;      // nxp * nyp
    int Np;          // population stride
    int zchunk;      // z planes per CTA
    float eps, inv_eps;   // psi_eps: eps and RN(1/eps) in binary32 (0 for psi = exp(-1/n))
    // F^2 variant (T = 2 u F - (A/tau) F F): -kA/2 and, per class, -4.5 cw kA
    // (kA = A/tau; all 0 for Guo's T = 2 u F)
    float mhkA, kq[3];
    long long max_polls;  // bound of every mbarrier wait of the TMA kernel
};

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// psi = exp(-1/n) in binary32: correctly rounded reciprocal, then expf
__device__ __forceinline__ float psi32(float n) { return expf(-__frcp_rn(n)); }

// the pseudopotential of a fused kernel: EPS false psi = exp(-1/n), EPS true
// psi_eps = (n/(eps + n))^(1/eps) (eq. psieps) as 2^((1/eps) log2(n/(eps + n)))
// (the base lies in (0, 1); about 2e-7 relative against the exact power);
// both are the binary32 expressions of the generic path, so psi is the same
// value on every path
template <bool EPS>
__device__ __forceinline__ float psi_fused(float n, float eps, float inv_eps) {
    if constexpr (EPS) return exp2f(inv_eps * log2f(n / (eps + n)));
    else return psi32(n);
}

__device__ __forceinline__ float dens(const float *g) {
    // pairwise tree keeps the binary32 sum short
    float a = (g[1] + g[2]) + (g[3] + g[4]);
    float b = (g[5] + g[6]) + (g[7] + g[8]);
    float c = (g[9] + g[10]) + (g[11] + g[12]);
    float d = (g[13] + g[14]) + (g[15] + g[16]);
    float e = (g[17] + g[18]) + g[0];
    return ((a + b) + (c + d)) + e;
}

// Stencil force of eq. sc_f from a ring of psi planes: pz[R + k] points at
// the node's psi in plane z + k, rows EX apart.  Accumulated per pair with
// the group weight folded into the FMA, then scaled by -G' psi(x).
template <int R, int NG, int EX>
__device__ __forceinline__ void force_ring(const float *const *pz, const Params &p, float *F) {
    F[0] = F[1] = F[2] = 0.f;
#pragma unroll
    for (int a = 0; a < group_end(NG - 1); ++a) {
        const int ex = pair_c(a, 0), ey = pair_c(a, 1), ez = pair_c(a, 2), gq = pair_c(a, 3);
        const float d = pz[R + ez][ey * EX + ex] - pz[R - ez][-ey * EX - ex];
        if (ex) F[0] = fmaf(ex == 1 ? p.W[gq] : ex == -1 ? -p.W[gq] : (float)ex * p.W[gq], d, F[0]);
        if (ey) F[1] = fmaf(ey == 1 ? p.W[gq] : ey == -1 ? -p.W[gq] : (float)ey * p.W[gq], d, F[1]);
        if (ez) F[2] = fmaf(ez == 1 ? p.W[gq] : ez == -1 ? -p.W[gq] : (float)ez * p.W[gq], d, F[2]);
    }
    const float pre = p.mGp * pz[R][0];
    F[0] *= pre;
    F[1] *= pre;
    F[2] *= pre;
}

// group index of |e|^2 = s among the seven E8 groups (-1: no group)
__host__ __device__ constexpr int group_of_sq(int s) {
    return s == 1 ? 0 : s == 2 ? 1 : s == 3 ? 2 : s == 4 ? 3 : s == 5 ? 4 : s == 6 ? 5 : s == 8 ? 6 : -1;
}

// acc += W(s) v (or 2 W(s) v) when the group of |e|^2 = s is among the first NG
template <int NG, int S, bool TWICE = false>
__device__ __forceinline__ void wfma(float &acc, const Params &p, float v) {
    constexpr int q = group_of_sq(S);
    if constexpr (q >= 0 && q < NG) acc = fmaf(TWICE ? p.W2[q] : p.W[q], v, acc);
}

// Plane-split form of the stencil force (eq. sc_f).  Grouping the vectors e
// by their z component d and in-plane ring k = e_x^2 + e_y^2, one plane of
// psi at z offset d from the target contributes
//   F_x += sum_k W(k + d^2) X_k,  F_y += sum_k W(k + d^2) Y_k,
//   F_z += d sum_k W(k + d^2) S_k,
// with X_k, Y_k, S_k the sums of e_x psi, e_y psi, psi over the ring.  One
// pass over a plane serves all 2R+1 targets it touches; the sums X_k, Y_k,
// cz of a plane depend on |d| only.  S_k is taken relative to the column's
// own psi0 (differences of nearby values are exact in binary32); the psi0
// part, sum_d d M_|d| psi0(z + d), is added at the target from its own
// column (M1, M2 are those weight sums, M2 doubled).
//   pc : this column's psi in a plane of rows EX apart; s0 = *pc
//   cx[d], cy[d] : in-plane parts for |d| = 0..R;  cz[d] : |d| (sum W S^) for d >= 1
template <int R, int NG, int EX>
__device__ __forceinline__ void plane_force(const float *pc, float s0, const Params &p, float *cx,
                                            float *cy, float *cz) {
    auto q = [&](int dx, int dy) { return pc[dy * EX + dx] - s0; };
    // ring k = 1
    const float e = q(1, 0), w = q(-1, 0), nn = q(0, 1), ss = q(0, -1);
    const float X1 = e - w, Y1 = nn - ss, S1 = (e + w) + (nn + ss);
    // ring k = 2
    const float a = q(1, 1), b = q(1, -1), c = q(-1, 1), d = q(-1, -1);
    const float ab = a + b, cd = c + d, ac = a + c, bd = b + d;
    const float X2 = ab - cd, Y2 = ac - bd, S2 = ab + cd;
#pragma unroll
    for (int k = 0; k <= R; ++k) cx[k] = cy[k] = cz[k] = 0.f;
    wfma<NG, 1>(cx[0], p, X1);
    wfma<NG, 2>(cx[0], p, X2);
    wfma<NG, 1>(cy[0], p, Y1);
    wfma<NG, 2>(cy[0], p, Y2);
    wfma<NG, 2>(cx[1], p, X1);
    wfma<NG, 3>(cx[1], p, X2);
    wfma<NG, 2>(cy[1], p, Y1);
    wfma<NG, 3>(cy[1], p, Y2);
    wfma<NG, 2>(cz[1], p, S1);
    wfma<NG, 3>(cz[1], p, S2);
    if constexpr (R >= 2) {
        // ring k = 4 (X, Y halved: e_x = +-2)
        const float e2 = q(2, 0), w2 = q(-2, 0), n2 = q(0, 2), s2 = q(0, -2);
        const float X4h = e2 - w2, Y4h = n2 - s2, S4 = (e2 + w2) + (n2 + s2);
        // ring k = 5: (+-2, +-1) and (+-1, +-2)
        const float r21 = q(2, 1), r2m = q(2, -1), rm21 = q(-2, 1), rm2m = q(-2, -1);
        const float r12 = q(1, 2), rm12 = q(-1, 2), r1m2 = q(1, -2), rm1m2 = q(-1, -2);
        const float A = r21 + r2m, B = rm21 + rm2m, C = r12 + r1m2, D = rm12 + rm1m2;
        const float E = r21 + rm21, Fv = r2m + rm2m, G = r12 + rm12, H = r1m2 + rm1m2;
        const float X5 = fmaf(2.f, A - B, C - D), Y5 = fmaf(2.f, G - H, E - Fv);
        const float S5 = (A + B) + (C + D);
        // ring k = 8 (halved), raw values
        const float k1 = pc[2 * EX + 2], k2 = pc[-2 * EX + 2], k3 = pc[2 * EX - 2], k4 = pc[-2 * EX - 2];
        const float X8h = (k1 + k2) - (k3 + k4), Y8h = (k1 + k3) - (k2 + k4);
        wfma<NG, 4, true>(cx[0], p, X4h);
        wfma<NG, 5>(cx[0], p, X5);
        wfma<NG, 8, true>(cx[0], p, X8h);
        wfma<NG, 4, true>(cy[0], p, Y4h);
        wfma<NG, 5>(cy[0], p, Y5);
        wfma<NG, 8, true>(cy[0], p, Y8h);
        wfma<NG, 5, true>(cx[1], p, X4h);
        wfma<NG, 6>(cx[1], p, X5);
        wfma<NG, 5, true>(cy[1], p, Y4h);
        wfma<NG, 6>(cy[1], p, Y5);
        wfma<NG, 5>(cz[1], p, S4);
        wfma<NG, 6>(cz[1], p, S5);
        wfma<NG, 5>(cx[2], p, X1);
        wfma<NG, 6>(cx[2], p, X2);
        wfma<NG, 8, true>(cx[2], p, X4h);
        wfma<NG, 5>(cy[2], p, Y1);
        wfma<NG, 6>(cy[2], p, Y2);
        wfma<NG, 8, true>(cy[2], p, Y4h);
        wfma<NG, 5, true>(cz[2], p, S1);
        wfma<NG, 6, true>(cz[2], p, S2);
        wfma<NG, 8, true>(cz[2], p, S4);
    }
}

// BGK + Guo of one node in shifted binary32 (eqs. f_eq, GuoForcing, omega_i).
// With u = (j + F/2)/n and base = dn - 1.5 n u.u (dn = n - rho0), a velocity
// class of weight w and forcing weight cw = (1 - 1/(2 tau)) w gives each pair
// of opposite velocities (xi, -xi)
//   even part  E = omega w (base + 4.5 n (xi.u)^2) + cw (9 (xi.u)(xi.F) - 3 u.F)
//   odd part   O = 3 omega w n (xi.u) + 3 cw (xi.F)
// and out(xi) = (1 - omega) g(xi) + E + O, out(-xi) = (1 - omega) g(-xi) + E - O.
// F2: the F^2 variant's extra source -cw kA (4.5 (xi.F)^2 - 1.5 F.F) (Sec. VI),
// its F.F part folded into u.F (u.F - (kA/2) F.F) and its (xi.F)^2 part
// added to each pair's even part.
template <bool F2 = false>
__device__ __forceinline__ void collide19(const float *g, float dn, const float *F, const Params &p,
                                          float *out) {
    const float n = dn + p.rho0;
    const float inv = __frcp_rn(n);
    const float d1 = g[1] - g[2], d3 = g[3] - g[4], d5 = g[5] - g[6];
    const float d7 = g[7] - g[8], d9 = g[9] - g[10], d11 = g[11] - g[12];
    const float d13 = g[13] - g[14], d15 = g[15] - g[16], d17 = g[17] - g[18];
    const float jx = ((d1 + d7) + (d9 + d11)) + d13;
    const float jy = ((d3 + d7) + (d15 - d9)) + d17;
    const float jz = ((d5 + d11) + (d15 - d13)) - d17;
    const float ux = fmaf(0.5f, F[0], jx) * inv;
    const float uy = fmaf(0.5f, F[1], jy) * inv;
    const float uz = fmaf(0.5f, F[2], jz) * inv;
    const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    float uF = fmaf(ux, F[0], fmaf(uy, F[1], uz * F[2]));
    if constexpr (F2) uF = fmaf(p.mhkA, fmaf(F[0], F[0], fmaf(F[1], F[1], F[2] * F[2])), uF);
    const float base = fmaf(-1.5f * n, uu, dn);
    out[0] = fmaf(p.keep, g[0], fmaf(p.omw[0], base, p.m3cw[0] * uF));
    const float a1 = fmaf(p.omw[1], base, p.m3cw[1] * uF);
    const float a2 = fmaf(p.omw[2], base, p.m3cw[2] * uF);
    const float b1 = p.b45[1] * n, b2 = p.b45[2] * n;
    const float e1 = p.d3[1] * n, e2 = p.d3[2] * n;
#define SCLBM_PAIR(I, C, CU, CF)                                                \
    {                                                                           \
        const float cu = (CU), cF = (CF);                                       \
        float aq = a##C;                                                        \
        if constexpr (F2) aq = fmaf(cF, p.kq[C] * cF, aq);                      \
        const float ev = fmaf(cu, fmaf(b##C, cu, p.c9[C] * cF), aq);            \
        const float od = fmaf(e##C, cu, p.c3[C] * cF);                          \
        out[I] = fmaf(p.keep, g[I], ev + od);                                   \
        out[I + 1] = fmaf(p.keep, g[I + 1], ev - od);                           \
    }
    SCLBM_PAIR(1, 1, ux, F[0])
    SCLBM_PAIR(3, 1, uy, F[1])
    SCLBM_PAIR(5, 1, uz, F[2])
    SCLBM_PAIR(7, 2, ux + uy, F[0] + F[1])
    SCLBM_PAIR(9, 2, ux - uy, F[0] - F[1])
    SCLBM_PAIR(11, 2, ux + uz, F[0] + F[2])
    SCLBM_PAIR(13, 2, ux - uz, F[0] - F[2])
    SCLBM_PAIR(15, 2, uy + uz, F[1] + F[2])
    SCLBM_PAIR(17, 2, uy - uz, F[1] - F[2])
#undef SCLBM_PAIR
}

// A node's j + F/2 and |u|^2 formed exactly as collide19 forms them (the
// same operations in the same order), for the fused kernel's measuring
// instantiation.
__device__ __forceinline__ void moments19(const float *g, float dn, const float *F,
                                          const Params &p, float *m, float &uu) {
    const float n = dn + p.rho0;
    const float inv = __frcp_rn(n);
    const float d1 = g[1] - g[2], d3 = g[3] - g[4], d5 = g[5] - g[6];
    const float d7 = g[7] - g[8], d9 = g[9] - g[10], d11 = g[11] - g[12];
    const float d13 = g[13] - g[14], d15 = g[15] - g[16], d17 = g[17] - g[18];
    const float jx = ((d1 + d7) + (d9 + d11)) + d13;
    const float jy = ((d3 + d7) + (d15 - d9)) + d17;
    const float jz = ((d5 + d11) + (d15 - d13)) - d17;
    m[0] = fmaf(0.5f, F[0], jx);
    m[1] = fmaf(0.5f, F[1], jy);
    m[2] = fmaf(0.5f, F[2], jz);
    const float ux = m[0] * inv, uy = m[1] * inv, uz = m[2] * inv;
    uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
}

// (s, e) += v with the rounding error kept (two_sum); s + e carries the
// running sum to about 2^-48 relative
__device__ __forceinline__ void ff_acc(float &s, float &e, float v) {
    const float t = s + v;
    const float bb = t - s;
    e += (s - (t - bb)) + (v - bb);
    s = t;
}

// Observables record of the fused kernel's measuring pass, in binary32
// pairs (value, error): v[0..1] shifted mass, v[2..7] momentum x, y, z;
// v[8] max |u|^2, v[9] min n, v[10] max n.
struct MeasRec {
    float v[11];
};

__device__ __forceinline__ MeasRec meas_zero() {
    MeasRec r;
#pragma unroll
    for (int k = 0; k < 8; ++k) r.v[k] = 0.f;
    r.v[8] = 0.f;
    r.v[9] = __int_as_float(0x7f800000);
    r.v[10] = -__int_as_float(0x7f800000);
    return r;
}

// (hi, lo) normalised from a value and its error
__device__ __forceinline__ void meas_pair(MeasRec &r, int k, float s, float e) {
    const float t = s + e;
    r.v[k] = t;
    r.v[k + 1] = e - (t - s);
}

// r += o: pairs added with their rounding errors kept (two_sum, then the
// errors and a renormalisation), extrema combined
__device__ __forceinline__ void meas_combine(MeasRec &r, const MeasRec &o) {
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const float s = r.v[k] + o.v[k];
        const float bb = s - r.v[k];
        const float err = (r.v[k] - (s - bb)) + (o.v[k] - bb);
        meas_pair(r, k, s, err + (r.v[k + 1] + o.v[k + 1]));
    }
    r.v[8] = fmaxf(r.v[8], o.v[8]);
    r.v[9] = fminf(r.v[9], o.v[9]);
    r.v[10] = fmaxf(r.v[10], o.v[10]);
}

// a warp's records combined by xor-shuffles (every lane ends with the sum)
__device__ __forceinline__ void meas_warp(MeasRec &r) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        MeasRec o;
#pragma unroll
        for (int k = 0; k < 11; ++k) o.v[k] = __shfl_xor_sync(0xffffffffu, r.v[k], off);
        meas_combine(r, o);
    }
}


// Write a node's 19 post-collision populations; on a padded layout also its
// periodic images in the ghost columns (x < 8, x >= nx-8) and rows (y < 3,
// y >= ny-3), so the next step's plane boxes read valid neighbours.
__device__ __forceinline__ void store19(float *__restrict__ B, const Params &p, int x, int y, int z,
                                        const float *out) {
    const int base = z * p.pplane + (y + p.oy) * p.nxp + (x + p.ox);
#pragma unroll
    for (int i = 0; i < 19; ++i) B[i * p.Np + base] = out[i];
    if (p.ox == 0 && p.oy == 0) return;
    const int gx = x < GHOST_X ? x + p.nx : (x >= p.nx - GHOST_X ? x - p.nx : INT_MIN);
    const int gy = y < p.oy ? y + p.ny : (y >= p.ny - p.oy ? y - p.ny : INT_MIN);
    if (gx == INT_MIN && gy == INT_MIN) return;
    const int zb = z * p.pplane;
    if (gx != INT_MIN) {
        const int o = zb + (y + p.oy) * p.nxp + (gx + p.ox);
#pragma unroll
        for (int i = 0; i < 19; ++i) B[i * p.Np + o] = out[i];
    }
    if (gy != INT_MIN) {
        const int o = zb + (gy + p.oy) * p.nxp + (x + p.ox);
#pragma unroll
        for (int i = 0; i < 19; ++i) B[i * p.Np + o] = out[i];
        if (gx != INT_MIN) {
            const int o2 = zb + (gy + p.oy) * p.nxp + (gx + p.ox);
#pragma unroll
            for (int i = 0; i < 19; ++i) B[i * p.Np + o2] = out[i];
        }
    }
}

// halo node t of a TX x TY tile extended by R, in extended coordinates
template <int R>
__device__ __forceinline__ void halo_coords(int t, int &hx, int &hy) {
    constexpr int EX = TX + 2 * R;
    const int top = R * EX;
    if (t < top) {
        hy = t / EX;
        hx = t % EX;
    } else if (t < top + TY * 2 * R) {
        const int k = t - top;
        hy = R + k / (2 * R);
        const int c = k % (2 * R);
        hx = c < R ? c : TX + c;
    } else {
        const int k = t - top - TY * 2 * R;
        hy = R + TY + k / EX;
        hx = k % EX;
    }
}

// the last block to finish a step advances the device step counter
__device__ __forceinline__ void finish_step(Flags *flags, int t) {
    __syncthreads();
    if (t == 0) {
        __threadfence();
        const unsigned long long total = (unsigned long long)gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(&flags->blocks_done, 1ULL) == total - 1) {
            flags->blocks_done = 0;
            flags->step = flags->step + 1;
        }
    }
}

}  // namespace fc
}  // namespace sclbm
