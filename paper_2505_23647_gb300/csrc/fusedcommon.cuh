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
    float omega;     // 1/tau
    float mGp;       // -G'
    float rho0;      // population shift
    float cw[3];     // (1 - 1/(2 tau)) w for |xi|^2 = 0, 1, 2
    int nx, ny, nz;  // lattice
    int nxp, nyp;    // padded population plane
    int ox, oy;      // node (0,0) inside a padded plane
    int pplane;      // nxp * nyp
    int Np;          // population stride
    int zchunk;      // z planes per CTA
};

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// psi = exp(-1/n) in binary32: correctly rounded reciprocal, then expf
__device__ __forceinline__ float psi32(float n) { return expf(-__frcp_rn(n)); }

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

// BGK + Guo of one node in shifted binary32 (eqs. f_eq, GuoForcing, omega_i):
// equilibrium and source split into parts even and odd in xi, one
// evaluation per pair of opposite velocities (i, i+1).
__device__ __forceinline__ void collide19(const float *g, const float *F, const Params &p,
                                          float *out) {
    const float dn = dens(g);
    const float n = dn + p.rho0;
    const float inv = __frcp_rn(n);
    const float jx = ((g[1] - g[2]) + (g[7] - g[8])) + ((g[9] - g[10]) + (g[11] - g[12])) + (g[13] - g[14]);
    const float jy = ((g[3] - g[4]) + (g[7] - g[8])) + ((g[10] - g[9]) + (g[15] - g[16])) + (g[17] - g[18]);
    const float jz = ((g[5] - g[6]) + (g[11] - g[12])) + ((g[14] - g[13]) + (g[15] - g[16])) + (g[18] - g[17]);
    const float ux = fmaf(0.5f, F[0], jx) * inv;
    const float uy = fmaf(0.5f, F[1], jy) * inv;
    const float uz = fmaf(0.5f, F[2], jz) * inv;
    const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float uF = fmaf(ux, F[0], fmaf(uy, F[1], uz * F[2]));
    const float om = p.omega, keep = 1.f - p.omega;
    const float w0 = 1.f / 3.f, w1 = 1.f / 18.f, w2 = 1.f / 36.f;
    {   // rest population: g_eq = w0 (dn - 1.5 n uu), S = cw0 (-3 uF)
        const float geq = w0 * fmaf(-1.5f * n, uu, dn);
        out[0] = fmaf(keep, g[0], fmaf(om, geq, p.cw[0] * (-3.f * uF)));
    }
    const float base1 = fmaf(-1.5f * n, uu, dn);   // dn - 1.5 n uu
    const float nb = 4.5f * n;
#define SCLBM_PAIR(I, W, CW, CU, CF)                                            \
    {                                                                           \
        const float cu = (CU), cF = (CF);                                       \
        const float ev = (W) * fmaf(nb * cu, cu, base1);                        \
        const float od = (W) * (3.f * n) * cu;                                  \
        const float sev = (CW) * fmaf(9.f * cu, cF, -3.f * uF);                 \
        const float sod = (CW) * 3.f * cF;                                      \
        out[I] = fmaf(keep, g[I], fmaf(om, ev + od, sev + sod));                \
        out[I + 1] = fmaf(keep, g[I + 1], fmaf(om, ev - od, sev - sod));        \
    }
    SCLBM_PAIR(1, w1, p.cw[1], ux, F[0])
    SCLBM_PAIR(3, w1, p.cw[1], uy, F[1])
    SCLBM_PAIR(5, w1, p.cw[1], uz, F[2])
    SCLBM_PAIR(7, w2, p.cw[2], ux + uy, F[0] + F[1])
    SCLBM_PAIR(9, w2, p.cw[2], ux - uy, F[0] - F[1])
    SCLBM_PAIR(11, w2, p.cw[2], ux + uz, F[0] + F[2])
    SCLBM_PAIR(13, w2, p.cw[2], ux - uz, F[0] - F[2])
    SCLBM_PAIR(15, w2, p.cw[2], uy + uz, F[1] + F[2])
    SCLBM_PAIR(17, w2, p.cw[2], uy - uz, F[1] - F[2])
#undef SCLBM_PAIR
}

// Write a node's 19 post-collision populations; on a padded layout also its
// periodic images in the ghost columns (x < 4, x >= nx-4) and rows (y < 3,
// y >= ny-3), so the next step's plane boxes read valid neighbours.
__device__ __forceinline__ void store19(float *__restrict__ B, const Params &p, int x, int y, int z,
                                        const float *out) {
    const int base = z * p.pplane + (y + p.oy) * p.nxp + (x + p.ox);
#pragma unroll
    for (int i = 0; i < 19; ++i) B[i * p.Np + base] = out[i];
    if (p.ox == 0 && p.oy == 0) return;
    const int gx = x < p.ox ? x + p.nx : (x >= p.nx - p.ox ? x - p.nx : INT_MIN);
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
