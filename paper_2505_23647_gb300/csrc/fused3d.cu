// fused3d.cu -- single-pass Shan-Chen step for D3Q19 with shifted binary32
// populations and forcing stencils made of the E8 groups (1,0,0), (1,1,0),
// (1,1,1), (2,0,0), (2,1,0), (2,1,1), (2,2,0) (any weights, radius <= 2).
//
// One launch = one step (eqs. lbm, omega_i, f_eq, GuoForcing, sc_f), so the
// populations cross HBM once each way (2 x 19 x 4 = 152 B per node) and psi
// never leaves the SM:
//   * a CTA owns a 32 x 8 column tile and marches a chunk of z planes;
//   * for plane zz it pulls the populations A_i(x - xi_i) of the tile plus a
//     radius-R halo, forms n and psi = exp(-1/n), and stores psi in a ring
//     of 2R+2 planes in shared memory (the halo psi is recomputed from
//     populations the neighbouring tiles read too, so those reads hit L2);
//   * then it collides plane zz - R: the stencil force reads the ring, the
//     tile's populations are pulled again (L1/L2 hits), BGK + Guo are applied
//     and the post-collision populations are written once, coalesced.
// The force is accumulated per symmetry group and weighted once per group;
// equilibrium and Guo source are formed from their parts even and odd in
// xi (one evaluation per pair of opposite velocities).  Binary32 arithmetic
// with FMA contraction; results agree with the binary64 reference within
// binary32 rounding (tested), not bit for bit.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace sclbm {

namespace fz {

constexpr int TX = 32, TY = 8;

// canonical (e,-e) pairs of the seven E8 groups: e_x, e_y, e_z, group
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
    int nx, ny, nz, plane, N, zchunk;
};

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// row offsets of the nine (c_y, c_x) pull sources of column (x, y)
__device__ __forceinline__ void row_offsets(int x, int y, const Params &p, int *ro) {
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
            ro[(cy + 1) * 3 + (cx + 1)] = wrap1(y - cy, p.ny) * p.nx + wrap1(x - cx, p.nx);
}

// pulled populations f_i(x,y,zz) = A_i((x,y,zz) - xi_i); zo[cz+1] = plane offset of zz - cz
__device__ __forceinline__ void pull19(const float *__restrict__ A, const int *ro, const int *zo,
                                       int N, float *g) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = cvel<19>(i, 0), cy = cvel<19>(i, 1), cz = cvel<19>(i, 2);
        g[i] = __ldg(A + i * N + zo[cz + 1] + ro[(cy + 1) * 3 + (cx + 1)]);
    }
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

// asynchronous 4-byte global -> shared copy (cp.async, L1-allocating)
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// stage the pulled populations of one plane (tile plus halo) into shared
// memory: stage[i * EXY + node] = A_i(node - xi_i)
template <int EXY>
__device__ __forceinline__ void stage_plane(const float *__restrict__ A, float *stage, int node,
                                            const int *ro, const int *zo, int N) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = cvel<19>(i, 0), cy = cvel<19>(i, 1), cz = cvel<19>(i, 2);
        cp_async4(stage + i * EXY + node, A + (i * N + zo[cz + 1] + ro[(cy + 1) * 3 + (cx + 1)]));
    }
}

template <int EXY>
__device__ __forceinline__ float psi_from_stage(const float *stage, int node, float rho0, bool &bad) {
    float g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) g[i] = stage[i * EXY + node];
    const float n = dens(g) + rho0;
    bad |= !(n > 0.f);
    return expf(-__frcp_rn(n));
}

__device__ __forceinline__ void plane_offsets(int zz, const Params &p, int *zo) {
    zo[0] = wrap1(zz + 1, p.nz) * p.plane;   // c_z = -1: source at zz + 1
    zo[1] = zz * p.plane;
    zo[2] = wrap1(zz - 1, p.nz) * p.plane;   // c_z = +1: source at zz - 1
}

template <int R, int NG>
__global__ void __launch_bounds__(TX * TY, 2)
    k_fused3d(const float *__restrict__ A, float *__restrict__ B, const Params p, Flags *flags) {
    constexpr int EX = TX + 2 * R, EY = TY + 2 * R, NS = 2 * R + 2, EXY = EX * EY;
    constexpr int HALO = EXY - TX * TY;
    extern __shared__ float smem[];
    float *ring = smem;                          // NS planes of psi
    float *stage0 = smem + NS * EXY;             // two planes of staged populations
    float *stage1 = stage0 + 19 * EXY;

    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool owner = gx < p.nx && gy < p.ny;
    const int xi = gx % p.nx, yi = gy % p.ny;   // ragged tiles wrap periodically

    int ro_i[9];
    row_offsets(xi, yi, p, ro_i);
    // halo node of this thread (if any), in extended coordinates (hx, hy)
    int ro_h[9];
    int hx = 0, hy = 0;
    const bool has_halo = t < HALO;
    if (has_halo) {
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
        const int ax = ((x0 + hx - R) % p.nx + p.nx) % p.nx;
        const int ay = ((y0 + hy - R) % p.ny + p.ny) % p.ny;
        row_offsets(ax, ay, p, ro_h);
    }
    const int cen = (ty + R) * EX + (tx + R);
    const int hof = hy * EX + hx;
    bool bad = false;

    const int nit = (z1 - z0) + 2 * R;
    {   // stage the first plane
        int zo[3];
        plane_offsets(wrap1(z0 - R, p.nz), p, zo);
        stage_plane<EXY>(A, stage0, cen, ro_i, zo, p.N);
        if (has_halo) stage_plane<EXY>(A, stage0, hof, ro_h, zo, p.N);
        cp_commit();
    }
    for (int it = 0; it < nit; ++it) {
        const int zz = wrap1(z0 - R + it, p.nz);
        float *cur = (it & 1) ? stage1 : stage0;
        float *nxt = (it & 1) ? stage0 : stage1;
        // prefetch plane it + 1 while this one is consumed
        if (it + 1 < nit) {
            int zo[3];
            plane_offsets(wrap1(zz + 1, p.nz), p, zo);
            stage_plane<EXY>(A, nxt, cen, ro_i, zo, p.N);
            if (has_halo) stage_plane<EXY>(A, nxt, hof, ro_h, zo, p.N);
        }
        cp_commit();
        cp_wait1();
        __syncthreads();
        float *slot = ring + (it % NS) * EXY;
        slot[cen] = psi_from_stage<EXY>(cur, cen, p.rho0, bad);
        if (has_halo) {
            bool dummy = false;
            slot[hof] = psi_from_stage<EXY>(cur, hof, p.rho0, dummy);
        }
        __syncthreads();
        if (it < 2 * R) continue;
        // ---- collide plane zc = zz - R --------------------------------------
        const int zc = wrap1(zz - R, p.nz);
        int zoc[3];
        plane_offsets(zc, p, zoc);
        float g[19];
        pull19(A, ro_i, zoc, p.N, g);            // in flight during the force loop
        const float *pz[2 * R + 1];
#pragma unroll
        for (int k = -R; k <= R; ++k) pz[k + R] = ring + ((it - R + k + NS) % NS) * EXY + cen;
        float F[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < group_end(NG - 1); ++a) {
            const int ex = pair_c(a, 0), ey = pair_c(a, 1), ez = pair_c(a, 2), gq = pair_c(a, 3);
            const float d = pz[R + ez][ey * EX + ex] - pz[R - ez][-ey * EX - ex];
            if (ex) F[0] = fmaf(ex == 1 ? p.W[gq] : ex == -1 ? -p.W[gq] : (float)ex * p.W[gq], d, F[0]);
            if (ey) F[1] = fmaf(ey == 1 ? p.W[gq] : ey == -1 ? -p.W[gq] : (float)ey * p.W[gq], d, F[1]);
            if (ez) F[2] = fmaf(ez == 1 ? p.W[gq] : ez == -1 ? -p.W[gq] : (float)ez * p.W[gq], d, F[2]);
        }
        {
            const float pre = p.mGp * pz[R][0];
            F[0] *= pre;
            F[1] *= pre;
            F[2] *= pre;
        }
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
        float out[19];
        {   // rest population: g_eq = w0 (dn - 1.5 n uu), S = cw0 (-3 uF)
            const float geq = w0 * fmaf(-1.5f * n, uu, dn);
            out[0] = fmaf(keep, g[0], fmaf(om, geq, p.cw[0] * (-3.f * uF)));
        }
        const float base1 = fmaf(-1.5f * n, uu, dn);   // dn - 1.5 n uu
        const float nb = 4.5f * n;
        // one evaluation per opposite pair (i, i+1): even part +/- odd part
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
        if (owner) {
            const int s = zc * p.plane + yi * p.nx + xi;
#pragma unroll
            for (int i = 0; i < 19; ++i) B[i * p.N + s] = out[i];
        }
    }
    if (bad) atomicMin(&flags->err_step, flags->step);
    // the last block to finish advances the device step counter
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

template <int R>
constexpr int smem_bytes() {
    return (2 * R + 2 + 2 * 19) * (TX + 2 * R) * (TY + 2 * R) * 4;
}

}  // namespace fz

bool fused3d_applicable(const lb_ctx *c, float *W, int *ng) {
    if (c->p.precision != LB_FP32_SHIFTED || c->Q != 19) return false;
    if (c->g.nx < 8 || c->g.ny < 8 || c->g.nz < 8) return false;
    if ((long long)19 * c->g.N >= (1LL << 31)) return false;
    static const int bases[7][3] = {{1, 0, 0}, {1, 1, 0}, {1, 1, 1}, {2, 0, 0},
                                    {2, 1, 0}, {2, 1, 1}, {2, 2, 0}};
    for (int q = 0; q < 7; ++q) W[q] = 0.f;
    int hi = 0;
    for (int gq = 0; gq < c->n_groups; ++gq) {
        int found = -1;
        for (int q = 0; q < 7; ++q)
            if (c->group_base[gq][0] == bases[q][0] && c->group_base[gq][1] == bases[q][1] &&
                c->group_base[gq][2] == bases[q][2])
                found = q;
        if (found < 0) return false;
        W[found] = (float)c->group_w[gq];
        hi = found + 1 > hi ? found + 1 : hi;
    }
    *ng = hi;
    return true;
}

cudaError_t f32_fused3d_step(lb_ctx *c, const float *W, int ng) {
    fz::Params p;
    for (int q = 0; q < 7; ++q) p.W[q] = W[q];
    p.omega = (float)c->k.omega;
    p.mGp = (float)c->k.mGp;
    p.rho0 = (float)c->k.rho0;
    const double pref = 1.0 - 1.0 / (2.0 * c->p.tau);
    p.cw[0] = (float)(pref / 3.0);
    p.cw[1] = (float)(pref / 18.0);
    p.cw[2] = (float)(pref / 36.0);
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    p.nz = c->g.nz;
    p.plane = c->g.nx * c->g.ny;
    p.N = (int)c->g.N;
    p.zchunk = c->fused_zchunk > 0 ? c->fused_zchunk : 32;
    dim3 block(fz::TX, fz::TY);
    dim3 grid((c->g.nx + fz::TX - 1) / fz::TX, (c->g.ny + fz::TY - 1) / fz::TY,
              (c->g.nz + p.zchunk - 1) / p.zchunk);
    const float *A = (const float *)c->f[c->cur];
    float *B = (float *)c->f[1 - c->cur];
    tm_begin(c, LB_KERNEL_FUSED);
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(fz::k_fused3d<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<1>());
        cudaFuncSetAttribute(fz::k_fused3d<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<1>());
        cudaFuncSetAttribute(fz::k_fused3d<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<1>());
        cudaFuncSetAttribute(fz::k_fused3d<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<2>());
        cudaFuncSetAttribute(fz::k_fused3d<2, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<2>());
        cudaFuncSetAttribute(fz::k_fused3d<2, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<2>());
        cudaFuncSetAttribute(fz::k_fused3d<2, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, fz::smem_bytes<2>());
        attr_done = true;
    }
    const int sm1 = fz::smem_bytes<1>(), sm2 = fz::smem_bytes<2>();
    if (ng <= 3) {
        switch (ng) {
            case 1: fz::k_fused3d<1, 1><<<grid, block, sm1, c->stream>>>(A, B, p, c->flags); break;
            case 2: fz::k_fused3d<1, 2><<<grid, block, sm1, c->stream>>>(A, B, p, c->flags); break;
            default: fz::k_fused3d<1, 3><<<grid, block, sm1, c->stream>>>(A, B, p, c->flags); break;
        }
    } else {
        switch (ng) {
            case 4: fz::k_fused3d<2, 4><<<grid, block, sm2, c->stream>>>(A, B, p, c->flags); break;
            case 5: fz::k_fused3d<2, 5><<<grid, block, sm2, c->stream>>>(A, B, p, c->flags); break;
            case 6: fz::k_fused3d<2, 6><<<grid, block, sm2, c->stream>>>(A, B, p, c->flags); break;
            default: fz::k_fused3d<2, 7><<<grid, block, sm2, c->stream>>>(A, B, p, c->flags); break;
        }
    }
    tm_end(c);
    c->launches += 1;
    c->cur = 1 - c->cur;
    return cudaGetLastError();
}

}  // namespace sclbm
