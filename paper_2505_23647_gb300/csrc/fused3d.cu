// fused3d.cu -- single-pass Shan-Chen step for D3Q19 with shifted binary32
// populations and forcing stencils made of the E8 groups (radius <= 2), for
// lattices of any size (the TMA variant in fused3d_tma.cu covers sizes that
// tile exactly and keeps a ghost-padded layout).
//
// One launch = one step (eqs. lbm, omega_i, f_eq, GuoForcing, sc_f): the
// populations cross HBM once each way (2 x 19 x 4 = 152 B per node) and psi
// never leaves the SM.
//   * a CTA owns a 32 x 8 column tile and marches a chunk of z planes;
//   * the pulled populations A_i(x - xi_i) of the next plane (tile plus a
//     radius-R halo) are copied into a double-buffered shared-memory stage
//     with cp.async while the current plane is processed;
//   * from the stage it forms n and psi (exp(-1/n) or psi_eps) of the plane into a ring
//     of 2R+2 planes (the halo psi is recomputed from populations the
//     neighbouring tiles read too, so those reads hit L2);
//   * then it collides plane zz - R: stencil force from the ring, the node's
//     populations pulled again (L1/L2), BGK + Guo, one coalesced write.
// Binary32 arithmetic with FMA contraction; results agree with the binary64
// reference within binary32 rounding (tested), not bit for bit.
#include <cuda_runtime.h>

#include <atomic>

#include "fusedcommon.cuh"

namespace sclbm {

namespace fz {

using namespace fc;

// row offsets (inside a padded plane) of the nine (c_y, c_x) pull sources
__device__ __forceinline__ void row_offsets(int x, int y, const Params &p, int *ro) {
#pragma unroll
    for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
            ro[(cy + 1) * 3 + (cx + 1)] =
                (wrap1(y - cy, p.ny) + p.oy) * p.nxp + wrap1(x - cx, p.nx) + p.ox;
}

__device__ __forceinline__ void plane_offsets(int zz, const Params &p, int *zo) {
    zo[0] = wrap1(zz + 1, p.nz) * p.pplane;   // c_z = -1: source at zz + 1
    zo[1] = zz * p.pplane;
    zo[2] = wrap1(zz - 1, p.nz) * p.pplane;   // c_z = +1: source at zz - 1
}

// pulled populations f_i(x,y,zz) = A_i((x,y,zz) - xi_i)
__device__ __forceinline__ void pull19(const float *__restrict__ A, const int *ro, const int *zo,
                                       int Np, float *g) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = cvel<19>(i, 0), cy = cvel<19>(i, 1), cz = cvel<19>(i, 2);
        g[i] = __ldg(A + i * Np + zo[cz + 1] + ro[(cy + 1) * 3 + (cx + 1)]);
    }
}

// asynchronous 4-byte global -> shared copy (cp.async, L1-allocating)
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// stage[i * EXY + node] = A_i(node - xi_i) for one plane
template <int EXY>
__device__ __forceinline__ void stage_plane(const float *__restrict__ A, float *stage, int node,
                                            const int *ro, const int *zo, int Np) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = cvel<19>(i, 0), cy = cvel<19>(i, 1), cz = cvel<19>(i, 2);
        cp_async4(stage + i * EXY + node, A + (i * Np + zo[cz + 1] + ro[(cy + 1) * 3 + (cx + 1)]));
    }
}

template <int EXY, bool EPS>
__device__ __forceinline__ float psi_from_stage(const float *stage, int node, const Params &p,
                                                bool &bad) {
    float g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) g[i] = stage[i * EXY + node];
    const float n = dens(g) + p.rho0;
    bad |= !(n > 0.f);
    return psi_fused<EPS>(n, p.eps, p.inv_eps);
}

template <int R, int NG, bool EPS, bool F2>
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
    int ro_h[9];
    int hx = 0, hy = 0;
    const bool has_halo = t < HALO;
    if (has_halo) {
        halo_coords<R>(t, hx, hy);
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
        stage_plane<EXY>(A, stage0, cen, ro_i, zo, p.Np);
        if (has_halo) stage_plane<EXY>(A, stage0, hof, ro_h, zo, p.Np);
        cp_commit();
    }
    for (int it = 0; it < nit; ++it) {
        const int zz = wrap1(z0 - R + it, p.nz);
        float *cur = (it & 1) ? stage1 : stage0;
        float *nxt = (it & 1) ? stage0 : stage1;
        if (it + 1 < nit) {   // prefetch plane it + 1 while this one is consumed
            int zo[3];
            plane_offsets(wrap1(zz + 1, p.nz), p, zo);
            stage_plane<EXY>(A, nxt, cen, ro_i, zo, p.Np);
            if (has_halo) stage_plane<EXY>(A, nxt, hof, ro_h, zo, p.Np);
        }
        cp_commit();
        cp_wait1();
        __syncthreads();
        float *slot = ring + (it % NS) * EXY;
        slot[cen] = psi_from_stage<EXY, EPS>(cur, cen, p, bad);
        if (has_halo) {
            bool dummy = false;
            slot[hof] = psi_from_stage<EXY, EPS>(cur, hof, p, dummy);
        }
        __syncthreads();
        if (it < 2 * R) continue;
        // ---- collide plane zc = zz - R --------------------------------------
        const int zc = wrap1(zz - R, p.nz);
        int zoc[3];
        plane_offsets(zc, p, zoc);
        float g[19];
        pull19(A, ro_i, zoc, p.Np, g);            // in flight during the force loop
        const float *pz[2 * R + 1];
#pragma unroll
        for (int k = -R; k <= R; ++k) pz[k + R] = ring + ((it - R + k + NS) % NS) * EXY + cen;
        float F[3];
        force_ring<R, NG, EX>(pz, p, F);
        float out[19];
        collide19<F2>(g, dens(g), F, p, out);
        if (owner) store19(B, p, xi, yi, zc, out);
    }
    if (bad) atomicMin(&flags->err_step, flags->step);
    finish_step(flags, t);
}

template <int R>
constexpr int smem_bytes() {
    return (2 * R + 2 + 2 * 19) * (TX + 2 * R) * (TY + 2 * R) * 4;
}

template <int R, int NG, bool EPS, bool F2>
void launch1(dim3 grid, dim3 block, const float *A, float *B, const Params &p, lb_ctx *c) {
    static std::atomic<unsigned long long> attr_done{0};   // devices done, one bit each
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ULL << (dev & 63);
    if (!(attr_done.load() & bit)) {
        cudaFuncSetAttribute(k_fused3d<R, NG, EPS, F2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<R>());
        attr_done.fetch_or(bit);
    }
    k_fused3d<R, NG, EPS, F2><<<grid, block, smem_bytes<R>(), c->stream>>>(A, B, p, c->flags);
}

// the instantiation for the stencil's widest group (ng = 1..7), the psi kind
// and the forcing variant
template <bool EPS, bool F2>
void launch(int ng, dim3 grid, dim3 block, const float *A, float *B, const Params &p, lb_ctx *c) {
    switch (ng) {
        case 1: launch1<1, 1, EPS, F2>(grid, block, A, B, p, c); break;
        case 2: launch1<1, 2, EPS, F2>(grid, block, A, B, p, c); break;
        case 3: launch1<1, 3, EPS, F2>(grid, block, A, B, p, c); break;
        case 4: launch1<2, 4, EPS, F2>(grid, block, A, B, p, c); break;
        case 5: launch1<2, 5, EPS, F2>(grid, block, A, B, p, c); break;
        case 6: launch1<2, 6, EPS, F2>(grid, block, A, B, p, c); break;
        default: launch1<2, 7, EPS, F2>(grid, block, A, B, p, c); break;
    }
}

}  // namespace fz

bool fused3d_applicable(const lb_ctx *c, float *W, int *ng) {
    if (c->p.precision != LB_FP32_SHIFTED || c->Q != 19)
        return false;
    if (c->g.nx < 8 || c->g.ny < 8 || c->g.nz < 8) return false;
    if ((long long)19 * c->g.Np >= (1LL << 31)) return false;
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

fc::Params fused_params(const lb_ctx *c, const float *W) {
    fc::Params p;
    for (int q = 0; q < 7; ++q) p.W[q] = W[q];
    double M1 = 0.0, M2 = 0.0;
    {   // plane-split force: weights summed over the in-plane rings k = 0,1,2,4,5
        // at z offsets 1 and 2 (|e|^2 = k + d^2; groups 0..6 have |e|^2 = 1,2,3,4,5,6,8)
        const double w[7] = {W[0], W[1], W[2], W[3], W[4], W[5], W[6]};
        M1 = w[0] + 4.0 * w[1] + 4.0 * w[2] + 4.0 * w[4] + 8.0 * w[5];
        M2 = 2.0 * (w[3] + 4.0 * w[4] + 4.0 * w[5] + 4.0 * w[6]);
    }
    for (int q = 0; q < 7; ++q) p.W2[q] = 2.f * W[q];
    p.M1 = (float)M1;
    p.M2 = (float)M2;
    const double om = c->k.omega;
    p.omega = (float)om;
    p.keep = c->k.keep32;
    p.mGp = (float)c->k.mGp;
    p.rho0 = (float)c->k.rho0;
    p.eps = c->k.psi_kind == LB_PSI_EPS ? (float)c->k.psi_eps : 0.f;
    p.inv_eps = c->k.psi_kind == LB_PSI_EPS ? (float)c->k.psi_inv : 0.f;
    const double pref = 1.0 - 1.0 / (2.0 * c->p.tau);
    const double wc[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    const double kA = c->k.kA;
    p.mhkA = (float)(-0.5 * kA);
    for (int k = 0; k < 3; ++k) {
        const double cw = pref * wc[k];
        p.kq[k] = (float)(-4.5 * cw * kA);
        p.omw[k] = c->k.omw32[k];   // mass-exact with keep
        p.m3cw[k] = (float)(-3.0 * cw);
        p.b45[k] = (float)(4.5 * om * wc[k]);
        p.d3[k] = (float)(3.0 * om * wc[k]);
        p.c9[k] = (float)(9.0 * cw);
        p.c3[k] = (float)(3.0 * cw);
    }
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    p.nz = c->g.nz;
    p.nxp = c->g.nxp;
    p.nyp = c->g.nyp;
    p.ox = c->g.ox;
    p.oy = c->g.oy;
    p.pplane = c->g.nxp * c->g.nyp;
    p.Np = (int)c->g.Np;
    p.zchunk = c->fused_zchunk > 0 ? c->fused_zchunk : 28;
    p.max_polls = c->wait_polls;
    return p;
}

cudaError_t f32_fused3d_step(lb_ctx *c, const float *W, int ng) {
    if (c->tma_ok && c->fused_tma) return f32_fused3d_tma_step(c, W, ng);
    fc::Params p = fused_params(c, W);
    dim3 block(fc::TX, fc::TY);
    dim3 grid((c->g.nx + fc::TX - 1) / fc::TX, (c->g.ny + fc::TY - 1) / fc::TY,
              (c->g.nz + p.zchunk - 1) / p.zchunk);
    const float *A = (const float *)c->f[c->cur];
    float *B = (float *)c->f[1 - c->cur];
    tm_begin(c, LB_KERNEL_FUSED);
    const bool eps = p.inv_eps != 0.f, f2 = c->k.kA != 0.0;
    if (eps && f2)
        fz::launch<true, true>(ng, grid, block, A, B, p, c);
    else if (eps)
        fz::launch<true, false>(ng, grid, block, A, B, p, c);
    else if (f2)
        fz::launch<false, true>(ng, grid, block, A, B, p, c);
    else
        fz::launch<false, false>(ng, grid, block, A, B, p, c);
    tm_end(c);
    c->launches += 1;
    c->cur = 1 - c->cur;
    return cudaGetLastError();
}

}  // namespace sclbm
