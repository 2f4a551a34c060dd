// fp32.cu -- binary32 path with shifted populations g_i = f_i - w_i rho0
// (generic kernels for every lattice and stencil).
#include <cuda_runtime.h>

#include "fusedcommon.cuh"

namespace sclbm {

fc::Params fused_params(const lb_ctx *c, const float *W);

// The generic binary32 collision.  A block of CT_X x CT_Y threads takes one
// brick (CT_X x CT_Y x CT_Z nodes in 3D, CT_X x CT_Y2 in 2D); the brick's
// psi box (PSI_HALO more on every side) is read from the halo'd field into
// shared memory once.  Each thread first forms the force sums of all its
// nodes (a column of NPT nodes), pair by pair, so that a pair's offset and
// folded weights are read once for NPT nodes; per node the operations are
// those of force_fast in the same order, so the result is bit for bit the
// one the global-memory form gives.  Then it pulls, collides (D3Q19: the
// fused kernels' pair-symmetric collide19 with their mass-exact constants,
// cp; D2Q9: the generic collision) and stores its
// nodes one by one, with their periodic images on a padded layout (as the
// fused kernels write them), so no separate ghost refresh follows the step.
// Requires the halo'd psi field (fewer than 2^31 of its nodes) and dynamic
// shared memory of ct_box(D) floats.
template <int D, int Q>
__global__ void __launch_bounds__(CT_X * CT_Y) k_collide_f32(const float *__restrict__ A, float *__restrict__ B,
                                                     const float *__restrict__ psi, Geom g,
                                                     const PairsFast PF, const ConstsT<float> k,
                                                     const fc::Params cp, Flags *flags) {
    extern __shared__ __align__(16) float sps[];
    constexpr int BX = CT_BX, BY = ct_by(D), BZ = ct_bz(D);
    constexpr int NPT = D == 3 ? CT_Z : CT_Y2 / CT_Y;   // nodes a thread takes
    // shared-memory distance between a thread's consecutive nodes
    constexpr int STEP = D == 3 ? BX * BY : CT_Y * BX;
    const int x0 = blockIdx.x * CT_X, y0 = blockIdx.y * (D == 3 ? CT_Y : CT_Y2);
    const int z0 = D == 3 ? blockIdx.z * CT_Z : 0;
    const int t = threadIdx.y * CT_X + threadIdx.x;
    // the box's origin in the halo'd field is node (x0 - H, y0 - H, z0 - Hz):
    // BY * BZ rows of BX floats from row (z0 + bz) * pyp + y0 + by, column x0
    const int fz_end = g.nz + 2 * PF.Hz;
    if ((PF.pxp & 3) == 0) {   // rows start on 16 bytes: float4 copies
        constexpr int V = BX / 4;
        for (int e = t; e < V * BY * BZ; e += CT_X * CT_Y) {
            const int r = e / V, q = e - r * V;
            const int by = r % BY, bz = r / BY;
            const int fx = x0 + 4 * q, fy = y0 + by, fz = z0 + bz;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (fx < PF.pxp && fy < PF.pyp && fz < fz_end)
                v = *reinterpret_cast<const float4 *>(psi + (fz * PF.pyp + fy) * PF.pxp + fx);
            reinterpret_cast<float4 *>(sps)[e] = v;
        }
    } else {
        for (int e = t; e < BX * BY * BZ; e += CT_X * CT_Y) {
            const int bx = e % BX, r = e / BX, by = r % BY, bz = r / BY;
            const int fx = x0 + bx, fy = y0 + by, fz = z0 + bz;
            float v = 0.f;
            if (fx < PF.pxp && fy < PF.pyp && fz < fz_end) v = psi[(fz * PF.pyp + fy) * PF.pxp + fx];
            sps[e] = v;
        }
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    // smem index of the thread's first node
    const int c0 = (PF.Hz * BY + threadIdx.y + PF.H) * BX + threadIdx.x + PF.H;
    float acc[NPT][3];
#pragma unroll
    for (int j = 0; j < NPT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = 0.f;
#pragma unroll 2
    for (int a = 0; a < PF.npairs; ++a) {
        const int o = PF.nbs[a];
        const float w0 = PF.we[a][0], w1 = PF.we[a][1], w2 = PF.we[a][2];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const float d = sps[c0 + j * STEP + o] - sps[c0 + j * STEP - o];
            acc[j][0] = fmaf(w0, d, acc[j][0]);
            acc[j][1] = fmaf(w1, d, acc[j][1]);
            if (D == 3) acc[j][2] = fmaf(w2, d, acc[j][2]);
        }
    }
    // the node loop is not unrolled (one copy of the pull, collision and
    // stores); acc[0] always holds the current node's sums, shifted down
    // after each node
#pragma unroll 1
    for (int j = 0; j < NPT; ++j) {
        const int y = D == 3 ? y0 + threadIdx.y : y0 + threadIdx.y + CT_Y * j;
        const int z = D == 3 ? z0 + j : 0;
        const float s0 = acc[0][0], s1 = acc[0][1], s2 = acc[0][2];
#pragma unroll
        for (int q = 0; q + 1 < NPT; ++q) {
            acc[q][0] = acc[q + 1][0];
            acc[q][1] = acc[q + 1][1];
            acc[q][2] = acc[q + 1][2];
        }
        if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
        float fi[Q];
        pull_f32<D, Q>(A, g, x, y, z, PF, fi);
        const float dn = sum_q<float, Q>(fi);
        const float n = dn + k.rho0;
        const float pre = k.mGp * sps[c0 + j * STEP];
        float F[3] = {0.f, 0.f, 0.f};
        F[0] = pre * s0;
        F[1] = pre * s1;
        if (D == 3) F[2] = pre * s2;
        float fo[Q];
        if constexpr (Q == 19) {   // the fused kernels' pair-symmetric collision
            if (cp.mhkA != 0.f) fc::collide19<true>(fi, dn, F, cp, fo);
            else fc::collide19<false>(fi, dn, F, cp, fo);
        } else {
            collide<float, D, Q, true>(fi, n, dn, F, k, fo, nullptr, nullptr);
        }
        // the node, and on a padded layout its periodic images (ghost
        // columns, rows, corners): one store loop over the destinations
        const long long zb = (long long)z * g.nyp;
        const long long p0 = (zb + (y + g.oy)) * g.nxp + (x + g.ox);
        long long p1 = 0, p2 = 0, p3 = 0;
        unsigned m = 1u;
        if (D == 3 && g.oy > 0) {
            const int gx = x < GHOST_X ? x + g.nx : (x >= g.nx - GHOST_X ? x - g.nx : INT_MIN);
            const int gy = y < g.oy ? y + g.ny : (y >= g.ny - g.oy ? y - g.ny : INT_MIN);
            if (gx != INT_MIN) {
                p1 = (zb + (y + g.oy)) * g.nxp + (gx + g.ox);
                m |= 2u;
            }
            if (gy != INT_MIN) {
                p2 = (zb + (gy + g.oy)) * g.nxp + (x + g.ox);
                m |= 4u;
                if (gx != INT_MIN) {
                    p3 = (zb + (gy + g.oy)) * g.nxp + (gx + g.ox);
                    m |= 8u;
                }
            }
        }
#pragma unroll 1
        for (int d = 0; d < 4; ++d) {
            if (!((m >> d) & 1u)) continue;
            const long long o = d == 0 ? p0 : (d == 1 ? p1 : (d == 2 ? p2 : p3));
#pragma unroll
            for (int i = 0; i < Q; ++i) B[(long long)i * g.Np + o] = fo[i];
        }
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && t == 0)
        flags->step = flags->step + 1;
}


cudaError_t ghosts_refresh(lb_ctx *c) {
    if (!c->padded) return cudaSuccess;
    const long long rows = (long long)c->g.nyp * c->g.nz * c->Q;   // one warp a row
    k_ghosts<float><<<grid_for(rows * 32), 256, 0, c->stream>>>((float *)c->f[c->cur], c->g, c->Q);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_init(lb_ctx *c, const double *rho, const double *u) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    float *A = (float *)c->f[c->cur];
    if (c->Q == 9)
        k_init<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, rho, u, k);
    else
        k_init<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, rho, u, k);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : ghosts_refresh(c);
}

cudaError_t f32_step(lb_ctx *c) {
    if (c->Q == 19 && c->fast3d_ok && c->fused_enabled)
        return f32_fused3d_step(c, c->fused_W, c->fused_ng);
    if (c->Q == 9 && c->fast2d_ok && c->fused_enabled) return f32_fused2d_step(c);
    auto k = consts_as<float>(c->k);
    const float *A = (const float *)c->f[c->cur];
    float *B = (float *)c->f[1 - c->cur];
    float *psi = (float *)c->psi;
    const float W0[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // the force is not the fused one
    const fc::Params cp = fused_params(c, W0);
    int gb = grid_for(c->g.N);
    if (!c->psi_halo) {   // beyond 32-bit node indices: the wrapped kernels
        if (c->Q == 9) {
            k_psi<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->flags, psik(c));
            k_collide<float, PairsF32, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, B, psi, c->g, c->pairs32, k, c->flags);
        } else {
            k_psi<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->flags, psik(c));
            k_collide<float, PairsF32, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, B, psi, c->g, c->pairs32, k, c->flags);
        }
    } else if (c->Q == 9) {
        tm_begin(c, LB_KERNEL_PSI);
        k_psi_f32<2, 9><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->pfast, c->flags, psik(c));
        tm_end(c);
        tm_begin(c, LB_KERNEL_COLLIDE);
        const dim3 grid((c->g.nx + CT_X - 1) / CT_X, (c->g.ny + CT_Y2 - 1) / CT_Y2, 1);
        k_collide_f32<2, 9><<<grid, dim3(CT_X, CT_Y), ct_box(2) * sizeof(float), c->stream>>>(
            A, B, psi, c->g, c->pfast, k, cp, c->flags);
        tm_end(c);
    } else {
        tm_begin(c, LB_KERNEL_PSI);
        k_psi_f32<3, 19><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->pfast, c->flags, psik(c));
        tm_end(c);
        tm_begin(c, LB_KERNEL_COLLIDE);
        const dim3 grid((c->g.nx + CT_X - 1) / CT_X, (c->g.ny + CT_Y - 1) / CT_Y,
                        (c->g.nz + CT_Z - 1) / CT_Z);
        k_collide_f32<3, 19><<<grid, dim3(CT_X, CT_Y), ct_box(3) * sizeof(float), c->stream>>>(
            A, B, psi, c->g, c->pfast, k, cp, c->flags);
        tm_end(c);
    }
    c->launches += 2;
    c->cur = 1 - c->cur;
    cudaError_t e = cudaGetLastError();
    // k_collide_f32 writes the ghost images itself; the wrapped kernels do not
    return e != cudaSuccess || c->psi_halo ? e : ghosts_refresh(c);
}

cudaError_t f32_density_psi(lb_ctx *c, double *n, double *psi) {
    int gb = grid_for(c->g.N);
    const float *A = (const float *)c->f[c->cur];
    if (c->Q == 9)
        k_density_psi64<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->k.rho0, n, psi, c->flags, psik(c));
    else
        k_density_psi64<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->k.rho0, n, psi, c->flags, psik(c));
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_fields(lb_ctx *c, double *n, double *u, double *mom) {
    cudaError_t e = f32_density_psi(c, n, n + c->g.N);
    if (e != cudaSuccess) return e;
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const float *A = (const float *)c->f[c->cur];
    // the widened populations keep their shift: n already includes rho0, and
    // j, u and j + F/2 do not depend on it (sum_i w_i xi_i = 0)
    if (c->Q == 9)
        k_fields64<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->pairs64, k, n, n + c->g.N, u, mom);
    else
        k_fields64<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->pairs64, k, n, n + c->g.N, u, mom);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_get_state(lb_ctx *c, double *f, int i0, int i1) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const float *A = (const float *)c->f[c->cur];
    if (c->Q == 9)
        k_get_state<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    else
        k_get_state<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_set_state(lb_ctx *c, const double *f, int i0, int i1) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    float *A = (float *)c->f[c->cur];
    if (c->Q == 9)
        k_set_state<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    else
        k_set_state<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace sclbm
