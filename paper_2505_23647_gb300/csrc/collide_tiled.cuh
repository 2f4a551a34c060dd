// collide_tiled.cuh -- the generic binary32 step's collision kernel (any
// stencil up to radius 4), shared by the D3Q19 and D2Q9 paths.
#pragma once
#include <cuda_runtime.h>

#include "fusedcommon.cuh"

namespace sclbm {

// Collisions of one node (fi pulled, dn shifted density, n = dn + rho0, F
// the force; fo out).  D3Q19: the fused kernels' pair-symmetric collide19
// with their mass-exact constants.
struct Col19 {
    fc::Params p;
    __device__ __forceinline__ void operator()(const float *fi, float dn, float, const float *F,
                                               float *fo) const {
        if (p.mhkA != 0.f) fc::collide19<true>(fi, dn, F, p, fo);
        else fc::collide19<false>(fi, dn, F, p, fo);
    }
};

// The generic binary32 collision.  A block of CT_X x CT_Y threads takes one
// brick (CT_X x CT_Y x CT_Z nodes in 3D, CT_X x CT_Y2 in 2D); the brick's
// psi box (PSI_HALO more on every side) is read from the halo'd field into
// shared memory once.  Each thread first forms the force sums of all its
// nodes (a column of NPT nodes), pair by pair, so that a pair's offset and
// folded weights are read once for NPT nodes; per node the operations are
// those of force_fast in the same order, so the result is bit for bit the
// one the global-memory form gives.  Then it pulls, collides (Col: the
// collision of one node: Col19 here, the D2Q9 one in batch2d.cu) and
// stores its nodes one by one, with their periodic images on a padded
// layout (as the fused kernels write them), so no separate ghost refresh
// follows the step.
// Requires the halo'd psi field (fewer than 2^31 of its nodes) and dynamic
// shared memory of ct_box(D) floats.
template <int D, int Q, class Col>
__global__ void __launch_bounds__(CT_X * CT_Y) k_collide_f32(const float *__restrict__ A, float *__restrict__ B,
                                                     const float *__restrict__ psi, Geom g,
                                                     const PairsFast PF, const ConstsT<float> k,
                                                     const Col col, Flags *flags) {
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
        col(fi, dn, n, F, fo);
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


}  // namespace sclbm
