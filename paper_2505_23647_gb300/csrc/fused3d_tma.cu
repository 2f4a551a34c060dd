// fused3d_tma.cu -- the fused single-pass D3Q19 step with TMA staging.
//
// Same model and schedule as fused3d.cu (32 x 8 column tiles marching z
// chunks, psi ring of 2R+2 planes in shared memory, collision of plane zz-R
// once psi of zz is known), but each plane's populations reach shared memory
// through the Tensor Memory Accelerator: one cp.async.bulk.tensor per
// population (19 per plane per CTA, issued by one thread and completed on an
// mbarrier) instead of one 4-byte copy per population and node.
//
// Layout: the population arrays carry periodic ghost columns (4 on each side
// in x) and rows (3 on each side in y) around every x-y plane, so the box a
// tile needs never wraps; the kernel writes a boundary node's values into its
// ghost images as well (fc::store19).  Population i of plane zz is read from
// A_i(x - xi_i): the box of A_i at plane zz - c_z covering rows
// y0 - R - c_y .. y0 + TY + R - c_y and columns x0 - 4 .. x0 + 36 (16-byte
// aligned start); the pull's x/y shift becomes a compile-time offset when the
// box is read.  Requires nx % 32 == 0, ny % 8 == 0.
//
// Every wait on an mbarrier is bounded: after MAX_POLLS unsuccessful polls
// the block records a timeout in the device counters, waits (bounded) for its
// other copy, and leaves the step; lb_sync reports LB_ECUDA.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "fusedcommon.cuh"

namespace sclbm {

namespace ft {

using namespace fc;

constexpr int BOXW = 40;                  // columns x0 - 4 .. x0 + 35
constexpr long long MAX_POLLS = 1LL << 26;

// floats between consecutive population boxes in a stage (boxes start on
// 128-byte boundaries)
template <int R>
__host__ __device__ constexpr int box_stride() {
    return ((TY + 2 * R) * BOXW + 31) / 32 * 32;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
    for (long long k = 0; k < MAX_POLLS; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(smem_u32(bar))
        : "memory");
}

// issue the 19 population boxes of plane zz into one stage
template <int R>
__device__ __forceinline__ void issue_plane(const CUtensorMap *map, float *stage,
                                            unsigned long long *bar, int zz, int x0, int y0,
                                            const Params &p) {
    constexpr int ROWS = TY + 2 * R, BOX = ROWS * BOXW;
    mbar_expect_tx(bar, 19u * BOX * 4u);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cy = cvel<19>(i, 1), cz = cvel<19>(i, 2);
        tma_load_3d(stage + i * box_stride<R>(), map, x0 + p.ox - 4, y0 + p.oy - R - cy,
                    i * p.nz + wrap1(zz - cz, p.nz), bar);
    }
}

// psi of extended node (ex, ey) of the tile from a stage
template <int R>
__device__ __forceinline__ float psi_from_boxes(const float *stage, int ex, int ey, float rho0,
                                                bool &bad) {
    float g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cx = cvel<19>(i, 0);
        g[i] = stage[i * box_stride<R>() + ey * BOXW + (ex + 4 - R - cx)];
    }
    const float n = dens(g) + rho0;
    bad |= !(n > 0.f);
    return psi32(n);
}

// issue the 19 population boxes of the tile's collision plane zc (rows
// y0 - c_y .. y0 + TY - c_y, the same 40 columns)
__device__ __forceinline__ void issue_collision_plane(const CUtensorMap *map, float *stage,
                                                      unsigned long long *bar, int zc, int x0,
                                                      int y0, const Params &p) {
    constexpr int BOX = TY * BOXW;
    mbar_expect_tx(bar, 19u * BOX * 4u);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cy = cvel<19>(i, 1), cz = cvel<19>(i, 2);
        tma_load_3d(stage + i * BOX, map, x0 + p.ox - 4, y0 + p.oy - cy,
                    i * p.nz + wrap1(zc - cz, p.nz), bar);
    }
}

// Schedule of one CTA (it = 0 .. nit-1, zz = z0 - R + it, zc = zz - R):
//   wait psi-stage(it); psi(zz) -> ring; barrier (+ timeout vote);
//   thread 0 issues psi-stage(it+1) into the single psi stage (all reads of
//   it are behind the barrier) and collision-stage(it+1) into buffer
//   (it+1)&1 (its last reader, collision(it-1), is behind the barrier too);
//   force(zc) from the ring; wait collision-stage(it); collide; store.
// Both copies therefore overlap at least the force and collision phase of
// the iteration before they are needed.
template <int R, int NG>
__global__ void __launch_bounds__(TX * TY, 2)
    k_fused3d_tma(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap cmap,
                  float *__restrict__ B, const Params p, Flags *flags) {
    constexpr int EX = TX + 2 * R, EY = TY + 2 * R, NS = 2 * R + 2, EXY = EX * EY;
    constexpr int HALO = EXY - TX * TY;
    constexpr int STAGE = 19 * box_stride<R>();
    constexpr int CSTAGE = 19 * TY * BOXW;
    extern __shared__ __align__(128) float smem[];
    float *stage = smem;                          // psi plane: 19 boxes, tile + halo
    float *cst0 = smem + STAGE;                   // collision plane, two buffers
    float *cst1 = cst0 + CSTAGE;
    float *ring = cst1 + CSTAGE;                  // NS planes of psi
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(ring + NS * EXY);

    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int xi = x0 + tx, yi = y0 + ty;
    int hx = 0, hy = 0;
    const bool has_halo = t < HALO;
    if (has_halo) halo_coords<R>(t, hx, hy);
    const int cen = (ty + R) * EX + (tx + R);
    const int hof = hy * EX + hx;
    bool bad = false;

    if (t == 0) {
        mbar_init(&bar[0], 1);   // psi stage full
        mbar_init(&bar[1], 1);   // collision buffer 0 full
        mbar_init(&bar[2], 1);   // collision buffer 1 full
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const int nit = (z1 - z0) + 2 * R;
    if (t == 0) issue_plane<R>(&map, stage, &bar[0], wrap1(z0 - R, p.nz), x0, y0, p);
    bool timed_out = false, late = false;
    for (int it = 0; it < nit; ++it) {
        const int zz = wrap1(z0 - R + it, p.nz);
        // each thread's own wait makes the stage visible to it; the vote on
        // a timed-out wait rides on the barrier that publishes psi
        const bool ok = mbar_wait_bounded(&bar[0], (unsigned)it & 1u);
        float *slot = ring + (it % NS) * EXY;
        slot[cen] = psi_from_boxes<R>(stage, tx + R, ty + R, p.rho0, bad);
        if (has_halo) {
            bool dummy = false;
            slot[hof] = psi_from_boxes<R>(stage, hx, hy, p.rho0, dummy);
        }
        if (!__syncthreads_and(ok && !late)) {
            timed_out = true;
            break;
        }
        if (t == 0) {
            // the stages' previous readers are all behind the barrier above;
            // order their generic-proxy reads before the async-proxy writes
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            if (it + 1 < nit)
                issue_plane<R>(&map, stage, &bar[0], wrap1(zz + 1, p.nz), x0, y0, p);
            if (it + 1 >= 2 * R && it + 1 < nit)
                issue_collision_plane(&cmap, ((it + 1) & 1) ? cst1 : cst0, &bar[1 + ((it + 1) & 1)],
                                      wrap1(zz + 1 - R, p.nz), x0, y0, p);
        }
        if (it < 2 * R) continue;
        // ---- collide plane zc = zz - R --------------------------------------
        const int zc = wrap1(zz - R, p.nz);
        const float *pz[2 * R + 1];
#pragma unroll
        for (int k = -R; k <= R; ++k) pz[k + R] = ring + ((it - R + k + NS) % NS) * EXY + cen;
        float F[3];
        force_ring<R, NG, EX>(pz, p, F);
        // a wait that gives up only marks the thread; the block leaves together
        // at the next vote (computing on an incomplete stage meanwhile is
        // harmless: every address stays in bounds)
        const int cb = it & 1;
        late |= !mbar_wait_bounded(&bar[1 + cb], (unsigned)((it - 2 * R) >> 1) & 1u);
        const float *cs = cb ? cst1 : cst0;
        float g[19];
#pragma unroll
        for (int i = 0; i < 19; ++i)
            g[i] = cs[i * (TY * BOXW) + ty * BOXW + (tx + 4 - cvel<19>(i, 0))];
        float out[19];
        collide19(g, F, p, out);
        store19(B, p, xi, yi, zc, out);
    }
    if (__syncthreads_or(timed_out || late)) {
        // a barrier gave up (never expected): record it, give copies still in
        // flight a bounded chance to land, and leave the step
        if (t == 0) {
            atomicAdd(&flags->timeouts, 1ULL);
            for (int k = 0; k < 3; ++k) {
                mbar_wait_bounded(&bar[k], 0u);
                mbar_wait_bounded(&bar[k], 1u);
            }
        }
        return;
    }
    if (bad) atomicMin(&flags->err_step, flags->step);
    finish_step(flags, t);
}

template <int R>
constexpr int smem_bytes() {
    return (19 * box_stride<R>() + 2 * 19 * TY * BOXW + (2 * R + 2) * (TX + 2 * R) * (TY + 2 * R)) *
               4 +
           32;
}

}  // namespace ft

fc::Params fused_params(const lb_ctx *c, const float *W);

// Host: tensor maps over the two (padded) population buffers, box rows for
// R = 1 and R = 2.  Returns false if the driver entry point is unavailable.
bool tma_make_maps(lb_ctx *c) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    for (int b = 0; b < 2; ++b)
        for (int r = 0; r < 3; ++r) {
            // boxes of TY + 2R rows (psi planes, R = 1, 2) and TY rows
            // (collision planes)
            const int rows = r < 2 ? fc::TY + 2 * (r + 1) : fc::TY;
            cuuint64_t dims[3] = {(cuuint64_t)c->g.nxp, (cuuint64_t)c->g.nyp,
                                  (cuuint64_t)c->Q * c->g.nz};
            cuuint64_t strides[2] = {(cuuint64_t)c->g.nxp * 4,
                                     (cuuint64_t)c->g.nxp * c->g.nyp * 4};
            cuuint32_t box[3] = {(cuuint32_t)ft::BOXW, (cuuint32_t)rows, 1};
            cuuint32_t es[3] = {1, 1, 1};
            CUresult res = encode(&c->tmap[b][r], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->f[b],
                                  dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (res != CUDA_SUCCESS) return false;
        }
    return true;
}

cudaError_t f32_fused3d_tma_step(lb_ctx *c, const float *W, int ng) {
    fc::Params p = fused_params(c, W);
    dim3 block(fc::TX, fc::TY);
    dim3 grid(c->g.nx / fc::TX, c->g.ny / fc::TY, (c->g.nz + p.zchunk - 1) / p.zchunk);
    const float *A = (const float *)c->f[c->cur];
    float *B = (float *)c->f[1 - c->cur];
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(ft::k_fused3d_tma<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<1>());
        cudaFuncSetAttribute(ft::k_fused3d_tma<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<1>());
        cudaFuncSetAttribute(ft::k_fused3d_tma<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<1>());
        cudaFuncSetAttribute(ft::k_fused3d_tma<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<2>());
        cudaFuncSetAttribute(ft::k_fused3d_tma<2, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<2>());
        cudaFuncSetAttribute(ft::k_fused3d_tma<2, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<2>());
        cudaFuncSetAttribute(ft::k_fused3d_tma<2, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, ft::smem_bytes<2>());
        attr_done = true;
    }
    const int sm1 = ft::smem_bytes<1>(), sm2 = ft::smem_bytes<2>();
    const CUtensorMap &m1 = c->tmap[c->cur][0], &m2 = c->tmap[c->cur][1];
    const CUtensorMap &mc = c->tmap[c->cur][2];
    (void)A;
    tm_begin(c, LB_KERNEL_FUSED);
    switch (ng) {
        case 1: ft::k_fused3d_tma<1, 1><<<grid, block, sm1, c->stream>>>(m1, mc, B, p, c->flags); break;
        case 2: ft::k_fused3d_tma<1, 2><<<grid, block, sm1, c->stream>>>(m1, mc, B, p, c->flags); break;
        case 3: ft::k_fused3d_tma<1, 3><<<grid, block, sm1, c->stream>>>(m1, mc, B, p, c->flags); break;
        case 4: ft::k_fused3d_tma<2, 4><<<grid, block, sm2, c->stream>>>(m2, mc, B, p, c->flags); break;
        case 5: ft::k_fused3d_tma<2, 5><<<grid, block, sm2, c->stream>>>(m2, mc, B, p, c->flags); break;
        case 6: ft::k_fused3d_tma<2, 6><<<grid, block, sm2, c->stream>>>(m2, mc, B, p, c->flags); break;
        default: ft::k_fused3d_tma<2, 7><<<grid, block, sm2, c->stream>>>(m2, mc, B, p, c->flags); break;
    }
    tm_end(c);
    c->launches += 1;
    c->cur = 1 - c->cur;
    return cudaGetLastError();
}

}  // namespace sclbm
