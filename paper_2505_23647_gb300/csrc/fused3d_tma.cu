// fused3d_tma.cu -- the fused single-pass D3Q19 step with TMA staging.
//
// A CTA owns a 32 x 8 column tile and marches a chunk of z planes.  Each
// plane's pulled populations A_i(x - xi_i) (tile plus a radius-R halo) reach
// shared memory through the Tensor Memory Accelerator: one
// cp.async.bulk.tensor per population (19 per plane, issued by one thread,
// completed on an mbarrier) into a double-buffered stage, two planes ahead.
// From the stage each thread forms n and psi (exp(-1/n), or psi_eps of eq.
// psieps in the EPS instantiation) of its node (and of
// a halo node) into a psi plane, keeping its node's 19 pulled populations in
// registers.  The stencil force is accumulated plane by plane in registers
// (plane_force: one pass over a psi plane serves every target plane within
// R), so psi planes never stay in shared memory beyond one step of the
// march; plane z - R is collided as soon as plane z has been added, from the
// populations held since then.
//
// Layout: the population arrays carry periodic ghost columns (images of the
// 8 columns next to each x edge; the interior starts 32 columns into a row
// so that a warp's row of 32 nodes is one 128-byte line) and rows (3 on each
// side in y) around every x-y plane, so the box a tile needs never wraps; the kernel writes a boundary node's values into its
// ghost images as well (fc::store19).  Population i of plane zz is read from
// A_i(x - xi_i): the box of A_i at plane zz - c_z covering rows
// y0 - R - c_y .. y0 + TY + R - c_y and columns x0 - 4 .. x0 + 35 (16-byte
// aligned start); the pull's x/y shift becomes a compile-time offset when the
// box is read.  Requires nx % 32 == 0, ny % 8 == 0.
//
// Every wait on an mbarrier is bounded (Params::max_polls tries, 2^26 by
// default): a block whose wait gives up records a timeout in the device
// counters, lets its copies in flight land, counts itself as finished and
// leaves the step; lb_sync reports LB_ECUDA.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cudaTypedefs.h>

#include "fusedcommon.cuh"

namespace sclbm {

namespace ft {

using namespace fc;

constexpr int BOXW = 40;                  // columns x0 - 4 .. x0 + 35
constexpr long long MAX_POLLS = 1LL << 26;   // default bound of a wait

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

// at most `polls` tries (0: gives up at once; used to test the timeout path)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  long long polls) {
    for (long long k = 0; k < polls; ++k)
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

// order this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
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

// Schedule of one CTA (it = 0 .. nit-1, plane zz = z0 - R + it, stage it & 1):
//   wait stage(it); pulled populations of the own node -> registers, psi of
//   the own and the halo node -> psi plane (it & 1); barrier (+ timeout vote);
//   the issuing thread refills stage(it) with plane zz + 2 (its readers are
//   all behind the barrier); add this plane's force contributions to the
//   2R+1 targets zz - R .. zz + R; collide target zz - R (complete now),
//   store it.
// The psi plane (it & 1) is rewritten at it + 2, after every thread has
// passed the barrier of it + 1, i.e. finished reading it.
//
// MEAS: the measuring instantiation.  The same march over the current state,
// but instead of colliding and storing, each node adds its widened density
// (the binary32 sum of its populations plus that sum's rounding errors), its
// j + F/2 and |u|^2 (formed as collide19 forms them) and its binary32 density
// to per-thread compensated sums and extrema; each block writes one MeasRec
// (binary32 pairs, shifted densities) to B[block].  Nothing else is written
// and the step counter does not move.  (Binary32 pairs, not binary64: this
// GPU's binary64 rate is a small fraction of its binary32 rate, and a
// binary64 tree over every block took longer than the march.)
template <int R, int NG, bool EPS, bool F2, bool MEAS>
__global__ void __launch_bounds__(TX * TY, 2)
    k_fused3d_tma(const __grid_constant__ CUtensorMap map, float *__restrict__ B, const Params p,
                  Flags *flags) {
    constexpr int EX = TX + 2 * R, EY = TY + 2 * R, EXY = EX * EY;
    constexpr int HALO = EXY - TX * TY, HALO_WARPS = (HALO + 31) / 32;
    constexpr int BS = box_stride<R>(), STAGE = 19 * BS;
    constexpr int ISSUER = TX * TY - 1;           // a thread of a warp without halo work
    static_assert(HALO_WARPS < TX * TY / 32, "the issuing warp must have no halo node");
    extern __shared__ __align__(128) float smem[];
    float *stage = smem;                          // two stages of 19 boxes
    float *pbuf = smem + 2 * STAGE;               // two psi planes (tile + halo)
    // bar[0], bar[1]: the stages' copies landed
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(pbuf + 2 * EXY);

    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int xi = x0 + tx, yi = y0 + ty;
    const bool halo_warp = (t >> 5) < HALO_WARPS;   // warp-uniform
    int hx = 0, hy = 0;
    if (halo_warp) halo_coords<R>(min(t, HALO - 1), hx, hy);
    const bool has_halo = t < HALO;
    const int cen = (ty + R) * EX + (tx + R);
    const int hof = hy * EX + hx;
    const int own = (ty + R) * BOXW + tx + 4;     // own node in a box, before the x shift
    const int hbx = hy * BOXW + hx + 4 - R;       // halo node in a box, before the x shift
    bool bad = false;

    if (t == ISSUER) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const int nit = (z1 - z0) + 2 * R;
    // issuing thread only: copies issued on / seen complete by it, per stage
    int issued0 = 0, issued1 = 0, seen0 = 0, seen1 = 0;
    if (t == ISSUER) {
        issue_plane<R>(&map, stage, &bar[0], wrap1(z0 - R, p.nz), x0, y0, p);
        issue_plane<R>(&map, stage + STAGE, &bar[1], wrap1(z0 - R + 1, p.nz), x0, y0, p);
        issued0 = issued1 = 1;
    }
    float gq[R + 1][19];        // pulled populations of planes zz - R .. zz
    float dq[R + 1];            // their shifted densities
    float ps[2 * R + 1];        // own psi of planes zz - 2R .. zz
    float acc[2 * R + 1][3];    // force sums of targets zz - R .. zz + R
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) acc[k][0] = acc[k][1] = acc[k][2] = ps[k] = 0.f;
    bool timed_out = false;
    // MEAS only: compensated sums (value, error) of the shifted density and
    // of j + F/2; the largest |u|^2; the density extrema
    float sm = 0.f, em = 0.f, sx = 0.f, ex = 0.f, sy = 0.f, ey = 0.f, sz = 0.f, ez = 0.f;
    float uu_max = 0.f, n_lo = __int_as_float(0x7f800000), n_hi = -__int_as_float(0x7f800000);

    // unrolled by 2: the stage and psi-plane parity (it & 1) becomes a
    // compile-time constant in each copy (measured 0.8-1.3 % faster; by 4 the
    // code no longer fits the instruction cache, 10 % slower)
#pragma unroll 2
    for (int it = 0; it < nit; ++it) {
        constexpr int PH = R, CS = 0;             // slots of planes zz and zz - R
        const int b = it & 1;
        const bool ok = mbar_wait_bounded(&bar[b], (unsigned)(it >> 1) & 1u, p.max_polls);
        if (t == ISSUER && ok) {
            if (b) seen1 = (it >> 1) + 1;
            else seen0 = (it >> 1) + 1;
        }
        const float *st = stage + b * STAGE;
        float *pb = pbuf + b * EXY;
#pragma unroll
        for (int i = 0; i < 19; ++i) gq[PH][i] = st[i * BS + own - cvel<19>(i, 0)];
        if (halo_warp) {
            // the halo node's chain interleaves with the own node's
            float gh[19];
#pragma unroll
            for (int i = 0; i < 19; ++i) gh[i] = st[i * BS + hbx - cvel<19>(i, 0)];
            dq[PH] = dens(gq[PH]);
            const float n = dq[PH] + p.rho0, nh = dens(gh) + p.rho0;
            bad |= !(n > 0.f);
            ps[2 * R] = psi_fused<EPS>(n, p.eps, p.inv_eps);
            const float psh = psi_fused<EPS>(nh, p.eps, p.inv_eps);
            pb[cen] = ps[2 * R];
            if (has_halo) pb[hof] = psh;
        } else {
            dq[PH] = dens(gq[PH]);
            const float n = dq[PH] + p.rho0;
            bad |= !(n > 0.f);
            ps[2 * R] = psi_fused<EPS>(n, p.eps, p.inv_eps);
            pb[cen] = ps[2 * R];
        }
        if (!__syncthreads_and(ok)) {
            timed_out = true;
            break;
        }
        if (t == ISSUER && it + 2 < nit) {
            // the stage's readers are all behind the barrier above; order
            // their generic-proxy reads before the async-proxy writes
            fence_proxy_async();
            issue_plane<R>(&map, stage + b * STAGE, &bar[b], wrap1(z0 - R + it + 2, p.nz), x0, y0, p);
            if (b) ++issued1;
            else ++issued0;
        }
        {   // this plane's share of the force on targets zz - R .. zz + R
            float cx[R + 1], cy[R + 1], cz[R + 1];
            plane_force<R, NG, EX>(pb + cen, ps[2 * R], p, cx, cy, cz);
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) {
                const int d = R - k, ad = d < 0 ? -d : d;   // plane offset from target
                acc[k][0] += cx[ad];
                acc[k][1] += cy[ad];
                if (d > 0) acc[k][2] += cz[ad];
                if (d < 0) acc[k][2] -= cz[ad];
            }
        }
        if (it >= 2 * R) {   // collide plane zz - R
            float F[3];
            float fz = fmaf(p.M1, ps[R + 1] - ps[R - 1], acc[0][2]);
            if constexpr (R >= 2) fz = fmaf(p.M2, ps[R + 2] - ps[R - 2], fz);
            const float pre = p.mGp * ps[R];
            F[0] = pre * acc[0][0];
            F[1] = pre * acc[0][1];
            F[2] = pre * fz;
            if constexpr (MEAS) {
                float m[3], uu;
                moments19(gq[CS], dq[CS], F, p, m, uu);
                float s = gq[CS][0], e = 0.f;
#pragma unroll
                for (int i = 1; i < 19; ++i) ff_acc(s, e, gq[CS][i]);
                ff_acc(sm, em, s);
                em += e;
                ff_acc(sx, ex, m[0]);
                ff_acc(sy, ey, m[1]);
                ff_acc(sz, ez, m[2]);
                uu_max = fmaxf(uu_max, uu);
                const float n = dq[CS] + p.rho0;
                n_lo = fminf(n_lo, n);
                n_hi = fmaxf(n_hi, n);
            } else {
                float out[19];
                collide19<F2>(gq[CS], dq[CS], F, p, out);
                store19(B, p, xi, yi, z0 - 2 * R + it, out);
            }
        }
        // advance the force and psi windows by one plane
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) {
            acc[k][0] = acc[k + 1][0];
            acc[k][1] = acc[k + 1][1];
            acc[k][2] = acc[k + 1][2];
            ps[k] = ps[k + 1];
        }
        acc[2 * R][0] = acc[2 * R][1] = acc[2 * R][2] = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            dq[r] = dq[r + 1];
#pragma unroll
            for (int i = 0; i < 19; ++i) gq[r][i] = gq[r + 1][i];
        }
    }
    if (__syncthreads_or(timed_out)) {
        // a wait gave up (never expected outside tests that set the bound to
        // zero): record it, let every copy still in flight land so that no
        // transfer touches this CTA's shared memory after it exits, then
        // count the block as finished so the step counter stays consistent
        if (t == ISSUER) {
            atomicAdd(&flags->timeouts, 1ULL);
            for (; seen0 < issued0; ++seen0)
                mbar_wait_bounded(&bar[0], (unsigned)seen0 & 1u, MAX_POLLS);
            for (; seen1 < issued1; ++seen1)
                mbar_wait_bounded(&bar[1], (unsigned)seen1 & 1u, MAX_POLLS);
        }
        if constexpr (MEAS) {
            if (t == 0) {   // a NaN mass marks the measurement as failed
                MeasRec r = meas_zero();
                r.v[0] = __int_as_float(0x7fc00000);
                reinterpret_cast<MeasRec *>(B)[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = r;
            }
        } else {
            finish_step(flags, t);
        }
        return;
    }
    if constexpr (MEAS) {
        // the block's record: warp trees, then the 8 warps' records in warp 0
        MeasRec r;
        meas_pair(r, 0, sm, em);
        meas_pair(r, 2, sx, ex);
        meas_pair(r, 4, sy, ey);
        meas_pair(r, 6, sz, ez);
        r.v[8] = uu_max;
        r.v[9] = n_lo;
        r.v[10] = n_hi;
        meas_warp(r);
        __shared__ MeasRec wred[TX * TY / 32];
        if ((t & 31) == 0) wred[t >> 5] = r;
        __syncthreads();
        if (t < 32) {
            r = t < TX * TY / 32 ? wred[t] : meas_zero();
            meas_warp(r);
            if (t == 0)
                reinterpret_cast<MeasRec *>(B)[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = r;
        }
    } else {
        if (bad) atomicMin(&flags->err_step, flags->step);
        finish_step(flags, t);
    }
}

template <int R>
constexpr int smem_bytes() {
    return (2 * 19 * box_stride<R>() + 2 * (TX + 2 * R) * (TY + 2 * R)) * 4 + 16;
}

template <int R, int NG, bool EPS, bool F2, bool MEAS>
void launch1(dim3 grid, dim3 block, const CUtensorMap &map, float *B, const Params &p, lb_ctx *c) {
    static std::atomic<unsigned long long> attr_done{0};   // devices done, one bit each
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ULL << (dev & 63);
    if (!(attr_done.load() & bit)) {
        cudaFuncSetAttribute(k_fused3d_tma<R, NG, EPS, F2, MEAS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<R>());
        attr_done.fetch_or(bit);
    }
    k_fused3d_tma<R, NG, EPS, F2, MEAS><<<grid, block, smem_bytes<R>(), c->stream>>>(map, B, p, c->flags);
}

// the instantiation for the stencil's widest group (ng = 1..7), the psi kind,
// the forcing variant and step or measurement; m1, m2: the tensor maps with
// boxes of TY + 2 and TY + 4 rows
template <bool EPS, bool F2, bool MEAS = false>
void launch(int ng, dim3 grid, dim3 block, const CUtensorMap &m1, const CUtensorMap &m2, float *B,
            const Params &p, lb_ctx *c) {
    switch (ng) {
        case 1: launch1<1, 1, EPS, F2, MEAS>(grid, block, m1, B, p, c); break;
        case 2: launch1<1, 2, EPS, F2, MEAS>(grid, block, m1, B, p, c); break;
        case 3: launch1<1, 3, EPS, F2, MEAS>(grid, block, m1, B, p, c); break;
        case 4: launch1<2, 4, EPS, F2, MEAS>(grid, block, m2, B, p, c); break;
        case 5: launch1<2, 5, EPS, F2, MEAS>(grid, block, m2, B, p, c); break;
        case 6: launch1<2, 6, EPS, F2, MEAS>(grid, block, m2, B, p, c); break;
        default: launch1<2, 7, EPS, F2, MEAS>(grid, block, m2, B, p, c); break;
    }
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
    // L2 fills promoted to 64 bytes only: a box row starts and ends inside a
    // 128-byte line, and with 256-byte promotion every row edge also pulled
    // the dead padding next to the ghost columns from DRAM (measured at
    // 256^3: 1.74 -> 1.55 GB read per step, the step time unchanged)
    for (int b = 0; b < 2; ++b)
        for (int r = 0; r < 2; ++r) {
            // boxes of TY + 2R rows (R = 1, 2)
            const int rows = fc::TY + 2 * (r + 1);
            cuuint64_t dims[3] = {(cuuint64_t)c->g.nxp, (cuuint64_t)c->g.nyp,
                                  (cuuint64_t)c->Q * c->g.nz};
            cuuint64_t strides[2] = {(cuuint64_t)c->g.nxp * 4,
                                     (cuuint64_t)c->g.nxp * c->g.nyp * 4};
            cuuint32_t box[3] = {(cuuint32_t)ft::BOXW, (cuuint32_t)rows, 1};
            cuuint32_t es[3] = {1, 1, 1};
            CUresult res = encode(&c->tmap[b][r], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->f[b],
                                  dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (res != CUDA_SUCCESS) return false;
        }
    return true;
}

cudaError_t f32_fused3d_tma_step(lb_ctx *c, const float *W, int ng) {
    fc::Params p = fused_params(c, W);
    dim3 block(fc::TX, fc::TY);
    dim3 grid(c->g.nx / fc::TX, c->g.ny / fc::TY, (c->g.nz + p.zchunk - 1) / p.zchunk);
    float *B = (float *)c->f[1 - c->cur];
    const CUtensorMap &m1 = c->tmap[c->cur][0], &m2 = c->tmap[c->cur][1];
    tm_begin(c, LB_KERNEL_FUSED);
    const bool eps = p.inv_eps != 0.f, f2 = c->k.kA != 0.0;
    if (eps && f2)
        ft::launch<true, true>(ng, grid, block, m1, m2, B, p, c);
    else if (eps)
        ft::launch<true, false>(ng, grid, block, m1, m2, B, p, c);
    else if (f2)
        ft::launch<false, true>(ng, grid, block, m1, m2, B, p, c);
    else
        ft::launch<false, false>(ng, grid, block, m1, m2, B, p, c);
    tm_end(c);
    c->launches += 1;
    c->cur = 1 - c->cur;
    return cudaGetLastError();
}

// All blocks' records in one block, then the observables in binary64 (the
// layout of the generic pass's results): mass (plus N rho0), momentum,
// max |u|, min n, max n.
__global__ void __launch_bounds__(256) k_meas_final(int nb, const fc::MeasRec *__restrict__ part,
                                                    double *out, double mass_add) {
    fc::MeasRec r = fc::meas_zero();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) fc::meas_combine(r, part[b]);
    fc::meas_warp(r);
    __shared__ fc::MeasRec wred[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wred[w] = r;
    __syncthreads();
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? wred[lane] : fc::meas_zero();
        fc::meas_warp(r);
        if (lane == 0) {
            out[0] = ((double)r.v[0] + mass_add) + (double)r.v[1];
            for (int k = 0; k < 3; ++k) out[1 + k] = (double)r.v[2 + 2 * k] + (double)r.v[3 + 2 * k];
            out[4] = sqrt((double)r.v[8]);
            out[5] = (double)r.v[9];
            out[6] = (double)r.v[10];
        }
    }
}

// The measuring pass over the current state (the MEAS instantiation; the
// forcing variant does not change n, j + F/2 or u): one record per block
// into part, then k_meas_final into res (7 doubles).
cudaError_t f32_fused3d_tma_measure(lb_ctx *c, void *part, double *res) {
    fc::Params p = fused_params(c, c->fused_W);
    dim3 block(fc::TX, fc::TY);
    dim3 grid(c->g.nx / fc::TX, c->g.ny / fc::TY, (c->g.nz + p.zchunk - 1) / p.zchunk);
    const CUtensorMap &m1 = c->tmap[c->cur][0], &m2 = c->tmap[c->cur][1];
    float *out = (float *)part;
    if (p.inv_eps != 0.f)
        ft::launch<true, false, true>(c->fused_ng, grid, block, m1, m2, out, p, c);
    else
        ft::launch<false, false, true>(c->fused_ng, grid, block, m1, m2, out, p, c);
    const int nb = (int)(grid.x * grid.y * grid.z);
    const double add = (double)c->g.N * (double)p.rho0;
    k_meas_final<<<1, 256, 0, c->stream>>>(nb, (const fc::MeasRec *)part, res, add);
    c->launches += 2;
    return cudaGetLastError();
}

}  // namespace sclbm
