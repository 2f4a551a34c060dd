// batch2d.cu -- fused single-pass D2Q9 steps in shifted binary32, for one
// lattice or for many independent lattices in one persistent launch.
//
// One launch = one step of every lattice it covers (eqs. lbm, omega_i, f_eq,
// GuoForcing, sc_f).  The unit of work is one warp marching a 32-column
// strip of a lattice over a chunk of rows (march below): each population is
// read once per step in coalesced rows, psi is formed once per node plus four
// halo columns, the stencil force is accumulated row by row in registers and
// a row is collided and written as soon as the two rows above it are known.
// Warps synchronise only with themselves, so there is no block-wide barrier
// in the step.  Forcing stencils are any weights on the 2D groups (1,0),
// (1,1), (2,0), (2,1), (2,2) (E4, E6, E8 and their tuned variants), and the
// pseudopotential is exp(-1/n) or psi_eps (eq. psieps), both per lattice.
//
// Batches (lb_batch_*): the (lattice, strip, row chunk) items of all lattices
// form one table walked by a grid of resident warps, so boxes of uneven size
// share one launch; 64 launches are captured into a CUDA graph and replayed.
// The row-chunk length is picked per batch by lb_batch_tune; it changes the
// schedule only, never what a node computes.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "collide_tiled.cuh"

namespace sclbm {
namespace b2 {

constexpr int R = 2;   // halo of the widest 2D group, (2,2)

// one lattice of a launch
struct Inst {
    float *f[2];        // population buffers [9][nx * ny]
    Flags *flags;
    int nx, ny;
    int cur0;           // buffer holding the state when the launch parity is 0
    float W[5];         // weights of groups (1,0), (1,1), (2,0), (2,1), (2,2)
    float W2[5];        // 2 W
    float mGp, rho0, keep;
    // collision constants per velocity class |xi|^2 = 0, 1, 2 (D2Q9 weights
    // 4/9, 1/9, 1/36; cw = (1 - 1/(2 tau)) w): omega w, -3 cw, 4.5 omega w,
    // 3 omega w, 9 cw, 3 cw
    float omw[3], m3cw[3], b45[3], d3[3], c9[3], c3[3];
    float M1, M2;       // row sums of the weights at |d| = 1, 2 (M2 doubled)
    float eps, inv_eps; // psi_eps: eps and RN(1/eps) (0 for psi = exp(-1/n))
    // F^2 variant (T = 2 u F - (A/tau) F F): -kA/2 and, per class, -4.5 cw kA
    // (kA = A/tau; all 0 for Guo's T = 2 u F)
    float mhkA, kq[3];
};

// one work item of a batch: rows [y0, y1) of the strip [x0, x0 + 32) of lattice inst
struct Tile {
    int inst, x0, y0, y1;
};

// Halo gather: lane l pulls population SLOT_POP[l >> 2] of halo column l & 3.
// Xor-shuffles over 4, 8 and 16 lanes then add the slots in pairs (1,3),
// (2,4), (5,7), (6,8), their pairs and the two halves -- dens9's tree, so the
// halo density equals the one the owning strip forms, bit for bit.
constexpr int SLOT_POP[8] = {1, 3, 2, 4, 5, 7, 6, 8};

__host__ __device__ constexpr unsigned slot_pack(int mu) {   // mu < 0: the population
    unsigned v = 0;
    for (int s = 0; s < 8; ++s)
        v |= mu < 0 ? (unsigned)SLOT_POP[s] << (4 * s)
                    : (unsigned)(cvel<9>(SLOT_POP[s], mu) + 1) << (2 * s);
    return v;
}
constexpr unsigned SLOT_P = slot_pack(-1), SLOT_X = slot_pack(0), SLOT_Y = slot_pack(1);

// shifted density: opposite pairs first (1,3), (2,4), (5,7), (6,8)
__device__ __forceinline__ float dens9(const float *g) {
    return g[0] + (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
}

// BGK + Guo of one D2Q9 node in shifted binary32, the even/odd split of
// fc::collide19: for a pair (xi, -xi) of class weight w,
//   E = omega w (base + 4.5 n (xi.u)^2) + cw (9 (xi.u)(xi.F) - 3 u.F)
//   O = 3 omega w n (xi.u) + 3 cw (xi.F),  out(+-xi) = (1 - omega) g(+-xi) + E +- O.
// F2: the F^2 variant's extra source -cw kA (4.5 (xi.F)^2 - 1.5 F.F) (Sec. VI),
// its F.F part folded into u.F and its (xi.F)^2 part added to E.
template <bool F2>
__device__ __forceinline__ void collide9(const float *g, float dn, float Fx, float Fy,
                                         const Inst &I, float *out) {
    const float n = dn + I.rho0;
    const float inv = __frcp_rn(n);
    const float d13 = g[1] - g[3], d24 = g[2] - g[4], d57 = g[5] - g[7], d68 = g[6] - g[8];
    const float jx = d13 + (d57 - d68);
    const float jy = d24 + (d57 + d68);
    const float ux = fmaf(0.5f, Fx, jx) * inv;
    const float uy = fmaf(0.5f, Fy, jy) * inv;
    const float uu = fmaf(ux, ux, uy * uy);
    float uF = fmaf(ux, Fx, uy * Fy);
    if constexpr (F2) uF = fmaf(I.mhkA, fmaf(Fx, Fx, Fy * Fy), uF);
    const float base = fmaf(-1.5f * n, uu, dn);
    out[0] = fmaf(I.keep, g[0], fmaf(I.omw[0], base, I.m3cw[0] * uF));
    const float a1 = fmaf(I.omw[1], base, I.m3cw[1] * uF);
    const float a2 = fmaf(I.omw[2], base, I.m3cw[2] * uF);
    const float b1 = I.b45[1] * n, b2 = I.b45[2] * n;
    const float e1 = I.d3[1] * n, e2 = I.d3[2] * n;
#define SCLBM_PAIR9(P, M, C, CU, CF)                                            \
    {                                                                           \
        const float cu = (CU), cF = (CF);                                       \
        float aq = a##C;                                                        \
        if constexpr (F2) aq = fmaf(cF, I.kq[C] * cF, aq);                      \
        const float ev = fmaf(cu, fmaf(b##C, cu, I.c9[C] * cF), aq);            \
        const float od = fmaf(e##C, cu, I.c3[C] * cF);                          \
        out[P] = fmaf(I.keep, g[P], ev + od);                                   \
        out[M] = fmaf(I.keep, g[M], ev - od);                                   \
    }
    SCLBM_PAIR9(1, 3, 1, ux, Fx)
    SCLBM_PAIR9(2, 4, 1, uy, Fy)
    SCLBM_PAIR9(5, 7, 2, ux + uy, Fx + Fy)
    SCLBM_PAIR9(6, 8, 2, uy - ux, Fy - Fx)
#undef SCLBM_PAIR9
}

// One warp marches rows y0 - 2 .. y1 + 1 of the 32-column strip [x0, x0 + 32)
// of lattice I and collides rows y0 .. y1 - 1.  Per row r: the lanes pull the
// row's populations f_i(x, r) = A_i(x - xi_i, r - xi_iy) (coalesced rows),
// form n and psi of their node, gather n of the halo columns x0 - 2, x0 - 1,
// x0 + 32, x0 + 33 (one load per lane, see SLOT_POP), put psi into the
// warp's row buffer, and add row r's share of the force to the five target
// rows r - 2 .. r + 2 it touches: with in-row sums X1 = psi(x+1) - psi(x-1),
// X2 = psi(x+2) - psi(x-2) and S1, S2 the pair sums relative to psi(x),
//   F_x(t) += W(1+d^2) X1 + 2 W(4+d^2) X2,  F_y(t) += d (W(1+d^2) S1 + W(4+d^2) S2)
// for d = r - t, plus (once per target) sum_d d M_d (psi(x, t+d) - psi(x, t-d))
// with M_d = sum over the row of W(dx^2 + d^2) -- the exact form of eq. sc_f
// for the 2D groups up to (2,2).  Row r - 2 is then complete: it is collided
// from the populations the lane has held since it pulled them, and written.
// Periodic wrap: the source columns of a lane are fixed for the march and
// the three source rows advance by one row offset per row, so no load
// computes a wrap.  Sizes that are not multiples of 32: lanes past the edge
// work on the periodic image and store nothing.  Offsets are 32-bit
// (9 nx ny < 2^31, checked when the path is chosen).  EPS: psi_eps instead
// of exp(-1/n); F2: the F^2 forcing variant in the collision.
template <bool EPS, bool F2>
__device__ __forceinline__ void march(const Inst &I, int x0, int y0, int y1, int parity,
                                      float *row, int lane) {
    const int nx = I.nx, ny = I.ny, N = nx * ny;
    const int cur = I.cur0 ^ parity;
    const float *__restrict__ A = I.f[cur];
    float *__restrict__ B = I.f[cur ^ 1];
    const int gx = x0 + lane;
    const bool xown = gx < nx;
    const int x = gx % nx;
    int cs[3];                         // source column x - c for c = -1, 0, 1
    cs[0] = x + 1 == nx ? 0 : x + 1;
    cs[1] = x;
    cs[2] = x == 0 ? nx - 1 : x - 1;
    // the lane's halo load: population hp of column hc
    const int slot = lane >> 2, hcol = lane & 3;
    int hc = (hcol < 2 ? x0 - 2 + hcol : x0 + 30 + hcol) % nx;
    hc += hc < 0 ? nx : 0;
    const int hp = (int)((SLOT_P >> (4 * slot)) & 15u);
    const int hcx = (int)((SLOT_X >> (2 * slot)) & 3u) - 1, hcy = (int)((SLOT_Y >> (2 * slot)) & 3u) - 1;
    int hs = hc - hcx;
    hs += hs < 0 ? nx : 0;
    hs -= hs >= nx ? nx : 0;
    const int hoff = hp * N + hs;
    const int hpos = lane < 2 ? lane : lane + 32;   // lanes 0..3: columns x0-2, x0-1, x0+32, x0+33
    // offsets of the source rows r + 1, r, r - 1 of the row being pulled
    int rr[3];
    {
        int r = y0 - 2;
        r += r < 0 ? ny : 0;
        rr[1] = r * nx;
        rr[0] = (r + 1 == ny ? 0 : r + 1) * nx;
        rr[2] = (r == 0 ? ny - 1 : r - 1) * nx;
    }
    float gq[3][9], dq[3];
    float ps[5], ax[5], ay[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) ps[k] = ax[k] = ay[k] = 0.f;
    bool bad = false;
    const int nit = (y1 - y0) + 4;
    // the next row's populations are in flight while this row is computed
    float gn[9], hn = 0.f, hn0 = 0.f;
    int colN[9];                       // population and source-column part of each load
#pragma unroll
    for (int i = 0; i < 9; ++i) colN[i] = i * N + cs[cvel<9>(i, 0) + 1];
    auto pull = [&]() {
        const float *Ar[3] = {A + rr[0], A + rr[1], A + rr[2]};   // the three source rows
#pragma unroll
        for (int i = 0; i < 9; ++i)
            gn[i] = __ldg(Ar[cvel<9>(i, 1) + 1] + colN[i]);
        hn = __ldg(A + (hoff + (hcy == 0 ? rr[1] : (hcy < 0 ? rr[0] : rr[2]))));
        if (lane < 4) hn0 = __ldg(A + (rr[1] + hc));
    };
    pull();
    int ot = y0 * nx;                  // offset of the next row to be written
    for (int it = 0; it < nit; ++it) {
        const float h1 = hn, h0 = hn0;
#pragma unroll
        for (int i = 0; i < 9; ++i) gq[2][i] = gn[i];
        if (it + 1 < nit) {
            rr[2] = rr[1];
            rr[1] = rr[0];
            rr[0] += nx;
            rr[0] = rr[0] == N ? 0 : rr[0];
            pull();
        }
        dq[2] = dens9(gq[2]);
        const float n = dq[2] + I.rho0;
        bad |= xown && it >= 2 && it < nit - 2 && !(n > 0.f);
        ps[4] = fc::psi_fused<EPS>(n, I.eps, I.inv_eps);
        float hsum = h1 + __shfl_xor_sync(0xffffffffu, h1, 4);
        hsum += __shfl_xor_sync(0xffffffffu, hsum, 8);
        hsum += __shfl_xor_sync(0xffffffffu, hsum, 16);
        float psh = 0.f;
        if (lane < 4) psh = fc::psi_fused<EPS>((h0 + hsum) + I.rho0, I.eps, I.inv_eps);
        __syncwarp();   // the previous row's readers are done
        row[lane + 2] = ps[4];
        if (lane < 4) row[hpos] = psh;
        __syncwarp();
        const float s0 = ps[4];
        const float p1 = row[lane + 3], m1 = row[lane + 1], p2 = row[lane + 4], m2 = row[lane];
        const float X1 = p1 - m1, X2 = p2 - m2;
        const float S1 = (p1 - s0) + (m1 - s0), S2 = (p2 - s0) + (m2 - s0);
        const float cx0 = fmaf(I.W2[2], X2, I.W[0] * X1);
        const float cx1 = fmaf(I.W2[3], X2, I.W[1] * X1);
        const float cx2 = fmaf(I.W2[4], X2, I.W[3] * X1);
        const float cz1 = fmaf(I.W[3], S2, I.W[1] * S1);
        const float cz2 = fmaf(I.W2[4], S2, I.W2[3] * S1);   // carries |d| = 2
        ax[0] += cx2;
        ay[0] += cz2;
        ax[1] += cx1;
        ay[1] += cz1;
        ax[2] += cx0;
        ax[3] += cx1;
        ay[3] -= cz1;
        ax[4] += cx2;
        ay[4] -= cz2;
        if (it >= 4) {   // row t = y0 - 4 + it is complete
            float fy = fmaf(I.M1, ps[3] - ps[1], ay[0]);
            fy = fmaf(I.M2, ps[4] - ps[0], fy);
            const float pre = I.mGp * ps[2];
            float out[9];
            collide9<F2>(gq[0], dq[0], pre * ax[0], pre * fy, I, out);
            if (xown) {
                float *dst = B + (ot + x);
#pragma unroll
                for (int i = 0; i < 9; ++i) __stwb(dst + i * N, out[i]);
            }
            ot += nx;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ps[k] = ps[k + 1];
            ax[k] = ax[k + 1];
            ay[k] = ay[k + 1];
        }
        ax[4] = ay[4] = 0.f;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            dq[r] = dq[r + 1];
#pragma unroll
            for (int i = 0; i < 9; ++i) gq[r][i] = gq[r + 1][i];
        }
    }
    // n <= 0 or NaN: one report per warp, none once the step is recorded (an
    // unstable lattice must not turn every node into an atomic)
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m && lane == __ffs(m) - 1) {
        const unsigned long long step = I.flags->step;
        if (I.flags->err_step > step) atomicMin(&I.flags->err_step, step);
    }
}

// march modes: bit 0 psi_eps, bit 1 the F^2 forcing variant; MIXED picks
// per lattice (a batch whose lattices differ in either)
constexpr int MIXED = 4;

__host__ __device__ inline int inst_mode(const Inst &I) {
    return (I.inv_eps != 0.f ? 1 : 0) | (I.mhkA != 0.f ? 2 : 0);
}

template <int MODE>
__device__ __forceinline__ void march_mode(const Inst &I, int x0, int y0, int y1, int parity,
                                           float *row, int lane) {
    if constexpr (MODE != MIXED) {
        march<(MODE & 1) != 0, (MODE & 2) != 0>(I, x0, y0, y1, parity, row, lane);
    } else {
        switch (inst_mode(I)) {
            case 0: march<false, false>(I, x0, y0, y1, parity, row, lane); break;
            case 1: march<true, false>(I, x0, y0, y1, parity, row, lane); break;
            case 2: march<false, true>(I, x0, y0, y1, parity, row, lane); break;
            default: march<true, true>(I, x0, y0, y1, parity, row, lane); break;
        }
    }
}

constexpr int WPB = 8;   // warps (strips) per block

// one lattice: warp k of the grid marches strip k % nstrips, row chunk
// k / nstrips; the last block advances the step counter
template <int MODE>
__global__ void __launch_bounds__(WPB * 32, 2) k_strip2d(const Inst I, int rows, int parity) {
    __shared__ float buf[WPB][32 + 2 * R];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nstrips = (I.nx + 31) / 32;
    const int k = blockIdx.x * WPB + w;
    const int y0 = (k / nstrips) * rows;
    if (y0 < I.ny)
        march_mode<MODE>(I, (k % nstrips) * 32, y0, min(y0 + rows, I.ny), parity, buf[w], lane);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&I.flags->blocks_done, 1ULL) == (unsigned long long)gridDim.x - 1) {
            I.flags->blocks_done = 0;
            I.flags->step = I.flags->step + 1;
        }
    }
}

// many lattices: a resident grid of warps walks the table of (lattice,
// strip, row chunk) items, dealt round-robin over the blocks first (item k
// to block k mod grid) so that a table shorter than the grid's warps still
// spreads over every block; the last block advances every lattice's counter
template <int MODE>
__global__ void __launch_bounds__(WPB * 32, 2) k_strip2d_batch(const Inst *__restrict__ insts,
                                                            const Tile *__restrict__ items,
                                                            int nitems, int ninst, int parity,
                                                            unsigned long long *done) {
    __shared__ float buf[WPB][32 + 2 * R];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w * gridDim.x + blockIdx.x; k < nitems; k += gridDim.x * WPB) {
        const Tile it = items[k];
        march_mode<MODE>(insts[it.inst], it.x0, it.y0, it.y1, parity, buf[w], lane);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1ULL) == gridDim.x - 1) {
            *done = 0;
            for (int i = 0; i < ninst; ++i) insts[i].flags->step = insts[i].flags->step + 1;
        }
    }
}

// work shapes lb_batch_tune chooses from: 32-column strips, row chunks of
// SHAPE_TY rows (shorter chunks balance better, longer ones repeat fewer
// warm-up rows)
constexpr int NSHAPE = 5;
constexpr int SHAPE_TX[NSHAPE] = {32, 32, 32, 32, 32};
constexpr int SHAPE_TY[NSHAPE] = {16, 8, 32, 64, 128};
constexpr int ROWS_ONE = 16;   // row chunk of a single lattice

void launch_one(const Inst &I, int parity, cudaStream_t st) {
    const int items = ((I.nx + 31) / 32) * ((I.ny + ROWS_ONE - 1) / ROWS_ONE);
    const int g = (items + WPB - 1) / WPB;
    switch (inst_mode(I)) {
        case 0: k_strip2d<0><<<g, WPB * 32, 0, st>>>(I, ROWS_ONE, parity); break;
        case 1: k_strip2d<1><<<g, WPB * 32, 0, st>>>(I, ROWS_ONE, parity); break;
        case 2: k_strip2d<2><<<g, WPB * 32, 0, st>>>(I, ROWS_ONE, parity); break;
        default: k_strip2d<3><<<g, WPB * 32, 0, st>>>(I, ROWS_ONE, parity); break;
    }
}

// the batch kernel of a mode (0..3: every lattice alike, MIXED)
using BatchKernel = void (*)(const Inst *, const Tile *, int, int, int, unsigned long long *);
inline BatchKernel batch_kernel(int mode) {
    switch (mode) {
        case 0: return k_strip2d_batch<0>;
        case 1: return k_strip2d_batch<1>;
        case 2: return k_strip2d_batch<2>;
        case 3: return k_strip2d_batch<3>;
        default: return k_strip2d_batch<MIXED>;
    }
}

void launch_batch_shape(int mode, const Inst *insts, const Tile *items, int nitems, int ninst,
                        int parity, unsigned long long *done, int grid, cudaStream_t st) {
    batch_kernel(mode)<<<grid, WPB * 32, 0, st>>>(insts, items, nitems, ninst, parity, done);
}

// blocks of the batch kernel of a mode resident on the whole GPU
int resident_grid(int mode) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel(mode), WPB * 32, 0) !=
            cudaSuccess || per < 1)
        per = 1;
    return (sms > 0 ? sms : 1) * per;
}

}  // namespace b2

// The 2D fused path applies to a shifted-binary32 D2Q9 context whose
// stencil uses only the five 2D groups up to (2,2).
bool fused2d_applicable(const lb_ctx *c, float *W5) {
    if (c->p.precision != LB_FP32_SHIFTED || c->Q != 9)
        return false;
    if (c->g.nx < 4 || c->g.ny < 4) return false;
    if ((long long)9 * c->g.N >= (1LL << 31)) return false;
    static const int bases[5][2] = {{1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
    for (int q = 0; q < 5; ++q) W5[q] = 0.f;
    for (int gq = 0; gq < c->n_groups; ++gq) {
        int found = -1;
        for (int q = 0; q < 5; ++q)
            if (c->group_base[gq][0] == bases[q][0] && c->group_base[gq][1] == bases[q][1]) found = q;
        if (found < 0) return false;
        W5[found] = (float)c->group_w[gq];
    }
    return true;
}

static void inst_from_ctx(const lb_ctx *c, b2::Inst *I) {
    std::memset(I, 0, sizeof *I);
    I->f[0] = (float *)c->f[0];
    I->f[1] = (float *)c->f[1];
    I->flags = c->flags;
    I->nx = c->g.nx;
    I->ny = c->g.ny;
    I->cur0 = c->cur;
    for (int q = 0; q < 5; ++q) {
        I->W[q] = c->fused2d_W[q];
        I->W2[q] = 2.f * c->fused2d_W[q];
    }
    {   // M_d = sum over dx of W(dx^2 + d^2): W(1) + 2 W(2) + 2 W(5), W(4) + 2 W(5) + 2 W(8)
        const double w0 = c->fused2d_W[0], w1 = c->fused2d_W[1], w2 = c->fused2d_W[2];
        const double w3 = c->fused2d_W[3], w4 = c->fused2d_W[4];
        I->M1 = (float)(w0 + 2.0 * w1 + 2.0 * w3);
        I->M2 = (float)(2.0 * (w2 + 2.0 * w3 + 2.0 * w4));
    }
    const double om = c->k.omega;
    I->mGp = (float)c->k.mGp;
    I->rho0 = (float)c->k.rho0;
    I->eps = c->k.psi_kind == LB_PSI_EPS ? (float)c->k.psi_eps : 0.f;
    I->inv_eps = c->k.psi_kind == LB_PSI_EPS ? (float)c->k.psi_inv : 0.f;
    I->keep = c->k.keep32;
    const double pref = 1.0 - 1.0 / (2.0 * c->p.tau);
    const double wc[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    const double kA = c->k.kA;
    I->mhkA = (float)(-0.5 * kA);
    for (int k = 0; k < 3; ++k) {
        const double cw = pref * wc[k];
        I->kq[k] = (float)(-4.5 * cw * kA);
        I->omw[k] = c->k.omw32[k];   // mass-exact with keep
        I->m3cw[k] = (float)(-3.0 * cw);
        I->b45[k] = (float)(4.5 * om * wc[k]);
        I->d3[k] = (float)(3.0 * om * wc[k]);
        I->c9[k] = (float)(9.0 * cw);
        I->c3[k] = (float)(3.0 * cw);
    }
}

// D2Q9 collision of one node for the generic tiled kernel: the batch
// kernels' pair-symmetric collide9 with the lattice's mass-exact constants
struct Col9 {
    b2::Inst I;
    __device__ __forceinline__ void operator()(const float *fi, float dn, float, const float *F,
                                               float *fo) const {
        if (I.mhkA != 0.f) b2::collide9<true>(fi, dn, F[0], F[1], I, fo);
        else b2::collide9<false>(fi, dn, F[0], F[1], I, fo);
    }
};

// the generic D2Q9 step's collision (after k_psi_f32 has filled psi)
void f32_collide2d_tiled(lb_ctx *c, const float *A, float *B, const float *psi) {
    Col9 col;
    inst_from_ctx(c, &col.I);
    const dim3 grid((c->g.nx + CT_X - 1) / CT_X, (c->g.ny + CT_Y2 - 1) / CT_Y2, 1);
    k_collide_f32<2, 9><<<grid, dim3(CT_X, CT_Y), ct_box(2) * sizeof(float), c->stream>>>(
        A, B, psi, c->g, c->pfast, consts_as<float>(c->k), col, c->flags);
}

cudaError_t f32_fused2d_step(lb_ctx *c) {
    b2::Inst I;
    inst_from_ctx(c, &I);
    I.cur0 = 0;
    tm_begin(c, LB_KERNEL_FUSED);
    b2::launch_one(I, c->cur, c->stream);
    tm_end(c);
    c->launches += 1;
    c->cur = 1 - c->cur;
    return cudaGetLastError();
}

}  // namespace sclbm

// ---- batches -------------------------------------------------------------------
using namespace sclbm;

struct lb_batch {
    std::vector<lb_ctx *> ctx;
    std::vector<b2::Inst> inst;        // host copy of the instance table
    b2::Inst *d_inst = nullptr;
    bool inst_dirty = true;
    b2::Tile *d_tiles[b2::NSHAPE] = {};
    int ntiles[b2::NSHAPE] = {};
    int grid[b2::NSHAPE] = {};
    int shape = 0;
    int mode = 0;                      // march mode of the batch kernel (b2::MIXED: per lattice)
    unsigned long long *d_done = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t done_ev = nullptr;
    std::vector<cudaEvent_t> ctx_ev;
    cudaGraphExec_t graph = nullptr;
    int graph_shape = -1;
    long long launches = 0;
};

namespace {

constexpr int kGraphSteps = 64;   // steps per graph replay (even: parity returns to 0)

lb_status bfail(cudaError_t e, const char *where) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", where, cudaGetErrorString(e));
    lb_set_error_message(msg);
    return LB_ECUDA;
}

lb_status ensure_tiles(lb_batch *b, int s) {
    if (b->d_tiles[s]) return LB_OK;
    const int TX = b2::SHAPE_TX[s], TY = b2::SHAPE_TY[s];
    std::vector<b2::Tile> t;
    // lattice by lattice, row chunk by row chunk, strips side by side: warps
    // running at the same time share their halo columns in L2
    for (int i = 0; i < (int)b->ctx.size(); ++i)
        for (int y0 = 0; y0 < b->inst[i].ny; y0 += TY)
            for (int x0 = 0; x0 < b->inst[i].nx; x0 += TX)
                t.push_back({i, x0, y0, y0 + TY < b->inst[i].ny ? y0 + TY : b->inst[i].ny});
    cudaError_t e = cudaMalloc(&b->d_tiles[s], t.size() * sizeof(b2::Tile));
    if (e != cudaSuccess) return bfail(e, "lb_batch tile table");
    e = cudaMemcpy(b->d_tiles[s], t.data(), t.size() * sizeof(b2::Tile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(e, "lb_batch tile table");
    b->ntiles[s] = (int)t.size();
    const int g = b2::resident_grid(b->mode), need = (b->ntiles[s] + b2::WPB - 1) / b2::WPB;
    b->grid[s] = g < need ? g : need;
    return LB_OK;
}

// contexts may have been stepped on their own since the last batch call:
// take their current buffers as parity 0
lb_status sync_inst(lb_batch *b) {
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (b->inst[i].cur0 != b->ctx[i]->cur) {
            b->inst[i].cur0 = b->ctx[i]->cur;
            b->inst_dirty = true;
        }
    if (!b->inst_dirty) return LB_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_inst, b->inst.data(), b->inst.size() * sizeof(b2::Inst),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bfail(e, "lb_batch instance table");
    e = cudaStreamSynchronize(b->stream);   // the host copy may change before the next call
    if (e != cudaSuccess) return bfail(e, "lb_batch instance table");
    b->inst_dirty = false;
    return LB_OK;
}

void launch_steps(lb_batch *b, int s, int n) {
    for (int k = 0; k < n; ++k)
        b2::launch_batch_shape(b->mode, b->d_inst, b->d_tiles[s], b->ntiles[s], (int)b->ctx.size(), k & 1,
                               b->d_done, b->grid[s], b->stream);
}

lb_status build_graph(lb_batch *b) {
    if (b->graph && b->graph_shape == b->shape) return LB_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(e, "lb_batch graph capture");
    launch_steps(b, b->shape, kGraphSteps);
    e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return bfail(e, "lb_batch graph capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(e, "lb_batch graph instantiate");
    b->graph_shape = b->shape;
    return LB_OK;
}

// every member's pending work before the batch's, the batch's before theirs
lb_status order_before(lb_batch *b) {
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cudaError_t e = cudaEventRecord(b->ctx_ev[i], b->ctx[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ctx_ev[i], 0);
        if (e != cudaSuccess) return bfail(e, "lb_batch ordering");
    }
    return LB_OK;
}

lb_status order_after(lb_batch *b) {
    cudaError_t e = cudaEventRecord(b->done_ev, b->stream);
    for (size_t i = 0; e == cudaSuccess && i < b->ctx.size(); ++i)
        e = cudaStreamWaitEvent(b->ctx[i]->stream, b->done_ev, 0);
    return e == cudaSuccess ? LB_OK : bfail(e, "lb_batch ordering");
}

void advance_members(lb_batch *b, int n) {
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        lb_ctx *c = b->ctx[i];
        c->steps += n;
        if (n & 1) c->cur = 1 - c->cur;
        b->inst[i].cur0 = c->cur;
    }
    if (n & 1) b->inst_dirty = true;
}

}  // namespace

extern "C" {

lb_status lb_batch_create(lb_ctx *const *ctxs, int n, void *cuda_stream, lb_batch **out) {
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (!ctxs || n < 1) return LB_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return LB_EINVAL;
        if (!ctxs[i]->stencil_set) return LB_ESTATE;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return LB_EINVAL;
        if (!ctxs[i]->fast2d_ok) return LB_EUNSUPPORTED;
    }
    lb_batch *b = new lb_batch();
    auto fail = [&](lb_status s) {
        lb_batch_destroy(b);
        return s;
    };
    b->ctx.assign(ctxs, ctxs + n);
    b->inst.resize(n);
    for (int i = 0; i < n; ++i) inst_from_ctx(ctxs[i], &b->inst[i]);
    b->mode = b2::inst_mode(b->inst[0]);
    for (int i = 1; i < n; ++i)
        if (b2::inst_mode(b->inst[i]) != b->mode) b->mode = b2::MIXED;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(bfail(e, "lb_batch_create stream"));
        b->own_stream = true;
    }
    e = cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming);
    b->ctx_ev.resize(n, nullptr);
    for (int i = 0; e == cudaSuccess && i < n; ++i)
        e = cudaEventCreateWithFlags(&b->ctx_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, n * sizeof(b2::Inst));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_done, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(bfail(e, "lb_batch_create"));
    lb_status s = ensure_tiles(b, 0);
    if (s != LB_OK) return fail(s);
    *out = b;
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch *b) {
    if (!b) return LB_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (int s = 0; s < b2::NSHAPE; ++s) cudaFree(b->d_tiles[s]);
    cudaFree(b->d_inst);
    cudaFree(b->d_done);
    for (cudaEvent_t ev : b->ctx_ev)
        if (ev) cudaEventDestroy(ev);
    if (b->done_ev) cudaEventDestroy(b->done_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch *b, int nsteps) {
    if (!b || nsteps < 0) return LB_EINVAL;
    if (nsteps == 0) return LB_OK;
    lb_status s = order_before(b);
    if (s == LB_OK) s = sync_inst(b);
    if (s == LB_OK) s = ensure_tiles(b, b->shape);
    if (s != LB_OK) return s;
    const int reps = nsteps / kGraphSteps, rest = nsteps % kGraphSteps;
    if (reps) {
        s = build_graph(b);
        if (s != LB_OK) return s;
        for (int r = 0; r < reps; ++r) {
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bfail(e, "lb_batch_step graph launch");
        }
    }
    launch_steps(b, b->shape, rest);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(e, "lb_batch_step");
    b->launches += nsteps;
    advance_members(b, nsteps);
    return order_after(b);
}

lb_status lb_batch_sync(lb_batch *b) {
    if (!b) return LB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(e, "lb_batch_sync");
    lb_status worst = LB_OK;
    for (lb_ctx *c : b->ctx) {
        lb_status s = lb_sync(c);
        if (s != LB_OK && worst == LB_OK) worst = s;
    }
    return worst;
}

long long lb_batch_launches(const lb_batch *b) { return b ? b->launches : -1; }

int lb_batch_tile_count(void) { return b2::NSHAPE; }

lb_status lb_batch_tile_shape(int index, int *tx, int *ty) {
    if (index < 0 || index >= b2::NSHAPE || !tx || !ty) return LB_EINVAL;
    *tx = b2::SHAPE_TX[index];
    *ty = b2::SHAPE_TY[index];
    return LB_OK;
}

lb_status lb_batch_set_tile(lb_batch *b, int index) {
    if (!b || index < 0 || index >= b2::NSHAPE) return LB_EINVAL;
    lb_status s = ensure_tiles(b, index);
    if (s != LB_OK) return s;
    b->shape = index;
    return LB_OK;
}

int lb_batch_get_tile(const lb_batch *b) { return b ? b->shape : -1; }

lb_status lb_batch_tune(lb_batch *b, int steps_per_trial, double *ms_out) {
    if (!b || steps_per_trial < 2) return LB_EINVAL;
    const int trial = steps_per_trial & ~1;   // even: every trial ends on parity 0
    lb_status s = order_before(b);
    if (s == LB_OK) s = sync_inst(b);
    if (s != LB_OK) return s;
    // keep the members' states and counters; every trial starts from them
    const size_t n = b->ctx.size();
    std::vector<float *> backup(n, nullptr);
    std::vector<Flags> flags(n);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
        lb_ctx *c = b->ctx[i];
        const size_t bytes = (size_t)9 * c->g.N * sizeof(float);
        e = cudaMalloc(&backup[i], bytes);
        if (e == cudaSuccess) e = cudaMemcpy(backup[i], c->f[c->cur], bytes, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(&flags[i], c->flags, sizeof(Flags), cudaMemcpyDeviceToHost);
    }
    auto restore = [&]() {
        cudaError_t r = cudaStreamSynchronize(b->stream);
        for (size_t i = 0; r == cudaSuccess && i < n; ++i) {
            lb_ctx *c = b->ctx[i];
            r = cudaMemcpy(c->f[c->cur], backup[i], (size_t)9 * c->g.N * sizeof(float),
                           cudaMemcpyDeviceToDevice);
            if (r == cudaSuccess) r = cudaMemcpy(c->flags, &flags[i], sizeof(Flags), cudaMemcpyHostToDevice);
        }
        return r;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e300;
    int best_s = b->shape;
    for (int sh = 0; e == cudaSuccess && sh < b2::NSHAPE; ++sh) {
        s = ensure_tiles(b, sh);
        if (s != LB_OK) break;
        launch_steps(b, sh, 2);   // warm-up
        e = cudaEventRecord(e0, b->stream);
        launch_steps(b, sh, trial);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (ms_out) ms_out[sh] = ms;
        if (e == cudaSuccess && ms < best) {
            best = ms;
            best_s = sh;
        }
        if (e == cudaSuccess) e = restore();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (float *p : backup) cudaFree(p);
    if (s != LB_OK) return s;
    if (e != cudaSuccess) return bfail(e, "lb_batch_tune");
    b->shape = best_s;
    return order_after(b);
}

}  // extern "C"
