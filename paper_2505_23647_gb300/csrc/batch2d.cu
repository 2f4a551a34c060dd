// batch2d.cu -- fused single-pass D2Q9 steps in shifted binary32, for one
// lattice or for many independent lattices in one persistent launch.
//
// One launch = one step of every lattice it covers (eqs. lbm, omega_i, f_eq,
// GuoForcing, sc_f).  A CTA owns a TX x TY tile: each thread pulls its
// node's populations f_i(x) = A_i(x - xi_i), forms n and psi = exp(-1/n)
// into a shared tile with a radius-2 halo (the halo's psi recomputed from
// populations its neighbours read too, so those loads hit L2), then forms
// the stencil force from the shared tile, collides and writes the node's
// post-collision populations once.  Forcing stencils are any weights on the
// 2D groups (1,0), (1,1), (2,0), (2,1), (2,2) (E4, E6, E8 and their tuned
// variants), per lattice.
//
// Batches (lb_batch_*): the tiles of all lattices form one table; a grid
// sized to the resident CTAs walks it, so boxes of uneven size share one
// launch; K launches are captured into a CUDA graph and replayed.  The tile
// shape is a template parameter picked per batch by lb_batch_tune.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fusedcommon.cuh"

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
    int wide;           // 1 if a radius-2 group has a nonzero weight
};

struct Tile {
    int inst, x0, y0;
};

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// pulled populations of node (x, y): g_i = A_i(x - xi_i), periodic
__device__ __forceinline__ void pull9(const float *__restrict__ A, int N, int nx, int ny, int x,
                                      int y, float *g) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = wrap1(x - cvel<9>(i, 0), nx), sy = wrap1(y - cvel<9>(i, 1), ny);
        g[i] = __ldg(A + (long long)i * N + (long long)sy * nx + sx);
    }
}

// shifted density: opposite pairs first (1,3), (2,4), (5,7), (6,8)
__device__ __forceinline__ float dens9(const float *g) {
    return g[0] + (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
}

// BGK + Guo of one D2Q9 node in shifted binary32, the even/odd split of
// fc::collide19: for a pair (xi, -xi) of class weight w,
//   E = omega w (base + 4.5 n (xi.u)^2) + cw (9 (xi.u)(xi.F) - 3 u.F)
//   O = 3 omega w n (xi.u) + 3 cw (xi.F),  out(+-xi) = (1 - omega) g(+-xi) + E +- O.
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
    const float uF = fmaf(ux, Fx, uy * Fy);
    const float base = fmaf(-1.5f * n, uu, dn);
    out[0] = fmaf(I.keep, g[0], fmaf(I.omw[0], base, I.m3cw[0] * uF));
    const float a1 = fmaf(I.omw[1], base, I.m3cw[1] * uF);
    const float a2 = fmaf(I.omw[2], base, I.m3cw[2] * uF);
    const float b1 = I.b45[1] * n, b2 = I.b45[2] * n;
    const float e1 = I.d3[1] * n, e2 = I.d3[2] * n;
#define SCLBM_PAIR9(P, M, C, CU, CF)                                            \
    {                                                                           \
        const float cu = (CU), cF = (CF);                                       \
        const float ev = fmaf(cu, fmaf(b##C, cu, I.c9[C] * cF), a##C);          \
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

// stencil force sums (eq. sc_f before the -G' psi(x) factor) from the
// shared psi tile around pc (rows EX apart): per in-plane ring
// k = |e|^2 the sums of e_x psi and e_y psi, taken as differences of
// opposite nodes
template <int EX>
__device__ __forceinline__ void force2d(const float *pc, const Inst &I, float &Fx, float &Fy) {
    auto P = [&](int dx, int dy) { return pc[dy * EX + dx]; };
    const float X1 = P(1, 0) - P(-1, 0), Y1 = P(0, 1) - P(0, -1);
    const float a = P(1, 1), b = P(1, -1), c = P(-1, 1), d = P(-1, -1);
    const float X2 = (a - c) + (b - d), Y2 = (a - b) + (c - d);
    Fx = fmaf(I.W[1], X2, I.W[0] * X1);
    Fy = fmaf(I.W[1], Y2, I.W[0] * Y1);
    if (I.wide) {
        const float X4h = P(2, 0) - P(-2, 0), Y4h = P(0, 2) - P(0, -2);
        const float p21 = P(2, 1), p2m = P(2, -1), m21 = P(-2, 1), m2m = P(-2, -1);
        const float p12 = P(1, 2), p1m = P(1, -2), m12 = P(-1, 2), m1m = P(-1, -2);
        const float X5 = fmaf(2.f, (p21 - m21) + (p2m - m2m), (p12 - m12) + (p1m - m1m));
        const float Y5 = fmaf(2.f, (p12 - p1m) + (m12 - m1m), (p21 - p2m) + (m21 - m2m));
        const float q1 = P(2, 2), q2 = P(2, -2), q3 = P(-2, 2), q4 = P(-2, -2);
        const float X8h = (q1 - q3) + (q2 - q4), Y8h = (q1 - q2) + (q3 - q4);
        Fx = fmaf(I.W2[2], X4h, Fx);
        Fy = fmaf(I.W2[2], Y4h, Fy);
        Fx = fmaf(I.W[3], X5, Fx);
        Fy = fmaf(I.W[3], Y5, Fy);
        Fx = fmaf(I.W2[4], X8h, Fx);
        Fy = fmaf(I.W2[4], Y8h, Fy);
    }
}

// halo node h (0 .. EXY - TX*TY - 1) of a TX x TY tile extended by R, in
// extended coordinates: R full rows on top, the side columns, R rows below
template <int TX, int TY>
__device__ __forceinline__ void halo_xy(int h, int &hx, int &hy) {
    constexpr int EX = TX + 2 * R;
    constexpr int top = R * EX, sides = TY * 2 * R;
    if (h < top) {
        hy = h / EX;
        hx = h % EX;
    } else if (h < top + sides) {
        const int k = h - top;
        hy = R + k / (2 * R);
        const int c = k % (2 * R);
        hx = c < R ? c : TX + c;
    } else {
        const int k = h - top - sides;
        hy = R + TY + k / EX;
        hx = k % EX;
    }
}

// One tile of one lattice; ps is the CTA's shared psi tile.  Tiles may run
// past the lattice edge (sizes that are not multiples of the tile): those
// threads work on the periodic image and store nothing.
template <int TX, int TY>
__device__ __forceinline__ void tile_step(const Inst &I, int x0, int y0, int parity, float *ps) {
    constexpr int EX = TX + 2 * R, EY = TY + 2 * R, EXY = EX * EY, NT = TX * TY;
    const int t = threadIdx.x, tx = t % TX, ty = t / TX;
    const int nx = I.nx, ny = I.ny, N = nx * ny;
    const int cur = I.cur0 ^ parity;
    const float *__restrict__ A = I.f[cur];
    float *__restrict__ B = I.f[cur ^ 1];
    const int gx = x0 + tx, gy = y0 + ty;
    const bool owner = gx < nx && gy < ny;
    const int x = gx % nx, y = gy % ny;
    float g[9];
    pull9(A, N, nx, ny, x, y, g);
    const float dn = dens9(g);
    const float n = dn + I.rho0;
    const bool bad = owner && !(n > 0.f);
    const float psi_c = fc::psi32(n);
    ps[(ty + R) * EX + tx + R] = psi_c;
    for (int h = t; h < EXY - NT; h += NT) {
        int hx, hy;
        halo_xy<TX, TY>(h, hx, hy);
        int ax = (x0 + hx - R) % nx, ay = (y0 + hy - R) % ny;
        ax += ax < 0 ? nx : 0;
        ay += ay < 0 ? ny : 0;
        float gh[9];
        pull9(A, N, nx, ny, ax, ay, gh);
        ps[hy * EX + hx] = fc::psi32(dens9(gh) + I.rho0);
    }
    __syncthreads();
    if (owner) {
        float Fx, Fy;
        force2d<EX>(ps + (ty + R) * EX + tx + R, I, Fx, Fy);
        const float pre = I.mGp * psi_c;
        float out[9];
        collide9(g, dn, pre * Fx, pre * Fy, I, out);
        const long long s = (long long)y * nx + x;
#pragma unroll
        for (int i = 0; i < 9; ++i) B[(long long)i * N + s] = out[i];
    }
    // n <= 0 or NaN: one report per warp, none once the step is recorded (an
    // unstable lattice must not turn every node into an atomic)
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m && (t & 31) == __ffs(m) - 1) {
        const unsigned long long step = I.flags->step;
        if (I.flags->err_step > step) atomicMin(&I.flags->err_step, step);
    }
    __syncthreads();   // the next tile reuses ps
}

// one lattice: one CTA per tile; the last CTA advances the step counter
template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_fused2d(const Inst I, int parity) {
    __shared__ float ps[(TX + 2 * R) * (TY + 2 * R)];
    tile_step<TX, TY>(I, blockIdx.x * TX, blockIdx.y * TY, parity, ps);
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&I.flags->blocks_done, 1ULL) == (unsigned long long)gridDim.x * gridDim.y - 1) {
            I.flags->blocks_done = 0;
            I.flags->step = I.flags->step + 1;
        }
    }
}

// many lattices: a resident grid walks the tile table
template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_fused2d_batch(const Inst *__restrict__ insts,
                                                           const Tile *__restrict__ tiles,
                                                           int ntiles, int ninst, int parity,
                                                           unsigned long long *done) {
    __shared__ float ps[(TX + 2 * R) * (TY + 2 * R)];
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = tiles[k];
        tile_step<TX, TY>(insts[tl.inst], tl.x0, tl.y0, parity, ps);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1ULL) == gridDim.x - 1) {
            *done = 0;
            for (int i = 0; i < ninst; ++i) insts[i].flags->step = insts[i].flags->step + 1;
        }
    }
}

// tile shapes lb_batch_tune chooses from
constexpr int NSHAPE = 5;
constexpr int SHAPE_TX[NSHAPE] = {32, 64, 32, 16, 32};
constexpr int SHAPE_TY[NSHAPE] = {8, 4, 16, 16, 4};

template <int S>
void launch_one(const Inst &I, int parity, cudaStream_t st) {
    constexpr int TX = SHAPE_TX[S], TY = SHAPE_TY[S];
    dim3 grid((I.nx + TX - 1) / TX, (I.ny + TY - 1) / TY);
    k_fused2d<TX, TY><<<grid, TX * TY, 0, st>>>(I, parity);
}

template <int S>
void launch_batch(const Inst *insts, const Tile *tiles, int ntiles, int ninst, int parity,
                  unsigned long long *done, int grid, cudaStream_t st) {
    constexpr int TX = SHAPE_TX[S], TY = SHAPE_TY[S];
    k_fused2d_batch<TX, TY><<<grid, TX * TY, 0, st>>>(insts, tiles, ntiles, ninst, parity, done);
}

void launch_batch_shape(int s, const Inst *insts, const Tile *tiles, int ntiles, int ninst,
                        int parity, unsigned long long *done, int grid, cudaStream_t st) {
    switch (s) {
        case 0: launch_batch<0>(insts, tiles, ntiles, ninst, parity, done, grid, st); break;
        case 1: launch_batch<1>(insts, tiles, ntiles, ninst, parity, done, grid, st); break;
        case 2: launch_batch<2>(insts, tiles, ntiles, ninst, parity, done, grid, st); break;
        case 3: launch_batch<3>(insts, tiles, ntiles, ninst, parity, done, grid, st); break;
        default: launch_batch<4>(insts, tiles, ntiles, ninst, parity, done, grid, st); break;
    }
}

int resident_grid(int s) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = SHAPE_TX[s] * SHAPE_TY[s];
    cudaError_t e = cudaSuccess;
    switch (s) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused2d_batch<32, 8>, threads, 0); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused2d_batch<64, 4>, threads, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused2d_batch<32, 16>, threads, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused2d_batch<16, 16>, threads, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused2d_batch<32, 4>, threads, 0); break;
    }
    if (e != cudaSuccess || per < 1) per = 1;
    return (sms > 0 ? sms : 1) * per;
}

}  // namespace b2

// The 2D fused path applies to a shifted-binary32 D2Q9 context whose
// stencil uses only the five 2D groups up to (2,2).
bool fused2d_applicable(const lb_ctx *c, float *W5) {
    if (c->p.precision != LB_FP32_SHIFTED || c->Q != 9 || c->p.psi_kind != LB_PSI_EXP ||
        c->p.forcing_A != 0.0)
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
    I->wide = (c->fused2d_W[2] != 0.f || c->fused2d_W[3] != 0.f || c->fused2d_W[4] != 0.f) ? 1 : 0;
    const double om = c->k.omega;
    I->mGp = (float)c->k.mGp;
    I->rho0 = (float)c->k.rho0;
    I->keep = (float)(1.0 - om);
    const double pref = 1.0 - 1.0 / (2.0 * c->p.tau);
    const double wc[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    for (int k = 0; k < 3; ++k) {
        const double cw = pref * wc[k];
        I->omw[k] = (float)(om * wc[k]);
        I->m3cw[k] = (float)(-3.0 * cw);
        I->b45[k] = (float)(4.5 * om * wc[k]);
        I->d3[k] = (float)(3.0 * om * wc[k]);
        I->c9[k] = (float)(9.0 * cw);
        I->c3[k] = (float)(3.0 * cw);
    }
}

cudaError_t f32_fused2d_step(lb_ctx *c) {
    b2::Inst I;
    inst_from_ctx(c, &I);
    I.cur0 = 0;
    tm_begin(c, LB_KERNEL_FUSED);
    b2::launch_one<0>(I, c->cur, c->stream);
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
    for (int i = 0; i < (int)b->ctx.size(); ++i)
        for (int y0 = 0; y0 < b->inst[i].ny; y0 += TY)
            for (int x0 = 0; x0 < b->inst[i].nx; x0 += TX) t.push_back({i, x0, y0});
    cudaError_t e = cudaMalloc(&b->d_tiles[s], t.size() * sizeof(b2::Tile));
    if (e != cudaSuccess) return bfail(e, "lb_batch tile table");
    e = cudaMemcpy(b->d_tiles[s], t.data(), t.size() * sizeof(b2::Tile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(e, "lb_batch tile table");
    b->ntiles[s] = (int)t.size();
    const int g = b2::resident_grid(s);
    b->grid[s] = g < b->ntiles[s] ? g : b->ntiles[s];
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
        b2::launch_batch_shape(s, b->d_inst, b->d_tiles[s], b->ntiles[s], (int)b->ctx.size(), k & 1,
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
