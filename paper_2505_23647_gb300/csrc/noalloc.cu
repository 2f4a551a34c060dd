// noalloc.cu -- one binary64 lattice-Boltzmann step that allocates nothing.
//
// Some callers cannot allocate device memory where they step a lattice: a
// host framework whose memory pool forbids direct cudaMalloc, a
// latency-critical loop in which an allocation (and the device-wide
// synchronisation cudaMalloc/cudaFree can imply) is not acceptable, or an
// embedding that may only touch buffers it already owns.  lb_step_fp64_static
// serves them: the caller passes the populations in and out as its own
// device buffers, and the one scratch the step needs -- the psi field of the
// lattice plus a few device counters -- lives in the fixed array g_scratch
// below, which every GPU that loads this library keeps until the process
// exits.
//
// The arithmetic is the library's binary64 step (same device functions, same
// rounding order), so results equal lb_step's bit for bit; the populations
// are read and written in the ABI's state layout (post-streaming f_i(x),
// [Q][N]), streaming by push into the separate output buffer.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "kernels.cuh"

namespace sclbm {
namespace {

// psi of up to kMaxNodes nodes, followed by the device counters
constexpr long long kMaxNodes = LB_STATIC_MAX_NODES;
constexpr long long kCounterWords = 8;
static __device__ __align__(256) double g_scratch[kMaxNodes + kCounterWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];   // device address of g_scratch, per device

// Device address of g_scratch on the current device (looked up once per
// device; host code cannot use the symbol itself as a device pointer).  The
// address belongs to the device's primary context: it does not survive
// cudaDeviceReset, after which this entry point must not be used again in
// the process.
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<double *>(g_addr[dev]);
    return cudaSuccess;
}

__global__ void k_static_reset(Flags *fl) {
    fl->err_step = ULLONG_MAX;
    fl->step = 0;
    fl->exp_amb = 0;
    fl->blocks_done = 0;
    fl->timeouts = 0;
}

// n and psi from populations stored in place (f_i(x) at index i*N + s)
template <int D, int Q>
__global__ void k_static_psi(const double *__restrict__ f, double *__restrict__ psi, Geom g,
                             Flags *fl) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        double fi[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fi[i] = f[(long long)i * g.N + s];
        const double n = sum_q<double, Q>(fi);
        psi[s] = psi_of<double>(n, &fl->exp_amb);   // counted, not reported
    }
}

// force, BGK + Guo, push streaming into the output buffer
template <int D, int Q>
__global__ void __launch_bounds__(256) k_static_collide(const double *__restrict__ f,
                                                        double *__restrict__ fo,
                                                        const double *__restrict__ psi, Geom g,
                                                        const PairsF64 P, const ConstsT<double> k) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        double fi[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fi[i] = f[(long long)i * g.N + s];
        const double n = sum_q<double, Q>(fi);
        double acc[3];
        force_acc<double, PairsF64, D>(psi, g, x, y, z, P, acc);
        const double pre = k.mGp * psi[s];
        double F[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int mu = 0; mu < D; ++mu) F[mu] = pre * acc[mu];
        double out[Q];
        collide<double, D, Q, false>(fi, n, n, F, k, out, nullptr, nullptr);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            fo[(long long)i * g.N + site(g, x + cvel<Q>(i, 0), y + cvel<Q>(i, 1), z + cvel<Q>(i, 2))] =
                out[i];
    }
}

}  // namespace
}  // namespace sclbm

extern "C" lb_status lb_step_fp64_static(int lattice, int nx, int ny, int nz, double tau, double G,
                                         int g_convention, int n_pairs, const int *pair_vec,
                                         const double *pair_w, const double *f_in, double *f_out,
                                         void *cuda_stream) {
    using namespace sclbm;
    if (lattice != LB_D2Q9 && lattice != LB_D3Q19) return LB_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == LB_D2Q9 && nz != 1)) return LB_EINVAL;
    const long long N = (long long)nx * ny * nz;
    if (N > kMaxNodes) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "lb_step_fp64_static: %lld nodes exceed the fixed scratch of %lld nodes",
                      N, kMaxNodes);
        lb_set_error_message(msg);
        return LB_EINVAL;
    }
    if (!(tau > 0.5) || !std::isfinite(tau) || !std::isfinite(G)) return LB_EINVAL;
    if (g_convention != LB_G_LITERAL && g_convention != LB_G_TIMES_CS2) return LB_EINVAL;
    if (n_pairs < 1 || n_pairs > LB_MAX_PAIRS || !pair_vec || !pair_w) return LB_EINVAL;
    if (!f_in || !f_out || f_in == f_out) return LB_EINVAL;
    const int D = lattice == LB_D2Q9 ? 2 : 3, Q = lattice == LB_D2Q9 ? 9 : 19;
    PairsF64 P;
    P.npairs = n_pairs;
    P.radius = 0;
    for (int a = 0; a < n_pairs; ++a) {
        for (int c = 0; c < 3; ++c) {
            const int v = pair_vec[3 * a + c];
            if (v < -LB_MAX_RADIUS || v > LB_MAX_RADIUS || (c == 2 && D == 2 && v != 0))
                return LB_EINVAL;
            P.v[a][c] = (signed char)v;
            P.radius = v > P.radius ? v : (-v > P.radius ? -v : P.radius);
        }
        if (!std::isfinite(pair_w[a])) return LB_EINVAL;
        P.w[a] = pair_w[a];
    }
    // collision constants, formed as lb_create forms them
    ConstsT<double> k;
    const double w9[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
    const double w19[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    const double pref = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < 19; ++i) {
        double w = 0.0;
        if (i < Q) {
            const int sq = D == 2 ? cvel<9>(i, 0) * cvel<9>(i, 0) + cvel<9>(i, 1) * cvel<9>(i, 1)
                                  : cvel<19>(i, 0) * cvel<19>(i, 0) + cvel<19>(i, 1) * cvel<19>(i, 1) +
                                        cvel<19>(i, 2) * cvel<19>(i, 2);
            w = D == 2 ? w9[sq] : w19[sq];
        }
        k.w[i] = w;
        k.cw[i] = pref * w;
    }
    k.omega = 1.0 / tau;
    const double Gp = g_convention == LB_G_TIMES_CS2 ? G / 3.0 : G;
    k.mGp = -Gp;
    k.rho0 = 0.0;
    k.kA = 0.0;   // Guo's T = 2 u F (no F^2 term on this entry point)
    Geom g = {nx, ny, nz, N, nx, ny, 0, 0, N};

    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        lb_set_error_message(cudaGetErrorString(e));
        return LB_ECUDA;
    }
    double *psi = scratch;
    Flags *fl = reinterpret_cast<Flags *>(scratch + kMaxNodes);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int gb = grid_for(N);
    k_static_reset<<<1, 1, 0, st>>>(fl);
    if (D == 2) {
        k_static_psi<2, 9><<<gb, 256, 0, st>>>(f_in, psi, g, fl);
        k_static_collide<2, 9><<<gb, 256, 0, st>>>(f_in, f_out, psi, g, P, k);
    } else {
        k_static_psi<3, 19><<<gb, 256, 0, st>>>(f_in, psi, g, fl);
        k_static_collide<3, 19><<<gb, 256, 0, st>>>(f_in, f_out, psi, g, P, k);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        lb_set_error_message(cudaGetErrorString(e));
        return LB_ECUDA;
    }
    return LB_OK;
}
