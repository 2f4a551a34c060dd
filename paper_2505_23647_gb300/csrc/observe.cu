// observe.cu -- what the library measures on a lattice (compiled with
// -fmad=false like the binary64 step: every binary64 expression rounds as
// written).
//
//  * lb_observables: one fused pass over the populations per call -- mass,
//    momentum sum_x (j + F/2), max |u| and the density extrema, reduced in
//    binary64 by warp shuffles in a fixed order.  Binary64 lattices take
//    every node quantity in binary64 (bit for bit the step's own values);
//    shifted-binary32 lattices take F, u and j + F/2 in binary32 (the
//    step's precision) and only the density, summed from the widened
//    populations, and the global sums in binary64.  Shifted-binary32 D3Q19
//    lattices on the TMA step kernel are measured by that kernel's
//    measuring instantiation (fused3d_tma.cu) instead of k_obs.
//  * the lattice pressure tensor (Appendices E, F) in binary64, the density
//    recomputed from the populations where it is needed;
//  * flat interfaces (Sec. III B, Sec. IV): the profiles of n and of
//    P_N - P_T along x (averaged over y, z) and, per interface window, the
//    line integrals sigma_0 = sum (P_N - P_T) (eq. sigma0pnpt), z_s (first
//    moment, eq. ZSDef), z_e (Gamma(z_e) = 0), delta = z_e - z_s (eq. zemzs)
//    and delta = Gamma(z_s) / (n_l - n_g) (eq. deltaads), in binary64;
//  * a droplet or bubble at rest (Sec. III B, Sec. V B): n_in, n_out, their
//    bulk pressures, the equimolar radius R_e, and the surface of tension
//    R_s with sigma_s = sigma[R_s] from the stationary point of the
//    generalized surface tension sigma[R] along the x axis through the
//    centre, in closed form (below).
//
// No call here allocates device memory: the binary64 fields a call needs
// (psi, the tensor, profiles) are staged in the lattice's second population
// buffer, which holds nothing between steps (every step rewrites all of it),
// and the reduction partials and results in the context's reduction buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "kernels.cuh"

namespace sclbm {

// warp tree, then the warps' results in one warp (block of 256 threads)
__device__ __forceinline__ Red red_block(Red r) {
    __shared__ Red sh[32];
    for (int off = 16; off > 0; off >>= 1) red_combine(r, red_shfl(r, off));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = r;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : red_zero();
        for (int off = 16; off > 0; off >>= 1) red_combine(r, red_shfl(r, off));
    }
    return r;
}

// Error-free binary32 sum of the Q populations: the pairwise rounding errors
// (two_sum) are kept and added back in binary64, so n is the widened sum to
// about 2^-47 relative at a fraction of the cost of 18 binary64 additions.
template <int Q>
__device__ __forceinline__ double sum_q_exactish(const float *fi) {
    float s = fi[0], err = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float t = s + fi[i];
        const float bb = t - s;
        err += (s - (t - bb)) + (fi[i] - bb);
        s = t;
    }
    return (double)s + (double)err;
}

// Index offsets of a node's neighbours that need no periodic wrap: pulled
// populations A_i(x - xi_i) relative to the node's own population index, and
// the stencil's psi neighbours psi(x + e_a) relative to its site index.
struct ObsOff {
    int pop[19];
    int nb[MAXP];
    int R;          // nodes at least R from every boundary use the offsets
};

// One pass: per node n (binary64), F from the psi field, u and j + F/2 in the
// context's precision T; accumulated per thread (binary64; compensated for
// binary64 lattices), then per block by warp shuffles.  Block b takes the
// rows (y, z) b, b + NB_OBS, ..., thread t the columns t, t + 256, ...: a
// fixed order, so the result does not depend on timing.
constexpr int NB_OBS = 1024;

template <typename T, typename PairsT, int D, int Q, bool SHIFT>
__global__ void __launch_bounds__(256) k_obs(const T *__restrict__ A, Geom g,
                                             const T *__restrict__ psi, const PairsT P,
                                             const ObsOff off, const PairsFast PF,
                                             const ConstsT<T> k, Red *partial) {
    Red r = red_zero();
    double mass = 0.0, mom[3] = {0.0, 0.0, 0.0};   // binary32 lattices: plain sums
    const int rows = g.ny * g.nz;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = row % g.ny, z = row / g.ny;
        const bool yz_in = y >= off.R && y < g.ny - off.R &&
                           (D == 2 || (z >= off.R && z < g.nz - off.R));
        const long long prow = ((long long)z * g.nyp + (y + g.oy)) * g.nxp + g.ox;
        for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
            const bool in = yz_in && x >= off.R && x < g.nx - off.R;
            const long long s = (long long)row * g.nx + x;
            T fi[Q];
            if constexpr (SHIFT) {
                pull_f32<D, Q>(A, g, x, y, z, PF, fi);
            } else if (in) {
#pragma unroll
                for (int i = 0; i < Q; ++i) fi[i] = A[(long long)i * g.Np + prow + x - off.pop[i]];
            } else {
                pull<T, D, Q>(A, g, x, y, z, fi);
            }
            const T dn = sum_q<T, Q>(fi);
            const T n = SHIFT ? dn + k.rho0 : dn;
            T acc[3] = {T(0), T(0), T(0)};
            long long sp = s;   // own psi index (halo'd field for binary32)
            if constexpr (SHIFT) {
                sp = psi_at(PF, x, y, z);
                force_fast<D>(psi, (int)sp, PF, acc);
            } else if (in) {
                for (int a = 0; a < P.npairs; ++a) {
                    const T t = P.w[a] * (psi[s + off.nb[a]] - psi[s - off.nb[a]]);
#pragma unroll
                    for (int mu = 0; mu < D; ++mu) {
                        const int c = P.v[a][mu];
                        if (c == 1) acc[mu] = acc[mu] + t;
                        else if (c == -1) acc[mu] = acc[mu] - t;
                        else if (c == 2) acc[mu] = acc[mu] + (t + t);
                        else if (c == -2) acc[mu] = acc[mu] - (t + t);
                        else if (c != 0) acc[mu] = acc[mu] + t * T(c);
                    }
                }
            } else {
                force_acc<T, PairsT, D>(psi, g, x, y, z, P, acc);
            }
            const T pre = k.mGp * psi[sp];
            T F[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int mu = 0; mu < D; ++mu) F[mu] = pre * acc[mu];
            T u[3], m[3];
            collide<T, D, Q, SHIFT>(fi, n, dn, F, k, nullptr, u, m);
            double n64;
            if constexpr (SHIFT) {
                n64 = sum_q_exactish<Q>(fi) + (double)k.rho0;
                mass = mass + n64;
                float uu = u[0] * u[0];
#pragma unroll
                for (int mu = 1; mu < D; ++mu) uu = uu + u[mu] * u[mu];
#pragma unroll
                for (int mu = 0; mu < D; ++mu) mom[mu] = mom[mu] + (double)m[mu];
                r.umax2 = fmax(r.umax2, (double)uu);
            } else {
                n64 = (double)n;
                r.mass = dd_add(r.mass, dd_two_sum(n64, 0.0));
                double uu = (double)u[0] * (double)u[0];
#pragma unroll
                for (int mu = 0; mu < D; ++mu) {
                    if (mu) uu = uu + (double)u[mu] * (double)u[mu];
                    r.mom[mu] = dd_add(r.mom[mu], ddv{(double)m[mu], 0.0});
                }
                r.umax2 = fmax(r.umax2, uu);
            }
            r.rmin = fmin(r.rmin, n64);
            r.rmax = fmax(r.rmax, n64);
        }
    }
    if constexpr (SHIFT) {
        r.mass = ddv{mass, 0.0};
        for (int mu = 0; mu < 3; ++mu) r.mom[mu] = ddv{mom[mu], 0.0};
    }
    r = red_block(r);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void __launch_bounds__(256) k_obs_final(int nb, const Red *__restrict__ partial,
                                                   double *out) {
    Red r = red_zero();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) red_combine(r, partial[b]);
    r = red_block(r);
    if (threadIdx.x == 0) {
        out[0] = r.mass.hi + r.mass.lo;
        for (int k = 0; k < 3; ++k) out[1 + k] = r.mom[k].hi + r.mom[k].lo;
        out[4] = sqrt(r.umax2);
        out[5] = r.rmin;
        out[6] = r.rmax;
    }
}

// device results of obs_fused, after the partials in the reduction buffer
double *obs_results(lb_ctx *c) {
    return reinterpret_cast<double *>(reinterpret_cast<char *>(c->red) + NB_OBS * sizeof(Red));
}

static ObsOff obs_offsets(const lb_ctx *c) {
    ObsOff o;
    const Geom &g = c->g;
    for (int i = 0; i < 19; ++i) {
        const int cx = i < c->Q ? (c->Q == 9 ? cvel<9>(i, 0) : cvel<19>(i, 0)) : 0;
        const int cy = i < c->Q ? (c->Q == 9 ? cvel<9>(i, 1) : cvel<19>(i, 1)) : 0;
        const int cz = i < c->Q ? (c->Q == 9 ? cvel<9>(i, 2) : cvel<19>(i, 2)) : 0;
        o.pop[i] = (cz * g.nyp + cy) * g.nxp + cx;
    }
    int R = 1;
    for (int a = 0; a < MAXP; ++a) {
        if (a >= c->pairs64.npairs) { o.nb[a] = 0; continue; }
        const int ex = c->pairs64.v[a][0], ey = c->pairs64.v[a][1], ez = c->pairs64.v[a][2];
        o.nb[a] = (ez * g.ny + ey) * g.nx + ex;
        const int m = std::max(std::abs(ex), std::max(std::abs(ey), std::abs(ez)));
        R = std::max(R, m);
    }
    o.R = R;
    return o;
}

cudaError_t obs_fused(lb_ctx *c) {
    static_assert(NB_OBS * sizeof(Red) + 64 * sizeof(double) <= 1024 * 128,
                  "reduction buffer too small");
    Red *part = reinterpret_cast<Red *>(c->red);
    double *res = obs_results(c);
    int gb = grid_for(c->g.N);
    if (c->p.precision != LB_FP64 && c->Q == 19 && c->fast3d_ok && c->fused_enabled &&
        c->tma_ok && c->fused_tma) {
        // the fused step kernel's measuring pass: one read of the populations,
        // the force from psi planes in registers; its per-block records go
        // to the idle population buffer
        return f32_fused3d_tma_measure(c, c->f[1 - c->cur], res);
    }
    const ObsOff off = obs_offsets(c);
    if (c->p.precision == LB_FP64) {
        const double *A = (const double *)c->f[c->cur];
        double *psi = (double *)c->psi;
        auto k = consts_as<double>(c->k);
        if (c->Q == 9) {
            k_psi<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, psi, c->g, 0.0, c->flags, psik(c));
            k_obs<double, PairsF64, 2, 9, false><<<NB_OBS, 256, 0, c->stream>>>(A, c->g, psi, c->pairs64, off, c->pfast, k, part);
        } else {
            k_psi<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, psi, c->g, 0.0, c->flags, psik(c));
            k_obs<double, PairsF64, 3, 19, false><<<NB_OBS, 256, 0, c->stream>>>(A, c->g, psi, c->pairs64, off, c->pfast, k, part);
        }
    } else {
        if (!c->psi_halo) return cudaErrorNotSupported;   // beyond 32-bit node indices
        const float *A = (const float *)c->f[c->cur];
        float *psi = (float *)c->psi;
        auto k = consts_as<float>(c->k);
        if (c->Q == 9) {
            k_psi_f32<2, 9><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->pfast, c->flags, psik(c));
            k_obs<float, PairsF32, 2, 9, true><<<NB_OBS, 256, 0, c->stream>>>(A, c->g, psi, c->pairs32, off, c->pfast, k, part);
        } else {
            k_psi_f32<3, 19><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->pfast, c->flags, psik(c));
            k_obs<float, PairsF32, 3, 19, true><<<NB_OBS, 256, 0, c->stream>>>(A, c->g, psi, c->pairs32, off, c->pfast, k, part);
        }
    }
    k_obs_final<<<1, 256, 0, c->stream>>>(NB_OBS, part, res);
    c->launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// binary64 density of one node from a state of either precision
template <typename T, int D, int Q, bool SHIFT>
__device__ __forceinline__ double node_n64(const T *__restrict__ A, const Geom &g, int x, int y,
                                           int z, double rho0) {
    double fi[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i)
        fi[i] = (double)A[(long long)i * g.Np +
                          popidx(g, x - cvel<Q>(i, 0), y - cvel<Q>(i, 1), z - cvel<Q>(i, 2))];
    double n = sum_q<double, Q>(fi);
    if (SHIFT) n = n + rho0;
    return n;
}

// Lattice pressure tensor at one node, components (xx, xy, yy) in 2D and
// (xx, xy, xz, yy, yz, zz) in 3D: n/3 on the diagonal plus, per pair (e, -e),
// s = W (kA A + kB B) e e with the endpoint products A = psi(x) (psi(x+e) +
// psi(x-e)) and the link products B of build_pt_pairs.
template <int D>
__device__ __forceinline__ void pt_node(const Geom &g, int x, int y, int z, double n,
                                        const double *__restrict__ psi, const PTPairs &P,
                                        double *Ps) {
    constexpr int NC = D == 2 ? 3 : 6;
    constexpr int cmu[6] = {0, 0, D == 2 ? 1 : 0, 1, 1, 2};
    constexpr int cnu[6] = {0, 1, D == 2 ? 1 : 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < NC; ++k) Ps[k] = (cmu[k] == cnu[k]) ? n / 3.0 : 0.0;
    const double p0 = psi[site(g, x, y, z)];
    for (int a = 0; a < P.npairs; ++a) {
        const int e0 = P.v[a][0], e1 = P.v[a][1], e2 = P.v[a][2];
        const double Aa = p0 * (psi[site(g, x + e0, y + e1, z + e2)] +
                                psi[site(g, x - e0, y - e1, z - e2)]);
        double B = 0.0;
        for (int l = 0; l < P.nlink[a]; ++l) {
            const signed char *q = &P.link[a][l][0][0];
            B = B + psi[site(g, x + q[0], y + q[1], z + q[2])] *
                        psi[site(g, x + q[3], y + q[4], z + q[5])];
        }
        const double sc = P.w[a] * (P.kA[a] * Aa + P.kB[a] * B);
        const int e[3] = {e0, e1, e2};
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const int ee = e[cmu[k]] * e[cnu[k]];
            if (ee) Ps[k] = Ps[k] + sc * (double)ee;
        }
    }
}

// binary64 psi of every node (the step's psi in binary64 mode)
template <typename T, int D, int Q, bool SHIFT>
__global__ void k_psi64(const T *__restrict__ A, Geom g, double rho0, double *__restrict__ psi,
                        Flags *flags, PsiK pk) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        psi[s] = psi_eval<double>(node_n64<T, D, Q, SHIFT>(A, g, x, y, z, rho0), pk, &flags->exp_amb);
    }
}

template <typename T, int D, int Q, bool SHIFT>
__global__ void __launch_bounds__(128) k_ptensor(const T *__restrict__ A, Geom g, double rho0,
                                                 const double *__restrict__ psi, const PTPairs P,
                                                 double *__restrict__ out) {
    constexpr int NC = D == 2 ? 3 : 6;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        double Ps[NC];
        pt_node<D>(g, x, y, z, node_n64<T, D, Q, SHIFT>(A, g, x, y, z, rho0), psi, P, Ps);
#pragma unroll
        for (int k = 0; k < NC; ++k) out[(long long)k * g.N + s] = Ps[k];
    }
}

// bytes of the second population buffer (staging for binary64 fields)
size_t stage_bytes(const lb_ctx *c) {
    return (size_t)c->Q * c->g.Np * (c->p.precision == LB_FP64 ? 8 : 4);
}
double *stage_ptr(lb_ctx *c) { return (double *)c->f[1 - c->cur]; }

template <typename T, int D, int Q, bool SHIFT>
static void launch_psi64(lb_ctx *c, double *psi) {
    k_psi64<T, D, Q, SHIFT><<<grid_for(c->g.N), 256, 0, c->stream>>>(
        (const T *)c->f[c->cur], c->g, c->k.rho0, psi, c->flags, psik(c));
}

void psi64_field(lb_ctx *c, double *psi) {
    if (c->p.precision == LB_FP64) {
        if (c->Q == 9) launch_psi64<double, 2, 9, false>(c, psi);
        else launch_psi64<double, 3, 19, false>(c, psi);
    } else {
        if (c->Q == 9) launch_psi64<float, 2, 9, true>(c, psi);
        else launch_psi64<float, 3, 19, true>(c, psi);
    }
    c->launches++;
}

// Pressure tensor into out (device, nc x N), psi64 staged at psi (device, N).
cudaError_t ptensor_field(lb_ctx *c, double *psi, double *out) {
    static PTPairs P;   // host staging (large); calls on one context are serialised
    if (!build_pt_pairs(c, &P)) return cudaErrorNotSupported;
    psi64_field(c, psi);
    const int gb = grid_for(c->g.N, 128);
    const double r0 = c->k.rho0;
    if (c->p.precision == LB_FP64) {
        const double *A = (const double *)c->f[c->cur];
        if (c->Q == 9) k_ptensor<double, 2, 9, false><<<gb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, out);
        else k_ptensor<double, 3, 19, false><<<gb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, out);
    } else {
        const float *A = (const float *)c->f[c->cur];
        if (c->Q == 9) k_ptensor<float, 2, 9, true><<<gb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, out);
        else k_ptensor<float, 3, 19, true><<<gb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, out);
    }
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Flat interfaces.  Profiles along x: the means over y, z of n, P^xx and
// P^yy.  Pass 1: block b sums rows [b rpb, (b+1) rpb) of the (y, z) rows,
// thread t the columns x = t, t + blockDim, ... (coalesced), compensated;
// pass 2 adds the blocks' partial sums per column in block order.
template <typename T, int D, int Q, bool SHIFT>
__global__ void __launch_bounds__(128) k_profile_rows(const T *__restrict__ A, Geom g, double rho0,
                                                      const double *__restrict__ psi,
                                                      const PTPairs P, int rows, int rpb,
                                                      double *__restrict__ part, int direct) {
    constexpr int NC = D == 2 ? 3 : 6;
    constexpr int YY = D == 2 ? 2 : 3;
    const int r0 = blockIdx.x * rpb, r1 = min(r0 + rpb, rows);
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
        ddv sn = {0.0, 0.0}, sxx = {0.0, 0.0}, syy = {0.0, 0.0};
        for (int r = r0; r < r1; ++r) {
            const int y = r % g.ny, z = r / g.ny;
            const double n = node_n64<T, D, Q, SHIFT>(A, g, x, y, z, rho0);
            double Ps[NC];
            pt_node<D>(g, x, y, z, n, psi, P, Ps);
            sn = dd_add(sn, ddv{n, 0.0});
            sxx = dd_add(sxx, ddv{Ps[0], 0.0});
            syy = dd_add(syy, ddv{Ps[YY], 0.0});
        }
        if (direct) {   // one block of rows: the means straight into the profiles
            part[x] = (sn.hi + sn.lo) / rows;
            part[g.nx + x] = (sxx.hi + sxx.lo) / rows;
            part[2 * g.nx + x] = (syy.hi + syy.lo) / rows;
        } else {
            double *o = part + ((long long)blockIdx.x * g.nx + x) * 6;
            o[0] = sn.hi; o[1] = sn.lo; o[2] = sxx.hi; o[3] = sxx.lo; o[4] = syy.hi; o[5] = syy.lo;
        }
    }
}

__global__ void k_profile_sum(const double *__restrict__ part, int nb, int nx, double rows,
                              double *__restrict__ prof) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
        ddv s[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        for (int b = 0; b < nb; ++b) {
            const double *o = part + ((long long)b * nx + x) * 6;
            for (int k = 0; k < 3; ++k) s[k] = dd_add(s[k], ddv{o[2 * k], o[2 * k + 1]});
        }
        // means: n, P_N = P^xx, P_T = P^yy
        for (int k = 0; k < 3; ++k) prof[(long long)k * nx + x] = (s[k].hi + s[k].lo) / rows;
    }
}

// Interface windows and their line integrals, one thread (the profile has nx
// values).  An interface lies between x and x + 1 (periodic) where the
// profile crosses the mid density (n_max + n_min)/2; a window runs half way
// to the neighbouring interfaces.  Site x is the cell [x - 1/2, x + 1/2]; n_l
// and n_g are the profile's values at the window's liquid and gas ends; the
// window is oriented from liquid to gas when forming delta.
__global__ void k_flat_windows(const double *__restrict__ prof, int nx, int maxw,
                               lb_flat_obs *out, int *count) {
    if (threadIdx.x || blockIdx.x) return;
    const double *n = prof, *PN = prof + nx, *PT = prof + 2 * nx;
    double lo = n[0], hi = n[0];
    for (int x = 1; x < nx; ++x) {
        lo = fmin(lo, n[x]);
        hi = fmax(hi, n[x]);
    }
    const double mid = 0.5 * (hi + lo);
    auto sgn = [&](int x) { const double d = n[x] - mid; return d > 0.0 ? 1 : (d < 0.0 ? -1 : 0); };
    // interfaces: positions i with a sign change between i and i + 1
    int k = 0;
    for (int i = 0; i < nx; ++i) {
        const int a = sgn(i), b = sgn((i + 1) % nx);
        if (a != b && a != 0 && b != 0) ++k;
    }
    *count = k;
    int q = 0, first = -1, prev = -1;
    // positions in order; window bounds need the previous and next interface
    for (int i = 0; i < nx && q < maxw; ++i) {
        const int a = sgn(i), b = sgn((i + 1) % nx);
        if (!(a != b && a != 0 && b != 0)) continue;
        if (first < 0) first = i;
        // previous interface (the last one for the first), next interface
        int pv = prev, nxt = -1;
        if (pv < 0) {
            for (int j = nx - 1; j > i; --j) {
                const int c0 = sgn(j), c1 = sgn((j + 1) % nx);
                if (c0 != c1 && c0 != 0 && c1 != 0) { pv = j; break; }
            }
            if (pv < 0) pv = i;
        }
        for (int j = i + 1; j < i + 1 + nx; ++j) {
            const int jj = j % nx;
            const int c0 = sgn(jj), c1 = sgn((jj + 1) % nx);
            if (c0 != c1 && c0 != 0 && c1 != 0) { nxt = jj; break; }
        }
        const int gprev = k > 1 ? ((i - pv) % nx + nx) % nx : nx;
        const int gnext = k > 1 ? ((nxt - i) % nx + nx) % nx : nx;
        const int wa = i - gprev / 2 + 1, wb = i + gnext / 2;
        const int rising = b > a;
        double sig = 0.0, mom = 0.0, M = 0.0;
        for (int x = wa; x <= wb; ++x) {
            const int xx = ((x % nx) + nx) % nx;
            const double d = PN[xx] - PT[xx];
            sig = sig + d;
            mom = mom + (double)x * d;
            M = M + n[xx];
        }
        const double zs = mom / sig;
        const double na = n[((wa % nx) + nx) % nx], nb = n[((wb % nx) + nx) % nx];
        double nl, ng, ze, gamma;
        double frac = 0.0;
        if (rising) {   // gas -> liquid along +x
            ng = na;
            nl = nb;
            for (int x = wa; x <= wb; ++x) frac = frac + (n[((x % nx) + nx) % nx] - ng) / (nl - ng);
            ze = ((double)wb + 0.5) - frac;
            gamma = M - ng * (zs - ((double)wa - 0.5)) - nl * (((double)wb + 0.5) - zs);
        } else {        // liquid -> gas along +x
            nl = na;
            ng = nb;
            for (int x = wa; x <= wb; ++x) frac = frac + (n[((x % nx) + nx) % nx] - ng) / (nl - ng);
            ze = ((double)wa - 0.5) + frac;
            gamma = M - nl * (zs - ((double)wa - 0.5)) - ng * (((double)wb + 0.5) - zs);
        }
        const double orient = rising ? -1.0 : 1.0;
        lb_flat_obs r;
        r.sigma = sig;
        r.z_s = zs;
        r.z_e = ze;
        r.delta = orient * (ze - zs);
        r.delta_ads = gamma / (nl - ng);
        r.n_l = nl;
        r.n_g = ng;
        r.window_lo = wa;
        r.window_hi = wb;
        r.rising = rising;
        out[q++] = r;
        prev = i;
    }
}

cudaError_t flat_interfaces(lb_ctx *c, int maxw, lb_flat_obs *out_dev, int *count_dev) {
    return flat_profiles(c, nullptr, maxw, out_dev, count_dev);
}

// The profiles of a slab along x -- means over y (and z) of n, P^xx, P^yy --
// into prof_out (device, [3][nx]; NULL: kept in the staging buffer), and,
// if out_dev, the interface windows and their integrals (k_flat_windows).
cudaError_t flat_profiles(lb_ctx *c, double *prof_out, int maxw, lb_flat_obs *out_dev,
                          int *count_dev) {
    static PTPairs P;
    if (!build_pt_pairs(c, &P)) return cudaErrorNotSupported;
    const long long N = c->g.N;
    const int nx = c->g.nx, rows = c->g.ny * c->g.nz;
    double *psi = stage_ptr(c);
    // staging: psi [N], partials [nb][nx][6] (unless direct), profiles [3][nx]
    const size_t cap = stage_bytes(c) / sizeof(double);
    long long room = (long long)cap - N - 3LL * nx;
    long long nbl = room / (6LL * nx);
    if (nbl > rows) nbl = rows;
    if (nbl > 256) nbl = 256;
    // too little room for partial sums (thin slabs): one block of rows
    // writes the profiles directly
    const int direct = nbl < 2;
    if (direct && room < 0) return cudaErrorInvalidValue;
    int nb = direct ? 1 : (int)nbl;
    const int rpb = (rows + nb - 1) / nb;
    nb = (rows + rpb - 1) / rpb;
    double *part = psi + N, *prof = direct ? part : part + (long long)nb * nx * 6;
    psi64_field(c, psi);
    const double r0 = c->k.rho0;
    if (c->p.precision == LB_FP64) {
        const double *A = (const double *)c->f[c->cur];
        if (c->Q == 9) k_profile_rows<double, 2, 9, false><<<nb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, rows, rpb, part, direct);
        else k_profile_rows<double, 3, 19, false><<<nb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, rows, rpb, part, direct);
    } else {
        const float *A = (const float *)c->f[c->cur];
        if (c->Q == 9) k_profile_rows<float, 2, 9, true><<<nb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, rows, rpb, part, direct);
        else k_profile_rows<float, 3, 19, true><<<nb, 128, 0, c->stream>>>(A, c->g, r0, psi, P, rows, rpb, part, direct);
    }
    if (!direct)
        k_profile_sum<<<(nx + 127) / 128, 128, 0, c->stream>>>(part, nb, nx, (double)rows, prof);
    if (prof_out) {
        cudaError_t e = cudaMemcpyAsync(prof_out, prof, 3 * (size_t)nx * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
    }
    if (out_dev) k_flat_windows<<<1, 1, 0, c->stream>>>(prof, nx, maxw, out_dev, count_dev);
    c->launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A droplet or bubble at rest, centred at (cx, cy[, cz]).
//
// Along the x axis through the centre the site values of P^yy (= P_T there)
// and n are taken on the rows (planes) next to the centre and interpolated
// linearly to the axis; P_T(r) on each ray (+x, -x) is sampled at r = 0, at
// every site with 0 < r < L/2 and at r = L/2, linear between the samples.
// With Delta P = P_in - P_out,
//   sigma[R] = R^(1-d) int_0^{L/2} r^(d-1) (P_J(r; R) - P_T(r)) dr
//            = C R^(1-d) + Delta P R / d,  C = int_0^{L/2} r^(d-1) (P_out - P_T) dr,
// so d sigma/dR = 0 gives R_s^d = d (d-1) C / Delta P and sigma_s =
// Delta P R_s / (d - 1) (eq. ExactLaplace); C is integrated exactly on the
// piecewise-linear P_T, averaged over the two rays.
template <typename T, int D, int Q, bool SHIFT>
__global__ void k_axis_rows(const T *__restrict__ A, Geom g, double rho0,
                            const double *__restrict__ psi, const PTPairs P, int y0, int z0,
                            double *__restrict__ line) {
    constexpr int NC = D == 2 ? 3 : 6;
    constexpr int YY = D == 2 ? 2 : 3;
    const int nrow = D == 2 ? 2 : 4;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nrow * g.nx + 1;
         t += gridDim.x * blockDim.x) {
        int x, y, z;
        if (t == nrow * g.nx) {   // the corner site
            x = y = z = 0;
        } else {
            const int r = t / g.nx;
            x = t % g.nx;
            y = y0 + (r & 1);
            z = D == 3 ? z0 + (r >> 1) : 0;
        }
        const double n = node_n64<T, D, Q, SHIFT>(A, g, x, y, z, rho0);
        double Ps[NC];
        pt_node<D>(g, x, y, z, n, psi, P, Ps);
        line[2 * t] = n;
        line[2 * t + 1] = Ps[YY];
    }
}

struct CurvedIn {
    double cx, cy, cz, Gp, e2, mass;
    int D, nx, ny, nz;
    PsiK pk;
};

// periodic linear interpolation of a site line v[0..nx-1] at x
__device__ double interp_line(const double *v, int nx, double x) {
    double xm = fmod(x, (double)nx);
    if (xm < 0.0) xm += nx;
    const int i = (int)floor(xm);
    const double t = xm - i;
    const double a = v[i % nx], b = v[(i + 1) % nx];
    return a + t * (b - a);
}

// int r^(d-1) (Po - (a + b r)) dr from lo to hi
__device__ double piece(double Po, double a, double b, double lo, double hi, int D) {
    auto F = [&](double t) {
        const double td = D == 2 ? t * t : t * t * t;
        return (Po - a) * td / D - b * td * t / (D + 1);
    };
    return F(hi) - F(lo);
}

__global__ void k_curved(const double *__restrict__ line, CurvedIn in, double *axisbuf,
                         unsigned long long *amb, lb_curved_obs *out) {
    if (threadIdx.x || blockIdx.x) return;
    const int nx = in.nx, D = in.D;
    const int nrow = D == 2 ? 2 : 4;
    const double ty = in.cy - floor(in.cy), tz = D == 3 ? in.cz - floor(in.cz) : 0.0;
    double *nl = axisbuf, *pl = axisbuf + nx;
    for (int x = 0; x < nx; ++x) {
        double sn = 0.0, sp = 0.0;
        for (int r = 0; r < nrow; ++r) {
            const double wy = (r & 1) ? ty : 1.0 - ty;
            const double wz = D == 3 ? ((r >> 1) ? tz : 1.0 - tz) : 1.0;
            const double w = wz * wy;
            if (w == 0.0) continue;
            sn = sn + w * line[2 * (r * nx + x)];
            sp = sp + w * line[2 * (r * nx + x) + 1];
        }
        nl[x] = sn;
        pl[x] = sp;
    }
    const double n_in = interp_line(nl, nx, in.cx);
    const double n_out = line[2 * (nrow * nx)];
    auto Pb = [&](double n) {
        const double ps = psi_eval<double>(n, in.pk, amb);
        return n * (1.0 / 3.0) + 0.5 * in.Gp * in.e2 * (ps * ps);
    };
    const double P_in = Pb(n_in), P_out = Pb(n_out), dP = P_in - P_out;
    const double rmax = 0.5 * nx;
    double C = 0.0;
    for (int ray = 0; ray < 2; ++ray) {
        const double sg = ray ? -1.0 : 1.0;
        // samples: r = 0, the sites at 0 < r < L/2 in increasing r, r = L/2
        double r_prev = 0.0, v_prev = interp_line(pl, nx, in.cx);
        double acc = 0.0;
        // first site beyond the centre along the ray
        double rk = sg > 0 ? floor(in.cx) + 1.0 - in.cx : in.cx - ceil(in.cx) + 1.0;
        if (sg < 0 && in.cx == floor(in.cx)) rk = 1.0;
        if (sg > 0 && rk == 0.0) rk = 1.0;
        for (;; rk += 1.0) {
            const double r = rk < rmax ? rk : rmax;
            const double v = interp_line(pl, nx, in.cx + sg * r);
            const double b = (v - v_prev) / (r - r_prev);
            const double a = v_prev - b * r_prev;
            acc = acc + piece(P_out, a, b, r_prev, r, D);
            r_prev = r;
            v_prev = v;
            if (r >= rmax) break;
        }
        C = C + 0.5 * acc;
    }
    const double Rs = D == 2 ? sqrt(2.0 * C / dP) : cbrt(6.0 * C / dP);
    const double V = (double)in.nx * in.ny * in.nz;
    const double num = in.mass - V * n_out;
    const double pi = 3.141592653589793;
    const double Re = D == 2 ? sqrt(num / (pi * (n_in - n_out)))
                             : cbrt(num / (4.0 / 3.0 * pi * (n_in - n_out)));
    lb_curved_obs o;
    o.n_in = n_in;
    o.n_out = n_out;
    o.P_in = P_in;
    o.P_out = P_out;
    o.dP = dP;
    o.R_e = Re;
    o.R_s = Rs;
    o.sigma_s = dP * Rs / (D - 1);
    o.bubble = n_in < n_out;
    *out = o;
}

cudaError_t curved_interface(lb_ctx *c, const double *center, double e2, lb_curved_obs *out_dev) {
    static PTPairs P;
    if (!build_pt_pairs(c, &P)) return cudaErrorNotSupported;
    // total mass first (the fused observables pass writes it to obs_results)
    cudaError_t e = obs_fused(c);
    if (e != cudaSuccess) return e;
    const long long N = c->g.N;
    const int D = c->D, nx = c->g.nx;
    const int nrow = D == 2 ? 2 : 4;
    double *psi = stage_ptr(c);
    double *line = psi + N, *axisbuf = line + 2LL * (nrow * nx + 1);
    if ((size_t)(N + 2LL * (nrow * nx + 1) + 2LL * nx) > stage_bytes(c) / sizeof(double))
        return cudaErrorInvalidValue;
    psi64_field(c, psi);
    const int y0 = (int)floor(center[1]);
    const int z0 = D == 3 ? (int)floor(center[2]) : 0;
    const int nt = nrow * nx + 1;
    const double r0 = c->k.rho0;
    if (c->p.precision == LB_FP64) {
        const double *A = (const double *)c->f[c->cur];
        if (c->Q == 9) k_axis_rows<double, 2, 9, false><<<(nt + 127) / 128, 128, 0, c->stream>>>(A, c->g, r0, psi, P, y0, z0, line);
        else k_axis_rows<double, 3, 19, false><<<(nt + 127) / 128, 128, 0, c->stream>>>(A, c->g, r0, psi, P, y0, z0, line);
    } else {
        const float *A = (const float *)c->f[c->cur];
        if (c->Q == 9) k_axis_rows<float, 2, 9, true><<<(nt + 127) / 128, 128, 0, c->stream>>>(A, c->g, r0, psi, P, y0, z0, line);
        else k_axis_rows<float, 3, 19, true><<<(nt + 127) / 128, 128, 0, c->stream>>>(A, c->g, r0, psi, P, y0, z0, line);
    }
    // the mass is read on the device from the observables' results
    CurvedIn in;
    in.cx = center[0];
    in.cy = center[1];
    in.cz = D == 3 ? center[2] : 0.0;
    in.Gp = c->Gp;
    in.e2 = e2;
    in.mass = 0.0;
    in.D = D;
    in.nx = nx;
    in.ny = c->g.ny;
    in.nz = c->g.nz;
    in.pk = psik(c);
    double h = 0.0;
    e = cudaMemcpyAsync(&h, obs_results(c), sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    in.mass = h;
    k_curved<<<1, 1, 0, c->stream>>>(line, in, axisbuf, &c->flags->exp_amb, out_dev);
    c->launches += 3;
    return cudaGetLastError();
}

}  // namespace sclbm
