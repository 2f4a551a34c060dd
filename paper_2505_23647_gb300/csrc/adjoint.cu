// adjoint.cu -- discrete adjoint of the step, in binary64, for gradients of
// what the method is tuned for (surface tension) with respect to the
// forcing-stencil weights, the coupling G and the state.
//
// The step, per node x, from the post-streaming populations g (the state):
//   n = sum g_i, psi = psi(n), acc = sum_pairs W_a (psi(x+e_a) - psi(x-e_a)) e_a,
//   F = -G' psi acc, j = sum g_i xi_i, u = (j + F/2)/n,
//   B_i = g_i - omega (g_i - f_eq_i(n,u)) + S_i(u,F),  g'_i(x + xi_i) = B_i(x)
// (eqs. lbm, omega_i, f_eq, GuoForcing, sc_f; the F^2 variant of Sec. VI
// subtracts cw_i (A/tau)(4.5 (xi.F)^2 - 1.5 F.F) from S_i).  Going backwards through it
// with lam' = dL/dg':
//   lamB_i(x) = lam'_i(x + xi_i);
//   lam_u = sum_i lamB_i (omega df_eq_i/du + dS_i/du), lam_n|u = omega sum_i lamB_i df_eq_i/dn,
//   lam_F|u = sum_i lamB_i dS_i/dF;  through u = (j + F/2)/n:
//   lam_j = lam_u/n, lam_F = lam_F|u + lam_u/(2n), lam_n = lam_n|u - lam_u.u/n;
//   through F: lam_psi(x) += -G' lam_F.acc, lam_acc = -G' psi lam_F,
//   dL/dG' += -psi acc.lam_F; through acc: dL/dW_a += (psi(x+e_a)-psi(x-e_a)) e_a.lam_acc,
//   lam_psi(y) += W_a e_a.(lam_acc(y-e_a) - lam_acc(y+e_a));
//   lam_n += psi'(n) lam_psi;  lam_i = (1-omega) lamB_i + lam_n + xi_i.lam_j.
// Kernel A does everything local to a node, kernel B the psi stencil.
// Parameter gradients accumulate per node (each node owned by one thread,
// no atomics) and are summed in a fixed order when read: results are
// deterministic.  Forward states of a segment are recomputed by the
// context's own step and recorded in the state layout (binary64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace sclbm {
namespace adj {

constexpr int MAXG = 32;   // stencil groups

struct PairGroups {
    int g[LB_MAX_PAIRS];   // group index of each canonical pair
};

template <int Q>
__device__ __forceinline__ double psi_and_dpsi(double n, const PsiK &pk, double &dpsi) {
    double p;
    if (pk.kind == 0) {
        p = exp(-1.0 / n);
        dpsi = p / (n * n);
    } else {
        p = pow(n / (pk.eps + n), pk.inv);
        dpsi = p / (n * (pk.eps + n));
    }
    return p;
}

// n and psi of a state in the state layout
template <int D, int Q>
__global__ void k_adj_fields(const double *__restrict__ st, Geom g, PsiK pk, double *__restrict__ n,
                             double *__restrict__ psi, double *__restrict__ dpsi) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        double v = st[s];
#pragma unroll
        for (int i = 1; i < Q; ++i) v += st[(long long)i * g.N + s];
        double d;
        n[s] = v;
        psi[s] = psi_and_dpsi<Q>(v, pk, d);
        dpsi[s] = d;
    }
}

// everything local to node x; writes lam (partial, without psi'(n) lam_psi),
// lam_acc [D][N], lam_psi [N] (local part) and the per-node gradient terms
template <int D, int Q>
__global__ void k_adj_a(const double *__restrict__ st, const double *__restrict__ n_f,
                        const double *__restrict__ psi, const double *__restrict__ lam_next,
                        Geom g, const PairsF64 P, const PairGroups PG, ConstsT<double> k,
                        double Gp, int ngroups, double *__restrict__ lam_out,
                        double *__restrict__ lacc, double *__restrict__ lpsi,
                        double *__restrict__ gnode) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double om = k.omega, kA = k.kA;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        double gi[Q], lb[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            gi[i] = st[(long long)i * g.N + s];
            lb[i] = lam_next[(long long)i * g.N +
                             site(g, x + cvel<Q>(i, 0), y + cvel<Q>(i, 1), z + cvel<Q>(i, 2))];
        }
        const double n = n_f[s], ps = psi[s];
        double acc[3];
        force_acc<double, PairsF64, D>(psi, g, x, y, z, P, acc);
        double F[3] = {0.0, 0.0, 0.0}, j[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < D; ++a) F[a] = -Gp * ps * acc[a];
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
            for (int a = 0; a < D; ++a) j[a] += cvel<Q>(i, a) * gi[i];
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = (j[a] + 0.5 * F[a]) / n;
        double uu = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) uu += u[a] * u[a];
        double lu[3] = {0.0, 0.0, 0.0}, lF[3] = {0.0, 0.0, 0.0}, ln = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            double cu = 0.0, cF = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                cu += cvel<Q>(i, a) * u[a];
                cF += cvel<Q>(i, a) * F[a];
            }
            const double w = k.w[i], cw = k.cw[i];
            ln += lb[i] * om * w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const double c = cvel<Q>(i, a);
                const double dfeq = w * n * (3.0 * c + 9.0 * cu * c - 3.0 * u[a]);
                const double dSu = cw * (9.0 * cF * c - 3.0 * F[a]);
                double dSF = cw * (3.0 * c + 9.0 * cu * c - 3.0 * u[a]);
                // F^2 variant: S_i gains -cw kA (4.5 cF^2 - 1.5 F.F)
                if (kA != 0.0) dSF -= cw * kA * (9.0 * cF * c - 3.0 * F[a]);
                lu[a] += lb[i] * (om * dfeq + dSu);
                lF[a] += lb[i] * dSF;
            }
        }
        double lj[3] = {0.0, 0.0, 0.0}, la[3] = {0.0, 0.0, 0.0}, lpl = 0.0, gG = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            lj[a] = lu[a] / n;
            lF[a] += lu[a] / (2.0 * n);
            ln -= lu[a] * u[a] / n;
            lpl += -Gp * lF[a] * acc[a];
            la[a] = -Gp * ps * lF[a];
            gG += -ps * acc[a] * lF[a];
            lacc[(long long)a * g.N + s] = la[a];
        }
        lpsi[s] = lpl;
        gnode[(long long)ngroups * g.N + s] += gG;
        for (int a = 0; a < P.npairs; ++a) {
            const int e0 = P.v[a][0], e1 = P.v[a][1], e2 = P.v[a][2];
            const double d = psi[site(g, x + e0, y + e1, z + e2)] - psi[site(g, x - e0, y - e1, z - e2)];
            double ela = e0 * la[0] + e1 * la[1];
            if (D == 3) ela += e2 * la[2];
            gnode[(long long)PG.g[a] * g.N + s] += d * ela;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            double v = (1.0 - om) * lb[i] + ln;
#pragma unroll
            for (int a = 0; a < D; ++a) v += cvel<Q>(i, a) * lj[a];
            lam_out[(long long)i * g.N + s] = v;
        }
    }
}

// the psi stencil: lam_psi(y) += sum W_a e_a.(lam_acc(y - e_a) - lam_acc(y + e_a)),
// then lam_i(y) += psi'(n) lam_psi(y)
template <int D, int Q>
__global__ void k_adj_b(const double *__restrict__ lacc, const double *__restrict__ lpsi,
                        const double *__restrict__ dpsi, Geom g, const PairsF64 P,
                        double *__restrict__ lam_out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        double lp = lpsi[s];
        for (int a = 0; a < P.npairs; ++a) {
            const int e0 = P.v[a][0], e1 = P.v[a][1], e2 = P.v[a][2];
            const long long sm = site(g, x - e0, y - e1, z - e2), sp = site(g, x + e0, y + e1, z + e2);
            double dm = e0 * lacc[sm] + e1 * lacc[g.N + sm];
            double dp = e0 * lacc[sp] + e1 * lacc[g.N + sp];
            if (D == 3) {
                dm += e2 * lacc[2 * g.N + sm];
                dp += e2 * lacc[2 * g.N + sp];
            }
            lp += P.w[a] * (dm - dp);
        }
        const double add = dpsi[s] * lp;
#pragma unroll
        for (int i = 0; i < Q; ++i) lam_out[(long long)i * g.N + s] += add;
    }
}

// sigma_0 of a flat slab (gradients along x): per node h(x) = sum_pairs W k
// (psi(x+e) + psi(x-e)), k = e_x^2 - e_y^2; sigma = G'/(2 n_if) sum psi h;
// seed lam_i = psi'(n) (G'/n_if) h; direct dsigma/dW per node
template <int D, int Q>
__global__ void k_sigma_seed(const double *__restrict__ psi, const double *__restrict__ dpsi,
                             Geom g, const PairsF64 P, const PairGroups PG, double Gp, double inv_nif,
                             int ngroups, double *__restrict__ lam, double *__restrict__ gnode,
                             double *__restrict__ snode) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        const double ps = psi[s];
        double h = 0.0;
        for (int a = 0; a < P.npairs; ++a) {
            const int e0 = P.v[a][0], e1 = P.v[a][1], e2 = P.v[a][2];
            const double kk = (double)(e0 * e0 - e1 * e1);
            if (kk == 0.0) continue;
            const double sm = psi[site(g, x + e0, y + e1, z + e2)] + psi[site(g, x - e0, y - e1, z - e2)];
            h += P.w[a] * kk * sm;
            gnode[(long long)PG.g[a] * g.N + s] += 0.5 * Gp * inv_nif * ps * kk * sm;
        }
        snode[s] = ps * h;
        const double l = dpsi[s] * Gp * inv_nif * h;
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[(long long)i * g.N + s] = l;
    }
}

// fixed-order partial sums of rows of a [rows][N] array: one block per (row, chunk)
__global__ void k_rowsum(const double *__restrict__ a, long long N, int chunks, double *__restrict__ out) {
    const int row = blockIdx.y, ch = blockIdx.x;
    const long long per = (N + chunks - 1) / chunks;
    const long long lo = ch * per, hi = lo + per < N ? lo + per : N;
    __shared__ double sh[256];
    double v = 0.0;
    for (long long s = lo + threadIdx.x; s < hi; s += blockDim.x) v += a[(long long)row * N + s];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[row * chunks + ch] = sh[0];
}

// L = sum_x m(x) (P_xx - P_yy)(x) for given site weights m (the normal and a
// tangential component of the Appendix E/F tensor of a slab with gradients
// along x; n/3 cancels).  Per site x and pair (e, -e), with k = e_x^2 - e_y^2,
// the tensor adds W k (kA psi(x)(psi(x+e) + psi(x-e)) + kB sum_l psi(x+q0) psi(x+q1)),
// so dL/dpsi(y) gathers, over the pair's links through y,
//   W k kA (m(y)(psi(y+e) + psi(y-e)) + m(y-e) psi(y-e) + m(y+e) psi(y+e))
//   + W k kB sum_l (m(y-q0) psi(y-q0+q1) + m(y-q1) psi(y-q1+q0)).
// lam_i(y) += psi'(n) dL/dpsi(y); the site's own terms give L (snode) and
// dL/dW (gnode); dL/dG' = L/G' (every term carries G').
template <int D, int Q>
__global__ void k_seed_pt(const double *__restrict__ psi, const double *__restrict__ dpsi,
                          const double *__restrict__ m, Geom g, const PTPairs P, const PairGroups PG,
                          double *__restrict__ lam, double *__restrict__ gnode,
                          double *__restrict__ snode) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        const double p0 = psi[s], m0 = m[s];
        double gp = 0.0, own = 0.0;
        for (int a = 0; a < P.npairs; ++a) {
            const int e0 = P.v[a][0], e1 = P.v[a][1], e2 = P.v[a][2];
            const double kk = (double)(e0 * e0 - e1 * e1);
            if (kk == 0.0) continue;
            const long long sp = site(g, x + e0, y + e1, z + e2), sm = site(g, x - e0, y - e1, z - e2);
            const double wa = P.w[a] * kk;
            double t = P.kA[a] * (m0 * (psi[sp] + psi[sm]) + m[sm] * psi[sm] + m[sp] * psi[sp]);
            double Bown = 0.0;
            for (int l = 0; l < P.nlink[a]; ++l) {
                const signed char *q = &P.link[a][l][0][0];
                const long long s0 = site(g, x - q[0], y - q[1], z - q[2]);
                const long long s1 = site(g, x - q[3], y - q[4], z - q[5]);
                t += P.kB[a] * (m[s0] * psi[site(g, x - q[0] + q[3], y - q[1] + q[4], z - q[2] + q[5])] +
                                m[s1] * psi[site(g, x - q[3] + q[0], y - q[4] + q[1], z - q[5] + q[2])]);
                Bown += psi[site(g, x + q[0], y + q[1], z + q[2])] * psi[site(g, x + q[3], y + q[4], z + q[5])];
            }
            gp += wa * t;
            const double c = m0 * kk * (P.kA[a] * p0 * (psi[sp] + psi[sm]) + P.kB[a] * Bown);
            own += P.w[a] * c;
            gnode[(long long)PG.g[a] * g.N + s] += c;
        }
        snode[s] = own;
        const double add = dpsi[s] * gp;
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[(long long)i * g.N + s] += add;
    }
}

// Quantity Q of a slab and its per-column derivatives from the profiles
// prof = [n][P^xx][P^yy] (means over y, z; one thread, nx columns):
// gn[x] = dQ/d n(x), gd[x] = dQ/d (P_N - P_T)(x).  Interface windows as in
// lb_flat_interfaces (crossings of the mid density, half way to the
// neighbours); site x is the cell [x - 1/2, x + 1/2]; delta oriented from
// liquid to gas.  val[0] = Q, val[1] = interfaces found.
__global__ void k_flat_seed(const double *__restrict__ prof, int nx, int q, double p0, double p1,
                            double p2, double *__restrict__ gn, double *__restrict__ gd,
                            double *val) {
    if (threadIdx.x || blockIdx.x) return;
    const double *n = prof, *PN = prof + nx, *PT = prof + 2 * nx;
    for (int x = 0; x < nx; ++x) gn[x] = gd[x] = 0.0;
    double lo = n[0], hi = n[0];
    for (int x = 1; x < nx; ++x) {
        lo = fmin(lo, n[x]);
        hi = fmax(hi, n[x]);
    }
    const double mid = 0.5 * (hi + lo);
    auto sgn = [&](int x) { const double d = n[x] - mid; return d > 0.0 ? 1 : (d < 0.0 ? -1 : 0); };
    auto cross = [&](int i) {
        const int a = sgn(i), b = sgn((i + 1) % nx);
        return a != b && a != 0 && b != 0;
    };
    int k = 0, last = -1, first = -1;
    for (int i = 0; i < nx; ++i)
        if (cross(i)) {
            if (first < 0) first = i;
            last = i;
            ++k;
        }
    val[1] = k;
    double Q = 0.0;
    if (q == 0) {             // sigma_0: the whole line's P_N - P_T per interface
        if (k == 0) { val[0] = nan(""); return; }
        for (int x = 0; x < nx; ++x) {
            Q = Q + (PN[x] - PT[x]);
            gd[x] = 1.0 / k;
        }
        val[0] = Q / k;
        return;
    }
    if (q == 1) {             // delta: per interface window
        if (k == 0) { val[0] = nan(""); return; }
        int prev = last;
        for (int i = 0; i < nx; ++i) {
            if (!cross(i)) continue;
            int nxt = i;
            for (int j = i + 1; j < i + 1 + nx; ++j)
                if (cross(j % nx)) { nxt = j % nx; break; }
            const int gp = k > 1 ? ((i - prev) % nx + nx) % nx : nx;
            const int gq = k > 1 ? ((nxt - i) % nx + nx) % nx : nx;
            const int wa = i - gp / 2 + 1, wb = i + gq / 2;
            const bool rising = sgn((i + 1) % nx) > sgn(i);
            prev = i;
            auto at = [&](int x) { return ((x % nx) + nx) % nx; };
            double S = 0.0, mom = 0.0;
            for (int x = wa; x <= wb; ++x) {
                const double d = PN[at(x)] - PT[at(x)];
                S = S + d;
                mom = mom + (double)x * d;
            }
            const double zs = mom / S;
            const int J = wb - wa + 1;
            double sumn = 0.0;
            for (int x = wa; x <= wb; ++x) sumn = sumn + n[at(x)];
            const double na = n[at(wa)], nb = n[at(wb)];
            // z_e and its derivative in the window's densities
            double ze, T, Dl;
            if (rising) {   // gas at wa, liquid at wb
                T = sumn - J * na;
                Dl = nb - na;
                ze = ((double)wb + 0.5) - T / Dl;
            } else {        // liquid at wa, gas at wb
                T = sumn - J * nb;
                Dl = na - nb;
                ze = ((double)wa - 0.5) + T / Dl;
            }
            const double orient = rising ? -1.0 : 1.0;
            Q = Q + orient * (ze - zs);
            for (int x = wa; x <= wb; ++x) {
                const int xx = at(x);
                // dT/dn(x) and dDl/dn(x)
                double dT = 1.0, dD = 0.0;
                if (rising) {
                    if (x == wa) { dT -= J; dD -= 1.0; }
                    if (x == wb) dD += 1.0;
                } else {
                    if (x == wb) { dT -= J; dD -= 1.0; }
                    if (x == wa) dD += 1.0;
                }
                const double dze = (rising ? -1.0 : 1.0) * (dT * Dl - T * dD) / (Dl * Dl);
                gn[xx] += orient * dze;
                gd[xx] += -orient * ((double)x - zs) / S;
            }
        }
        Q = Q / k;
        for (int x = 0; x < nx; ++x) {
            gn[x] /= k;
            gd[x] /= k;
        }
    } else if (q == 2) {      // smooth interface width
        const double nl = p0, ng = p1, ni = p2 > 0.0 ? p2 : (double)k;
        if (!(ni > 0.0)) { val[0] = nan(""); return; }
        const double dl = nl - ng;
        for (int x = 0; x < nx; ++x) {
            Q = Q + (n[x] - ng) * (nl - n[x]);
            gn[x] = 6.0 * (nl + ng - 2.0 * n[x]) / (dl * dl) / ni;
        }
        Q = 6.0 * Q / (dl * dl) / ni;
    } else {                  // density ratio n(x_l) / n(x_g)
        const int xl = (int)p0, xg = (int)p1;
        const double nl = n[xl], ng = n[xg];
        Q = nl / ng;
        gn[xl] += 1.0 / ng;
        gn[xg] += -nl / (ng * ng);
    }
    val[0] = Q;
}

// lam_i(s) += w gn[x(s)] / rows (every i: n = sum_i f_i); m(s) = w gd[x(s)] / rows
__global__ void k_broadcast_seed(double *__restrict__ lam, double *__restrict__ m,
                                 const double *__restrict__ gn, const double *__restrict__ gd,
                                 Geom g, int Q, double w) {
    const double rows = (double)g.ny * g.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        const int x = (int)(s % g.nx);
        const double a = w * gn[x] / rows;
        if (a != 0.0)
            for (int i = 0; i < Q; ++i) lam[(long long)i * g.N + s] += a;
        m[s] = w * gd[x] / rows;
    }
}

}  // namespace adj
}  // namespace sclbm

using namespace sclbm;

struct lb_adjoint {
    lb_ctx *c = nullptr;
    Geom g{};                  // plain state geometry
    int D = 0, Q = 0, ngroups = 0;
    adj::PairGroups pg{};
    double *lam = nullptr, *lam2 = nullptr, *lacc = nullptr, *lpsi = nullptr;
    double *n = nullptr, *psi = nullptr, *dpsi = nullptr;
    double *gnode = nullptr;   // [ngroups + 1][N] per-node gradient terms (last row: G')
    double *snode = nullptr;   // [N] per-node sigma terms
    double *states = nullptr;  // [cap][Q][N]
    int cap = 0;
    double dGp_direct = 0.0;   // host-side terms of dL/dG'
    // a captured lb_adjoint_run (run_graph), valid for one run length, one
    // starting buffer parity and adjoint buffer, and one context state
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    int runs = 0;              // runs so far (the first one runs directly)
    int g_nsteps = 0, g_cur = 0;
    double *g_lam = nullptr, *g_states = nullptr;
    unsigned long long g_key = 0;
    long long g_launches = 0;
};

namespace {

lb_status afail(cudaError_t e, const char *where) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", where, cudaGetErrorString(e));
    lb_set_error_message(msg);
    return LB_ECUDA;
}

PsiK adj_psik(const lb_ctx *c) { return PsiK{c->k.psi_kind, c->k.psi_eps, c->k.psi_inv}; }

lb_status fields_of(lb_adjoint *a, const double *st) {
    const int gb = grid_for(a->g.N);
    if (a->D == 2)
        adj::k_adj_fields<2, 9><<<gb, 256, 0, a->c->stream>>>(st, a->g, adj_psik(a->c), a->n, a->psi, a->dpsi);
    else
        adj::k_adj_fields<3, 19><<<gb, 256, 0, a->c->stream>>>(st, a->g, adj_psik(a->c), a->n, a->psi, a->dpsi);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : afail(e, "adjoint fields");
}

// fixed-order sum of each row of a [rows][N] device array into host out[rows]
lb_status rowsums(lb_adjoint *a, const double *d, int rows, double *out) {
    const int chunks = 64;
    double *part = nullptr;
    cudaError_t e = cudaMalloc(&part, (size_t)rows * chunks * sizeof(double));
    if (e != cudaSuccess) return afail(e, "adjoint reduction");
    adj::k_rowsum<<<dim3(chunks, rows), 256, 0, a->c->stream>>>(d, a->g.N, chunks, part);
    std::vector<double> h((size_t)rows * chunks);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, a->c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->c->stream);
    cudaFree(part);
    if (e != cudaSuccess) return afail(e, "adjoint reduction");
    for (int r = 0; r < rows; ++r) {
        double s = 0.0;
        for (int k = 0; k < chunks; ++k) s += h[(size_t)r * chunks + k];
        out[r] = s;
    }
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_adjoint_create(lb_ctx *c, lb_adjoint **out) {
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (!c) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    if (c->n_groups > adj::MAXG) return LB_EUNSUPPORTED;
    lb_adjoint *a = new lb_adjoint();
    a->c = c;
    a->D = c->D;
    a->Q = c->Q;
    a->g = Geom{c->g.nx, c->g.ny, c->g.nz, c->g.N, c->g.nx, c->g.ny, 0, 0, c->g.N};
    a->ngroups = c->n_groups;
    // group of each canonical pair: the group whose base has the same sorted
    // absolute components
    for (int p = 0; p < c->pairs64.npairs; ++p) {
        int v[3] = {std::abs((int)c->pairs64.v[p][0]), std::abs((int)c->pairs64.v[p][1]),
                    std::abs((int)c->pairs64.v[p][2])};
        std::sort(v, v + 3);
        int found = -1;
        for (int q = 0; q < c->n_groups && found < 0; ++q) {
            int b[3] = {std::abs(c->group_base[q][0]), std::abs(c->group_base[q][1]),
                        std::abs(c->group_base[q][2])};
            std::sort(b, b + 3);
            if (b[0] == v[0] && b[1] == v[1] && b[2] == v[2]) found = q;
        }
        if (found < 0) {
            delete a;
            return LB_EINVAL;
        }
        a->pg.g[p] = found;
    }
    const long long N = c->g.N;
    const size_t QN = (size_t)c->Q * N * sizeof(double);
    cudaError_t e = cudaMalloc(&a->lam, QN);
    if (e == cudaSuccess) e = cudaMalloc(&a->lam2, QN);
    if (e == cudaSuccess) e = cudaMalloc(&a->lacc, 3 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->lpsi, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->n, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->psi, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->dpsi, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->gnode, (size_t)(a->ngroups + 1) * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&a->snode, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(a->lam, 0, QN);
    if (e == cudaSuccess) e = cudaMemset(a->gnode, 0, (size_t)(a->ngroups + 1) * N * sizeof(double));
    if (e != cudaSuccess) {
        lb_adjoint_destroy(a);
        return afail(e, "lb_adjoint_create");
    }
    *out = a;
    return LB_OK;
}

lb_status lb_adjoint_destroy(lb_adjoint *a) {
    if (!a) return LB_OK;
    if (a->c && a->c->stream) cudaStreamSynchronize(a->c->stream);
    cudaFree(a->lam);
    cudaFree(a->lam2);
    cudaFree(a->lacc);
    cudaFree(a->lpsi);
    cudaFree(a->n);
    cudaFree(a->psi);
    cudaFree(a->dpsi);
    cudaFree(a->gnode);
    cudaFree(a->snode);
    cudaFree(a->states);
    if (a->graph_valid) cudaGraphExecDestroy(a->graph);
    delete a;
    return LB_OK;
}

lb_status lb_adjoint_set(lb_adjoint *a, const double *lam) {
    if (!a) return LB_EINVAL;
    const size_t QN = (size_t)a->Q * a->g.N * sizeof(double);
    cudaError_t e = lam ? cudaMemcpyAsync(a->lam, lam, QN, cudaMemcpyHostToDevice, a->c->stream)
                        : cudaMemsetAsync(a->lam, 0, QN, a->c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->c->stream);
    return e == cudaSuccess ? LB_OK : afail(e, "lb_adjoint_set");
}

lb_status lb_adjoint_get(lb_adjoint *a, double *lam) {
    if (!a || !lam) return LB_EINVAL;
    cudaError_t e = cudaMemcpyAsync(lam, a->lam, (size_t)a->Q * a->g.N * sizeof(double),
                                    cudaMemcpyDeviceToHost, a->c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->c->stream);
    return e == cudaSuccess ? LB_OK : afail(e, "lb_adjoint_get");
}

lb_status lb_adjoint_zero_grad(lb_adjoint *a) {
    if (!a) return LB_EINVAL;
    a->dGp_direct = 0.0;
    cudaError_t e = cudaMemsetAsync(a->gnode, 0, (size_t)(a->ngroups + 1) * a->g.N * sizeof(double),
                                    a->c->stream);
    return e == cudaSuccess ? LB_OK : afail(e, "lb_adjoint_zero_grad");
}

lb_status lb_adjoint_seed_sigma(lb_adjoint *a, int n_interfaces, double *sigma) {
    if (!a || n_interfaces < 1) return LB_EINVAL;
    lb_ctx *c = a->c;
    cudaError_t e = c->p.precision == LB_FP64 ? f64_get_state(c, a->lam2, 0, c->Q) : f32_get_state(c, a->lam2, 0, c->Q);
    if (e != cudaSuccess) return afail(e, "lb_adjoint_seed_sigma state");
    lb_status s = fields_of(a, a->lam2);
    if (s != LB_OK) return s;
    const double inv = 1.0 / n_interfaces;
    const int gb = grid_for(a->g.N);
    if (a->D == 2)
        adj::k_sigma_seed<2, 9><<<gb, 256, 0, c->stream>>>(a->psi, a->dpsi, a->g, c->pairs64, a->pg, c->Gp,
                                                         inv, a->ngroups, a->lam, a->gnode, a->snode);
    else
        adj::k_sigma_seed<3, 19><<<gb, 256, 0, c->stream>>>(a->psi, a->dpsi, a->g, c->pairs64, a->pg, c->Gp,
                                                          inv, a->ngroups, a->lam, a->gnode, a->snode);
    e = cudaGetLastError();
    if (e != cudaSuccess) return afail(e, "lb_adjoint_seed_sigma");
    double tot = 0.0;
    s = rowsums(a, a->snode, 1, &tot);
    if (s != LB_OK) return s;
    const double sig = 0.5 * c->Gp * inv * tot;
    a->dGp_direct += c->Gp != 0.0 ? sig / c->Gp : 0.0;
    if (sigma) *sigma = sig;
    return LB_OK;
}

namespace {
// the tensor seed of lb_adjoint_seed_pt for site weights dm already on the
// device (a->n, a->psi, a->dpsi hold the current state's fields)
lb_status seed_pt_dev(lb_adjoint *a, const double *dm, double *value);
}  // namespace

lb_status lb_adjoint_seed_pt(lb_adjoint *a, const double *m, double *value) {
    if (!a || !m) return LB_EINVAL;
    lb_ctx *c = a->c;
    PTPairs probe;
    if (!build_pt_pairs(c, &probe)) return LB_EUNSUPPORTED;
    const long long N = a->g.N;
    double *dm = nullptr;
    cudaError_t e = cudaMalloc(&dm, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dm, m, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = c->p.precision == LB_FP64 ? f64_get_state(c, a->lam2, 0, c->Q) : f32_get_state(c, a->lam2, 0, c->Q);
    if (e != cudaSuccess) {
        cudaFree(dm);
        return afail(e, "lb_adjoint_seed_pt");
    }
    lb_status s = fields_of(a, a->lam2);
    if (s == LB_OK) s = seed_pt_dev(a, dm, value);
    cudaFree(dm);
    return s;
}

lb_status lb_adjoint_seed_flat(lb_adjoint *a, int quantity, const double *params, double weight,
                               double *value) {
    if (!a || quantity < LB_FLAT_SIGMA || quantity > LB_FLAT_RATIO || !std::isfinite(weight))
        return LB_EINVAL;
    if ((quantity == LB_FLAT_WIDTH || quantity == LB_FLAT_RATIO) && !params) return LB_EINVAL;
    lb_ctx *c = a->c;
    PTPairs probe;
    if ((quantity == LB_FLAT_SIGMA || quantity == LB_FLAT_DELTA) && !build_pt_pairs(c, &probe))
        return LB_EUNSUPPORTED;
    const int nx = a->g.nx;
    double p[3] = {0.0, 0.0, 0.0};
    if (params) {
        const int np = quantity == LB_FLAT_WIDTH ? 3 : (quantity == LB_FLAT_RATIO ? 2 : 0);
        for (int k = 0; k < np; ++k) p[k] = params[k];
    }
    if (quantity == LB_FLAT_RATIO &&
        !(p[0] >= 0 && p[0] < nx && p[1] >= 0 && p[1] < nx && p[0] == (int)p[0] && p[1] == (int)p[1]))
        return LB_EINVAL;
    if (quantity == LB_FLAT_WIDTH && !(p[0] != p[1])) return LB_EINVAL;
    // profiles of the current state (binary64, on the device)
    double *buf = nullptr;   // prof [3 nx], gn [nx], gd [nx], val [2]
    cudaError_t e = cudaMalloc(&buf, (5 * (size_t)nx + 2) * sizeof(double));
    if (e != cudaSuccess) return afail(e, "lb_adjoint_seed_flat");
    double *prof = buf, *gn = buf + 3 * nx, *gd = buf + 4 * nx, *val = buf + 5 * nx;
    e = flat_profiles(c, prof, 0, nullptr, nullptr);
    if (e == cudaErrorNotSupported) {
        cudaFree(buf);
        return LB_EUNSUPPORTED;
    }
    if (e == cudaSuccess) {
        adj::k_flat_seed<<<1, 1, 0, c->stream>>>(prof, nx, quantity, p[0], p[1], p[2], gn, gd, val);
        e = cudaGetLastError();
    }
    double hv[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv, val, sizeof hv, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return afail(e, "lb_adjoint_seed_flat");
    }
    if (!std::isfinite(hv[0])) {
        cudaFree(buf);
        lb_set_error_message("lb_adjoint_seed_flat: no interface in the state");
        return LB_EINVAL;
    }
    // the state's fields (for the tensor seed), then the seeds; lam2 is free
    // once fields_of has read it and serves as the site weights m
    e = c->p.precision == LB_FP64 ? f64_get_state(c, a->lam2, 0, c->Q) : f32_get_state(c, a->lam2, 0, c->Q);
    lb_status s = e == cudaSuccess ? fields_of(a, a->lam2) : afail(e, "lb_adjoint_seed_flat");
    if (s == LB_OK) {
        adj::k_broadcast_seed<<<grid_for(a->g.N), 256, 0, c->stream>>>(a->lam, a->lam2, gn, gd, a->g,
                                                                      a->Q, weight);
        e = cudaGetLastError();
        if (e != cudaSuccess) s = afail(e, "lb_adjoint_seed_flat");
    }
    if (s == LB_OK && (quantity == LB_FLAT_SIGMA || quantity == LB_FLAT_DELTA)) {
        double tv = 0.0;
        s = seed_pt_dev(a, a->lam2, &tv);
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(buf);
    if (s != LB_OK) return s;
    if (value) *value = hv[0];
    return LB_OK;
}

namespace {
lb_status seed_pt_dev(lb_adjoint *a, const double *dm, double *value) {
    lb_ctx *c = a->c;
    static PTPairs P;   // host staging (large); calls are serialised per adjoint
    if (!build_pt_pairs(c, &P)) return LB_EUNSUPPORTED;
    const long long N = a->g.N;
    lb_status s = LB_OK;
    cudaError_t e;
    const int gb = grid_for(N);
    if (a->D == 2)
        adj::k_seed_pt<2, 9><<<gb, 256, 0, c->stream>>>(a->psi, a->dpsi, dm, a->g, P, a->pg, a->lam,
                                                      a->gnode, a->snode);
    else
        adj::k_seed_pt<3, 19><<<gb, 256, 0, c->stream>>>(a->psi, a->dpsi, dm, a->g, P, a->pg, a->lam,
                                                       a->gnode, a->snode);
    e = cudaGetLastError();
    double tot = 0.0;
    if (e == cudaSuccess) s = rowsums(a, a->snode, 1, &tot);
    if (e != cudaSuccess) return afail(e, "lb_adjoint_seed_pt");
    if (s != LB_OK) return s;
    a->dGp_direct += c->Gp != 0.0 ? tot / c->Gp : 0.0;
    if (value) *value = tot;
    return LB_OK;
}
}  // namespace

}  // extern "C"

namespace {

// the run itself: nsteps forward steps recorded, then nsteps adjoint steps
lb_status run_direct(lb_adjoint *a, int nsteps) {
    lb_ctx *c = a->c;
    const long long N = a->g.N;
    const size_t QN = (size_t)a->Q * N;
    // forward: record the state before each step, then step
    for (int t = 0; t < nsteps; ++t) {
        double *st = a->states + (size_t)t * QN;
        cudaError_t e = c->p.precision == LB_FP64 ? f64_get_state(c, st, 0, c->Q) : f32_get_state(c, st, 0, c->Q);
        if (e != cudaSuccess) return afail(e, "lb_adjoint_run record");
        lb_status s = lb_step(c, 1);
        if (s != LB_OK) return s;
    }
    // backward
    auto k = consts_as<double>(c->k);
    const int gb = grid_for(N);
    for (int t = nsteps - 1; t >= 0; --t) {
        const double *st = a->states + (size_t)t * QN;
        lb_status s = fields_of(a, st);
        if (s != LB_OK) return s;
        if (a->D == 2) {
            adj::k_adj_a<2, 9><<<gb, 256, 0, c->stream>>>(st, a->n, a->psi, a->lam, a->g, c->pairs64, a->pg, k,
                                                        c->Gp, a->ngroups, a->lam2, a->lacc, a->lpsi, a->gnode);
            adj::k_adj_b<2, 9><<<gb, 256, 0, c->stream>>>(a->lacc, a->lpsi, a->dpsi, a->g, c->pairs64, a->lam2);
        } else {
            adj::k_adj_a<3, 19><<<gb, 256, 0, c->stream>>>(st, a->n, a->psi, a->lam, a->g, c->pairs64, a->pg, k,
                                                         c->Gp, a->ngroups, a->lam2, a->lacc, a->lpsi, a->gnode);
            adj::k_adj_b<3, 19><<<gb, 256, 0, c->stream>>>(a->lacc, a->lpsi, a->dpsi, a->g, c->pairs64, a->lam2);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return afail(e, "lb_adjoint_run kernels");
        std::swap(a->lam, a->lam2);
    }
    return LB_OK;
}

// what the kernels of a run read from the context: its parameters, stencil,
// constants, options and buffers (the bytes from p to wait_polls, and the
// buffer pointers and stream)
unsigned long long ctx_key(const lb_ctx *c) {
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
    };
    const char *b0 = reinterpret_cast<const char *>(&c->p);
    const char *b1 = reinterpret_cast<const char *>(&c->tmap);
    mix(b0, (size_t)(b1 - b0));
    mix(&c->f, sizeof c->f);
    mix(&c->psi, sizeof c->psi);
    mix(&c->psi_halo, sizeof c->psi_halo);
    mix(&c->flags, sizeof c->flags);
    mix(&c->stream, sizeof c->stream);
    return h;
}

// A run of the same length from the same buffers repeats once per segment of
// a checkpointed backward pass: it is captured once as a CUDA graph (its
// host effects undone after the capture) and replayed, with the host effects
// (buffer parity, step and launch counts, adjoint buffer swap) applied here.
lb_status run_graph(lb_adjoint *a, int nsteps) {
    lb_ctx *c = a->c;
    const unsigned long long key = ctx_key(c);
    const bool same = a->graph_valid && a->g_nsteps == nsteps && a->g_cur == c->cur &&
                      a->g_lam == a->lam && a->g_states == a->states && a->g_key == key;
    if (!same) {
        if (a->graph_valid) cudaGraphExecDestroy(a->graph);
        a->graph_valid = false;
        const int cur0 = c->cur;
        const long long steps0 = c->steps, l0 = c->launches;
        double *lam0 = a->lam, *lam20 = a->lam2;
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return afail(e, "adjoint graph capture");
        lb_status s = run_direct(a, nsteps);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
        a->g_launches = c->launches - l0;
        c->cur = cur0;
        c->steps = steps0;
        c->launches = l0;
        a->lam = lam0;
        a->lam2 = lam20;
        if (s == LB_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&a->graph, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (s != LB_OK) return s;
        if (e2 != cudaSuccess) return afail(e2, "adjoint graph");
        a->graph_valid = true;
        a->g_nsteps = nsteps;
        a->g_cur = cur0;
        a->g_lam = lam0;
        a->g_states = a->states;
        a->g_key = key;
    }
    cudaError_t e = cudaGraphLaunch(a->graph, c->stream);
    if (e != cudaSuccess) return afail(e, "adjoint graph launch");
    if (nsteps & 1) {
        c->cur = 1 - c->cur;
        std::swap(a->lam, a->lam2);
    }
    c->steps += nsteps;
    c->launches += a->g_launches;
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_adjoint_run(lb_adjoint *a, int nsteps) {
    if (!a || nsteps < 0) return LB_EINVAL;
    if (nsteps == 0) return LB_OK;
    lb_ctx *c = a->c;
    const size_t QN = (size_t)a->Q * a->g.N;
    if (a->cap < nsteps) {
        cudaFree(a->states);
        a->states = nullptr;
        a->cap = 0;
        cudaError_t e = cudaMalloc(&a->states, (size_t)nsteps * QN * sizeof(double));
        if (e != cudaSuccess) return afail(e, "lb_adjoint_run states");
        a->cap = nsteps;
    }
    // the first run launches every kernel once directly; later runs of 4 or
    // more steps replay a captured graph (not while lb_timing records events)
    const bool graph = a->runs > 0 && nsteps >= 4 && !c->timing;
    ++a->runs;
    return graph ? run_graph(a, nsteps) : run_direct(a, nsteps);
}

lb_status lb_adjoint_gradient(lb_adjoint *a, double *dW, double *dG) {
    if (!a) return LB_EINVAL;
    std::vector<double> r(a->ngroups + 1);
    lb_status s = rowsums(a, a->gnode, a->ngroups + 1, r.data());
    if (s != LB_OK) return s;
    if (dW)
        for (int q = 0; q < a->ngroups; ++q) dW[q] = r[q];
    // G' = G (literal) or G/3 (G c_s^2 in the force)
    const double dGp = r[a->ngroups] + a->dGp_direct;
    if (dG) *dG = a->c->p.g_convention == LB_G_TIMES_CS2 ? dGp / 3.0 : dGp;
    return LB_OK;
}

}  // extern "C"
