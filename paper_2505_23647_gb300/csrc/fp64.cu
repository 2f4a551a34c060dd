// fp64.cu -- binary64 path (compiled with -fmad=false: every product and sum
// below rounds exactly as written, matching the documented FP64 order), the
// FP64 reductions for lb_observables, the lattice pressure tensor
// (Appendices E and F) and the exp diagnostic.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace sclbm {

#define SCLBM_DISPATCH(c, FN2, FN3) \
    ((c)->Q == 9 ? (FN2) : (FN3))

cudaError_t f64_init(lb_ctx *c, const double *rho, const double *u) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    double *A = (double *)c->f[c->cur];
    if (c->Q == 9)
        k_init<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, rho, u, k);
    else
        k_init<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, rho, u, k);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f64_step(lb_ctx *c) {
    auto k = consts_as<double>(c->k);
    const double *A = (const double *)c->f[c->cur];
    double *B = (double *)c->f[1 - c->cur];
    double *psi = (double *)c->psi;
    int gb = grid_for(c->g.N);
    if (c->Q == 9) {
        tm_begin(c, LB_KERNEL_PSI);
        k_psi<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, psi, c->g, 0.0, c->flags, psik(c));
        tm_end(c);
        tm_begin(c, LB_KERNEL_COLLIDE);
        k_collide<double, PairsF64, 2, 9, false>
            <<<gb, 256, 0, c->stream>>>(A, B, psi, c->g, c->pairs64, k, c->flags);
        tm_end(c);
    } else {
        tm_begin(c, LB_KERNEL_PSI);
        k_psi<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, psi, c->g, 0.0, c->flags, psik(c));
        tm_end(c);
        tm_begin(c, LB_KERNEL_COLLIDE);
        k_collide<double, PairsF64, 3, 19, false>
            <<<gb, 256, 0, c->stream>>>(A, B, psi, c->g, c->pairs64, k, c->flags);
        tm_end(c);
    }
    c->launches += 2;
    c->cur = 1 - c->cur;
    return cudaGetLastError();
}

cudaError_t f64_density_psi(lb_ctx *c, double *n, double *psi) {
    int gb = grid_for(c->g.N);
    const double *A = (const double *)c->f[c->cur];
    if (c->Q == 9)
        k_density_psi64<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, 0.0, n, psi, c->flags, psik(c));
    else
        k_density_psi64<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, 0.0, n, psi, c->flags, psik(c));
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f64_fields(lb_ctx *c, double *n, double *u, double *mom) {
    cudaError_t e = f64_density_psi(c, n, n + c->g.N);
    if (e != cudaSuccess) return e;
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const double *A = (const double *)c->f[c->cur];
    if (c->Q == 9)
        k_fields64<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, c->pairs64, k, n, n + c->g.N, u, mom);
    else
        k_fields64<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, c->pairs64, k, n, n + c->g.N, u, mom);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f64_get_state(lb_ctx *c, double *f) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const double *A = (const double *)c->f[c->cur];
    if (c->Q == 9)
        k_get_state<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k);
    else
        k_get_state<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f64_set_state(lb_ctx *c, const double *f) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    double *A = (double *)c->f[c->cur];
    if (c->Q == 9)
        k_set_state<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k);
    else
        k_set_state<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 reductions: compensated (double-double) sums in a fixed order.
struct Red {
    ddv mass, mom[3];
    double umax2, rmin, rmax;
};

__device__ __forceinline__ void red_combine(Red &a, const Red &b) {
    a.mass = dd_add(a.mass, b.mass);
#pragma unroll
    for (int k = 0; k < 3; ++k) a.mom[k] = dd_add(a.mom[k], b.mom[k]);
    a.umax2 = fmax(a.umax2, b.umax2);
    a.rmin = fmin(a.rmin, b.rmin);
    a.rmax = fmax(a.rmax, b.rmax);
}

__device__ __forceinline__ Red red_shfl(const Red &r, int off) {
    Red o;
    o.mass.hi = __shfl_down_sync(0xffffffffu, r.mass.hi, off);
    o.mass.lo = __shfl_down_sync(0xffffffffu, r.mass.lo, off);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.mom[k].hi = __shfl_down_sync(0xffffffffu, r.mom[k].hi, off);
        o.mom[k].lo = __shfl_down_sync(0xffffffffu, r.mom[k].lo, off);
    }
    o.umax2 = __shfl_down_sync(0xffffffffu, r.umax2, off);
    o.rmin = __shfl_down_sync(0xffffffffu, r.rmin, off);
    o.rmax = __shfl_down_sync(0xffffffffu, r.rmax, off);
    return o;
}

__device__ __forceinline__ Red red_block(Red r) {
    __shared__ Red sh[32];
    for (int off = 16; off > 0; off >>= 1) {
        Red o = red_shfl(r, off);
        red_combine(r, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = r;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (wid == 0) {
        if (lane < nw) r = sh[lane];
        else {
            r.mass = {0.0, 0.0};
            for (int k = 0; k < 3; ++k) r.mom[k] = {0.0, 0.0};
            r.umax2 = 0.0;
            r.rmin = __longlong_as_double(0x7ff0000000000000ULL);
            r.rmax = -__longlong_as_double(0x7ff0000000000000ULL);
        }
        for (int off = 16; off > 0; off >>= 1) {
            Red o = red_shfl(r, off);
            red_combine(r, o);
        }
    }
    return r;
}

__device__ __forceinline__ Red red_zero() {
    Red r;
    r.mass = {0.0, 0.0};
    for (int k = 0; k < 3; ++k) r.mom[k] = {0.0, 0.0};
    r.umax2 = 0.0;
    r.rmin = __longlong_as_double(0x7ff0000000000000ULL);
    r.rmax = -__longlong_as_double(0x7ff0000000000000ULL);
    return r;
}

__global__ void __launch_bounds__(256) k_reduce1(long long N, int D, const double *__restrict__ n,
                                                 const double *__restrict__ u,
                                                 const double *__restrict__ mom, Red *partial) {
    Red r = red_zero();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += stride) {
        const double ns = n[s];
        r.mass = dd_add(r.mass, dd_two_sum(ns, 0.0));
        double uu = u[s] * u[s];
        for (int mu = 0; mu < D; ++mu) {
            if (mu) uu = uu + u[(long long)mu * N + s] * u[(long long)mu * N + s];
            r.mom[mu] = dd_add(r.mom[mu], ddv{mom[(long long)mu * N + s], 0.0});
        }
        r.umax2 = fmax(r.umax2, uu);
        r.rmin = fmin(r.rmin, ns);
        r.rmax = fmax(r.rmax, ns);
    }
    r = red_block(r);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void __launch_bounds__(256) k_reduce2(int nb, const Red *__restrict__ partial,
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

cudaError_t obs_reduce(lb_ctx *c, const double *n, const double *u, const double *mom,
                       double *out_dev) {
    const int nb = 1024;
    k_reduce1<<<nb, 256, 0, c->stream>>>(c->g.N, c->D, n, u, mom, (Red *)c->red);
    k_reduce2<<<1, 256, 0, c->stream>>>(nb, (const Red *)c->red, out_dev);
    c->launches += 2;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lattice pressure tensor.  Per pair e (with -e): the endpoint products
// A = psi(x) (psi(x+e) + psi(x-e)) and the interior/midpoint link products
template <int D>
__global__ void __launch_bounds__(128) k_ptensor(Geom g, const double *__restrict__ n,
                                                 const double *__restrict__ psi, const PTPairs P,
                                                 double *__restrict__ out) {
    constexpr int NC = D == 2 ? 3 : 6;
    constexpr int cmu[6] = {0, 0, D == 2 ? 1 : 0, 1, 1, 2};
    constexpr int cnu[6] = {0, 1, D == 2 ? 1 : 2, 1, 2, 2};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        int x, y, z;
        coords(g, s, x, y, z);
        double Ps[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) Ps[k] = (cmu[k] == cnu[k]) ? n[s] / 3.0 : 0.0;
        const double p0 = psi[s];
        for (int a = 0; a < P.npairs; ++a) {
            const int e0 = P.v[a][0], e1 = P.v[a][1], e2 = P.v[a][2];
            const double A = p0 * (psi[site(g, x + e0, y + e1, z + e2)] +
                                   psi[site(g, x - e0, y - e1, z - e2)]);
            double B = 0.0;
            for (int l = 0; l < P.nlink[a]; ++l) {
                const signed char *q = &P.link[a][l][0][0];
                B = B + psi[site(g, x + q[0], y + q[1], z + q[2])] *
                            psi[site(g, x + q[3], y + q[4], z + q[5])];
            }
            const double sc = P.w[a] * (P.kA[a] * A + P.kB[a] * B);
            const int e[3] = {e0, e1, e2};
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const int ee = e[cmu[k]] * e[cnu[k]];
                if (ee) Ps[k] = Ps[k] + sc * (double)ee;
            }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) out[(long long)k * g.N + s] = Ps[k];
    }
}

static int igcd(int a, int b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) { int t = a % b; a = b; b = t; }
    return a;
}

// Host: classify pairs and build the link lists (returns false for a group
// outside Appendices E/F).
bool build_pt_pairs(const lb_ctx *c, PTPairs *P) {
    P->npairs = c->pairs64.npairs;
    for (int a = 0; a < P->npairs; ++a) {
        int e[3] = {c->pairs64.v[a][0], c->pairs64.v[a][1], c->pairs64.v[a][2]};
        for (int k = 0; k < 3; ++k) P->v[a][k] = (signed char)e[k];
        P->w[a] = c->pairs64.w[a];
        int mag[3] = {e[0] < 0 ? -e[0] : e[0], e[1] < 0 ? -e[1] : e[1], e[2] < 0 ? -e[2] : e[2]};
        int ref = 0, alleq = 1, mx = 0;
        for (int k = 0; k < 3; ++k) {
            if (mag[k]) { if (!ref) ref = mag[k]; else if (mag[k] != ref) alleq = 0; }
            if (mag[k] > mx) mx = mag[k];
        }
        if (alleq) {
            if (mx > 4) return false;
            int m = igcd(igcd(e[0], e[1]), e[2]);
            int h[3] = {e[0] / m, e[1] / m, e[2] / m};
            P->nlink[a] = (signed char)(m - 1);
            for (int j = 1; j < m; ++j)
                for (int k = 0; k < 3; ++k) {
                    P->link[a][j - 1][0][k] = (signed char)(-j * h[k]);
                    P->link[a][j - 1][1][k] = (signed char)((m - j) * h[k]);
                }
            P->kA[a] = c->Gp / (2.0 * (double)m);
            P->kB[a] = c->Gp / (double)m;
        } else {
            int s2 = 0, s1 = 0, s0 = 0;
            for (int k = 0; k < 3; ++k) {
                if (mag[k] == 2) s2++; else if (mag[k] == 1) s1++; else if (mag[k] == 0) s0++;
            }
            if (!((s2 == 1 && s1 == 1 && s0 == 1) || (s2 == 1 && s1 == 2) || (s2 == 2 && s1 == 1)))
                return false;
            int odd[3], nodd = 0;
            for (int k = 0; k < 3; ++k) if (mag[k] % 2) odd[nodd++] = k;
            int nmid = 1 << nodd;
            P->nlink[a] = (signed char)nmid;
            for (int b = 0; b < nmid; ++b) {
                int off[3];
                for (int k = 0; k < 3; ++k) off[k] = -e[k] / 2;
                for (int q = 0; q < nodd; ++q) {
                    int k = odd[q];
                    int sg = ((b >> (nodd - 1 - q)) & 1) ? -1 : 1;
                    off[k] = (sg - e[k]) / 2;
                }
                for (int k = 0; k < 3; ++k) {
                    P->link[a][b][0][k] = (signed char)off[k];
                    P->link[a][b][1][k] = (signed char)(off[k] + e[k]);
                }
            }
            P->kA[a] = c->Gp / 4.0;
            P->kB[a] = c->Gp / (2.0 * (double)nmid);
        }
    }
    return true;
}

cudaError_t ptensor(lb_ctx *c, const double *n, const double *psi, double *out) {
    static PTPairs P;   // host staging (large); calls on one context are serialised
    if (!build_pt_pairs(c, &P)) return cudaErrorNotSupported;
    int gb = grid_for(c->g.N, 128);
    if (c->D == 2)
        k_ptensor<2><<<gb, 128, 0, c->stream>>>(c->g, n, psi, P, out);
    else
        k_ptensor<3><<<gb, 128, 0, c->stream>>>(c->g, n, psi, P, out);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_exp_batch(const double *__restrict__ x, double *__restrict__ y, long long n,
                            unsigned long long *amb) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = exp_cr(x[i], amb);
}

cudaError_t exp_batch(const double *x, double *y, long long n, unsigned long long *amb,
                      cudaStream_t s) {
    k_exp_batch<<<grid_for(n), 256, 0, s>>>(x, y, n, amb);
    return cudaGetLastError();
}

__global__ void k_psi_batch(const double *__restrict__ n_in, double *__restrict__ psi,
                            long long n, PsiK pk, unsigned long long *amb) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        psi[i] = psi_eval<double>(n_in[i], pk, amb);
}

cudaError_t psi_batch(const double *n_in, double *psi, long long n, int kind, double eps,
                      unsigned long long *amb, cudaStream_t s) {
    const PsiK pk{kind, kind == LB_PSI_EPS ? eps : 0.0, kind == LB_PSI_EPS ? 1.0 / eps : 0.0};
    k_psi_batch<<<grid_for(n), 256, 0, s>>>(n_in, psi, n, pk, amb);
    return cudaGetLastError();
}

}  // namespace sclbm
