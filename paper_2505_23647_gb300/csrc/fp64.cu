// fp64.cu -- binary64 path (compiled with -fmad=false: every product and sum
// below rounds exactly as written, matching the documented FP64 order), the
// link tables of the lattice pressure tensor (Appendices E and F; the tensor
// itself is in observe.cu) and the exp diagnostic.
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

cudaError_t f64_get_state(lb_ctx *c, double *f, int i0, int i1) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const double *A = (const double *)c->f[c->cur];
    if (c->Q == 9)
        k_get_state<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    else
        k_get_state<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f64_set_state(lb_ctx *c, const double *f, int i0, int i1) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    double *A = (double *)c->f[c->cur];
    if (c->Q == 9)
        k_set_state<double, 2, 9, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    else
        k_set_state<double, 3, 19, false><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
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
