// fp32.cu -- binary32 path with shifted populations g_i = f_i - w_i rho0
// (generic kernels for every lattice and stencil).
#include <cuda_runtime.h>

#include "collide_tiled.cuh"

namespace sclbm {

fc::Params fused_params(const lb_ctx *c, const float *W);
// the D2Q9 tiled collision with the batch kernels' pair-symmetric collide9
// (batch2d.cu)
void f32_collide2d_tiled(lb_ctx *c, const float *A, float *B, const float *psi);

cudaError_t ghosts_refresh(lb_ctx *c) {
    if (!c->padded) return cudaSuccess;
    const long long rows = (long long)c->g.nyp * c->g.nz * c->Q;   // one warp a row
    k_ghosts<float><<<grid_for(rows * 32), 256, 0, c->stream>>>((float *)c->f[c->cur], c->g, c->Q);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_init(lb_ctx *c, const double *rho, const double *u) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    float *A = (float *)c->f[c->cur];
    if (c->Q == 9)
        k_init<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, rho, u, k);
    else
        k_init<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, rho, u, k);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : ghosts_refresh(c);
}

cudaError_t f32_step(lb_ctx *c) {
    if (c->Q == 19 && c->fast3d_ok && c->fused_enabled)
        return f32_fused3d_step(c, c->fused_W, c->fused_ng);
    if (c->Q == 9 && c->fast2d_ok && c->fused_enabled) return f32_fused2d_step(c);
    auto k = consts_as<float>(c->k);
    const float *A = (const float *)c->f[c->cur];
    float *B = (float *)c->f[1 - c->cur];
    float *psi = (float *)c->psi;
    int gb = grid_for(c->g.N);
    if (!c->psi_halo) {   // beyond 32-bit node indices: the wrapped kernels
        if (c->Q == 9) {
            k_psi<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->flags, psik(c));
            k_collide<float, PairsF32, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, B, psi, c->g, c->pairs32, k, c->flags);
        } else {
            k_psi<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->flags, psik(c));
            k_collide<float, PairsF32, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, B, psi, c->g, c->pairs32, k, c->flags);
        }
    } else if (c->Q == 9) {
        tm_begin(c, LB_KERNEL_PSI);
        k_psi_f32<2, 9><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->pfast, c->flags, psik(c));
        tm_end(c);
        tm_begin(c, LB_KERNEL_COLLIDE);
        f32_collide2d_tiled(c, A, B, psi);
        tm_end(c);
    } else {
        tm_begin(c, LB_KERNEL_PSI);
        k_psi_f32<3, 19><<<gb, 256, 0, c->stream>>>(A, psi, c->g, k.rho0, c->pfast, c->flags, psik(c));
        tm_end(c);
        tm_begin(c, LB_KERNEL_COLLIDE);
        // the collision constants of the fused kernels (their force weights
        // are not used here)
        const float W0[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const Col19 col{fused_params(c, W0)};
        const dim3 grid((c->g.nx + CT_X - 1) / CT_X, (c->g.ny + CT_Y - 1) / CT_Y,
                        (c->g.nz + CT_Z - 1) / CT_Z);
        k_collide_f32<3, 19><<<grid, dim3(CT_X, CT_Y), ct_box(3) * sizeof(float), c->stream>>>(
            A, B, psi, c->g, c->pfast, k, col, c->flags);
        tm_end(c);
    }
    c->launches += 2;
    c->cur = 1 - c->cur;
    cudaError_t e = cudaGetLastError();
    // k_collide_f32 writes the ghost images itself; the wrapped kernels do not
    return e != cudaSuccess || c->psi_halo ? e : ghosts_refresh(c);
}

cudaError_t f32_density_psi(lb_ctx *c, double *n, double *psi) {
    int gb = grid_for(c->g.N);
    const float *A = (const float *)c->f[c->cur];
    if (c->Q == 9)
        k_density_psi64<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->k.rho0, n, psi, c->flags, psik(c));
    else
        k_density_psi64<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->k.rho0, n, psi, c->flags, psik(c));
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_fields(lb_ctx *c, double *n, double *u, double *mom) {
    cudaError_t e = f32_density_psi(c, n, n + c->g.N);
    if (e != cudaSuccess) return e;
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const float *A = (const float *)c->f[c->cur];
    // the widened populations keep their shift: n already includes rho0, and
    // j, u and j + F/2 do not depend on it (sum_i w_i xi_i = 0)
    if (c->Q == 9)
        k_fields64<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->pairs64, k, n, n + c->g.N, u, mom);
    else
        k_fields64<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, c->pairs64, k, n, n + c->g.N, u, mom);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_get_state(lb_ctx *c, double *f, int i0, int i1) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    const float *A = (const float *)c->f[c->cur];
    if (c->Q == 9)
        k_get_state<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    else
        k_get_state<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t f32_set_state(lb_ctx *c, const double *f, int i0, int i1) {
    auto k = consts_as<double>(c->k);
    int gb = grid_for(c->g.N);
    float *A = (float *)c->f[c->cur];
    if (c->Q == 9)
        k_set_state<float, 2, 9, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    else
        k_set_state<float, 3, 19, true><<<gb, 256, 0, c->stream>>>(A, c->g, f, k, i0, i1);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace sclbm
