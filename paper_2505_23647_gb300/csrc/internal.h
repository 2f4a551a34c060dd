// internal.h -- context layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cmath>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sclbm.h"

namespace sclbm {

constexpr int MAXP = LB_MAX_PAIRS;

// Canonical (e,-e) pairs of the forcing stencil, passed by value to kernels
// (kernel parameters live in the constant bank, so every thread of a warp
// reading the same pair is a broadcast).
struct PairsF64 {
    int npairs;
    int radius;
    signed char v[MAXP][3];
    double w[MAXP];
};
struct PairsF32 {
    int npairs;
    int radius;
    signed char v[MAXP][3];
    float w[MAXP];
};
// The binary32 stencil of the generic kernels, ready for nodes at least R
// from every boundary: per pair the site offset of e_a and W_a e_a folded
// per component (the force is three FMAs per pair), and the population
// index offsets of the pulls A_i(x - xi_i).  Boundary nodes use PairsF32.
struct PairsFast {
    int npairs, R;
    int nb[MAXP];         // offsets of e_a in the halo'd psi field
    int nbs[MAXP];        // offsets of e_a in a collision tile's psi box
    float we[MAXP][3];
    int pop[19];
    int H, Hz;            // psi halo in x, y and in z (0 in 2D)
    int pxp, pyp;         // halo'd psi row and plane extents
    int pull_pad;         // populations carry x/y ghosts: only z needs wrapping
};
// binary32 psi fields of the generic kernels carry a periodic halo of
// PSI_HALO nodes on every side (x, y and, in 3D, z)
constexpr int PSI_HALO = LB_MAX_RADIUS;
// Padded binary32 D3Q19 layouts: the columns next to each x edge written
// again as periodic images.  A TMA plane box reads 4 of them; 8 make each
// image one whole 32-byte sector of the row (measured 0.537 -> 0.520 ms per
// 256^3 step against 4).  The ghost rows are Geom::oy on each side.
constexpr int GHOST_X = 8;
// Tile of the generic binary32 collision (k_collide_f32): 32 x 8 threads
// take a brick of 32 x 8 x 8 nodes (3D) or 32 x 32 nodes (2D, four rows a
// thread); the brick's psi box carries a PSI_HALO halo on every side.
constexpr int CT_X = 32, CT_Y = 8, CT_Z = 8, CT_Y2 = 32;
constexpr int CT_BX = CT_X + 2 * PSI_HALO;
constexpr int ct_by(int D) { return (D == 3 ? CT_Y : CT_Y2) + 2 * PSI_HALO; }
constexpr int ct_bz(int D) { return D == 3 ? CT_Z + 2 * PSI_HALO : 1; }
constexpr int ct_box(int D) { return CT_BX * ct_by(D) * ct_bz(D); }

// Per-context constants of the collision (formed on the host once, in the
// same expressions as the reference: omega = 1/tau, cw_i = (1 - 1/(2 tau)) w_i).
struct Consts {
    double w[19];
    double cw[19];
    double omega;
    double mGp;     // -G'
    double rho0;    // FP32 shift
    double kA;      // A/tau of the F^2 forcing variant (0: Guo's T = 2 u F)
    int psi_kind;   // LB_PSI_EXP or LB_PSI_EPS
    double psi_eps, psi_inv;   // eps and RN(1/eps) of psi_eps
    // binary32 forms that move no mass systematically (mass_exact_f32, set
    // once at creation): the velocity weights (summing to 1 exactly), and the
    // fused kernels' keep = 1 - omega with the per-class omega w of the
    // classes |xi|^2 = 0, 1, 2 (keep + sum_c multiplicity_c omega w_c == 1)
    float w32[19];
    float keep32, omw32[3];
};

// Mass-exact binary32 constants.  A binary32 step's density coefficient is
// sum_c mult[c] v[c] (+ keep = 1 - omega for BGK in the even/odd form of
// the fused kernels); with each constant rounded on its own that sum misses
// its exact value by a few 1e-8, the same way every step, and the lattice
// mass drifts by as much per step.  mass_exact_f32 nudges v[1] and v[2] by
// at most a few ulps and gives v[0] (multiplicity 1) the remainder, so that
// sum_c mult[c] v[c] == target holds exactly (every term and partial sum is
// exact in binary64).  Returns false, leaving v as it was, if no such
// choice is found.
inline float nudge_f32(float x, int k) {
    for (; k > 0; --k) x = nextafterf(x, 1e30f);
    for (; k < 0; ++k) x = nextafterf(x, -1e30f);
    return x;
}

inline bool mass_exact_f32(float *v, const int *mult, double target) {
    for (int radius = 0; radius <= 6; ++radius)
        for (int k1 = -radius; k1 <= radius; ++k1)
            for (int k2 = -radius; k2 <= radius; ++k2) {
                if ((k1 < 0 ? -k1 : k1) != radius && (k2 < 0 ? -k2 : k2) != radius) continue;
                const float v1 = nudge_f32(v[1], k1), v2 = nudge_f32(v[2], k2);
                const double rest = target - (double)mult[1] * v1 - (double)mult[2] * v2;
                const float v0 = (float)rest;
                if ((double)v0 != rest) continue;
                v[0] = v0;
                v[1] = v1;
                v[2] = v2;
                return true;
            }
    return false;
}

// Consts::w32, keep32 and omw32 for a D2Q9 (Q = 9) or D3Q19 lattice, from
// its binary64 weights and omega.  keep = 1 - omega is first put on a 2^-26
// grid (a change of at most 7.5e-9 in the relaxation rate), which the
// axis and diagonal classes' ulp steps can always compensate.
inline void fill_mass_exact_f32(Consts &k, int Q) {
    const double wc[3] = {k.w[0], k.w[1], k.w[Q - 1]};   // rest, axis, diagonal
    const int mult[3] = {1, Q == 9 ? 4 : 6, Q == 9 ? 4 : 12};
    float v[3] = {(float)wc[0], (float)wc[1], (float)wc[2]};
    mass_exact_f32(v, mult, 1.0);
    for (int i = 0; i < 19; ++i) {
        k.w32[i] = 0.f;
        if (i < Q)
            for (int c = 0; c < 3; ++c)
                if (k.w[i] == wc[c]) k.w32[i] = v[c];
    }
    const double g = 67108864.0;   // 2^26
    const float keep = (float)(std::nearbyint((double)(float)(1.0 - k.omega) * g) / g);
    float o[3] = {(float)(k.omega * wc[0]), (float)(k.omega * wc[1]), (float)(k.omega * wc[2])};
    mass_exact_f32(o, mult, 1.0 - (double)keep);
    k.keep32 = keep;
    for (int c = 0; c < 3; ++c) k.omw32[c] = o[c];
}


struct Geom {
    int nx, ny, nz;
    long long N;        // nodes
    int nxp, nyp;       // padded plane of the population arrays
    int ox, oy;         // offset of node (0,0) inside a padded plane
    long long Np;       // population stride (nxp * nyp * nz)
};

// Device-side counters of a context.
struct Flags {
    unsigned long long err_step;   // first failing step (ULLONG_MAX: none)
    unsigned long long step;       // steps completed on the device
    unsigned long long exp_amb;    // uncertified exp roundings
    unsigned long long blocks_done;  // blocks finished in the current fused step
    unsigned long long timeouts;     // bounded barrier waits that gave up
};

}  // namespace sclbm

struct lb_ctx {
    lb_params p;
    int D, Q;
    sclbm::Geom g;
    double Gp;
    sclbm::Consts k;
    sclbm::PairsF64 pairs64;
    sclbm::PairsF32 pairs32;
    sclbm::PairsFast pfast;
    int n_groups;
    double e2;                // second moment of the stencil (lb_stencil_info.e2)
    int group_base[LB_MAX_PAIRS][3];
    double group_w[LB_MAX_PAIRS];
    bool stencil_set;
    bool fast3d_ok;           // the fused FP32 D3Q19 path applies
    bool fused_enabled;       // option LB_OPT_FUSED (default on)
    float fused_W[7];         // group weights for the fused kernel
    int fused_ng;             // number of E8 groups the fused kernel visits
    int fused_zchunk;         // z planes per CTA (option LB_OPT_ZCHUNK)
    bool fast2d_ok;           // the fused FP32 D2Q9 path applies (batch2d.cu)
    float fused2d_W[5];       // its group weights: (1,0), (1,1), (2,0), (2,1), (2,2)
    bool padded;              // populations carry periodic ghost columns/rows
    bool tma_ok;              // tensor maps built for the padded buffers
    bool fused_tma;           // option LB_OPT_TMA (default on)
    long long wait_polls;     // option LB_OPT_WAIT_POLLS: bound of the TMA kernel's waits
    CUtensorMap tmap[2][2];   // [buffer][R-1] plane boxes of TY + 2R rows
    void *f[2];               // population buffers [Q][N] (post-collision, pre-stream)
    int cur;                  // buffer holding the current state
    void *psi;                // psi of the precision in use: [N], or for binary32 with
                              // a halo of psi_halo nodes per side (PairsFast)
    int psi_halo;
    double *red;              // reduction partials and small results (128 KB)
    sclbm::Flags *flags;      // device counters
    cudaStream_t stream;
    bool own_stream;
    cudaGraphExec_t graph;    // kStepGraph steps, captured on first long lb_step
    bool graph_valid;
    int graph_cur;            // buffer parity the graph starts (and ends) on
    long long graph_launches; // kernels one replay launches
    long long steps;          // host-side step count
    long long launches;       // kernels launched
    // per-kernel timing (lb_timing)
    bool timing;
    cudaEvent_t *ev;          // event pool
    int ev_cap, ev_used;
    int *ev_kind;             // kind of each (start, stop) pair
    double kind_ms[LB_KERNEL_KINDS];
    long long kind_n[LB_KERNEL_KINDS];
};

// set the thread's last-error message returned by lb_last_cuda_error
void lb_set_error_message(const char *msg);

namespace sclbm {
// per-kernel timing brackets (no-ops unless lb_timing is enabled)
void tm_begin(lb_ctx *c, int kind);
void tm_end(lb_ctx *c);
// precision-specific launchers (fp64.cu / fp32.cu)
cudaError_t f64_init(lb_ctx *c, const double *rho, const double *u);
cudaError_t f64_step(lb_ctx *c);          // one step, swaps buffers
cudaError_t f64_psi(lb_ctx *c);           // psi of current state into c->psi
cudaError_t f64_fields(lb_ctx *c, double *n, double *u, double *mom);
cudaError_t f64_get_state(lb_ctx *c, double *f, int i0, int i1);   // populations [i0, i1)
cudaError_t f64_set_state(lb_ctx *c, const double *f, int i0, int i1);
cudaError_t f64_density_psi(lb_ctx *c, double *n, double *psi);
cudaError_t f32_init(lb_ctx *c, const double *rho, const double *u);
cudaError_t f32_step(lb_ctx *c);
cudaError_t f32_psi(lb_ctx *c);
cudaError_t f32_fields(lb_ctx *c, double *n, double *u, double *mom);
cudaError_t f32_get_state(lb_ctx *c, double *f, int i0, int i1);
cudaError_t f32_set_state(lb_ctx *c, const double *f, int i0, int i1);   // no ghost refresh
cudaError_t f32_density_psi(lb_ctx *c, double *n, double *psi);
// fused single-pass D3Q19 step (fused3d.cu)
bool fused3d_applicable(const lb_ctx *c, float *W, int *ng);
cudaError_t f32_fused3d_step(lb_ctx *c, const float *W, int ng);
cudaError_t f32_fused3d_tma_step(lb_ctx *c, const float *W, int ng);
// the fused TMA kernel's measuring pass: per-block records staged in part,
// the 7 observables (binary64, the generic pass's layout) into res
cudaError_t f32_fused3d_tma_measure(lb_ctx *c, void *part, double *res);
bool tma_make_maps(lb_ctx *c);
// fused single-pass D2Q9 step (batch2d.cu)
bool fused2d_applicable(const lb_ctx *c, float *W5);
cudaError_t f32_fused2d_step(lb_ctx *c);
cudaError_t ghosts_refresh(lb_ctx *c);   // padded layouts: refresh ghost cells of f[cur]
// observe.cu: what is measured on a lattice, all staged without allocation
// in the idle population buffer (stage_ptr, stage_bytes bytes) and the
// context's reduction buffer
size_t stage_bytes(const lb_ctx *c);
double *stage_ptr(lb_ctx *c);
cudaError_t obs_fused(lb_ctx *c);          // 7 results at obs_results(c)
double *obs_results(lb_ctx *c);
void psi64_field(lb_ctx *c, double *psi);  // binary64 psi of every node
cudaError_t ptensor_field(lb_ctx *c, double *psi, double *out);
cudaError_t flat_interfaces(lb_ctx *c, int maxw, lb_flat_obs *out_dev, int *count_dev);
// profiles of n, P^xx, P^yy along x into prof_out (device [3][nx]); windows too if out_dev
cudaError_t flat_profiles(lb_ctx *c, double *prof_out, int maxw, lb_flat_obs *out_dev,
                          int *count_dev);
cudaError_t curved_interface(lb_ctx *c, const double *center, double e2, lb_curved_obs *out_dev);
// lattice pressure tensor of Appendices E/F, per pair (e, -e): A = psi(x) (psi(x+e) +
// psi(x-e)), B = sum over the pair's links of psi(x+a) psi(x+b) (links prepared
// on the host), s = W (kA A + kB B), P^{mu nu}(x) += s e^mu e^nu, from (n/3) delta
struct PTPairs {
    int npairs;
    signed char v[MAXP][3];
    signed char nlink[MAXP];
    signed char link[MAXP][4][2][3];
    double w[MAXP], kA[MAXP], kB[MAXP];
};
// classify the context's pairs and build their link lists (false: a group
// outside Appendices E/F)
bool build_pt_pairs(const lb_ctx *c, PTPairs *P);
cudaError_t exp_batch(const double *x, double *y, long long n,
                      unsigned long long *amb, cudaStream_t s);
cudaError_t psi_batch(const double *n_in, double *psi, long long n, int kind, double eps,
                      unsigned long long *amb, cudaStream_t s);
}  // namespace sclbm
