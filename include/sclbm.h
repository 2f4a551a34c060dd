/*
 * sclbm.h -- C ABI of the GB300 (sm_103a) Shan-Chen multiphase
 * lattice-Boltzmann library with extended, tunable forcing stencils
 * (Lulli & Ching, "Higher-order Tuning of Interface Physics in Multiphase
 * Lattice Boltzmann").
 *
 * Model (one step, every node x of a fully periodic lattice; Sec. II and
 * Sec. III A of the paper):
 *   n = sum_i f_i,  psi = exp(-1/n)
 *   F(x) = -G' psi(x) sum_a W(|e_a|^2) psi(x + e_a) e_a          (eq. sc_f)
 *   u = (sum_i f_i xi_i + F/2) / n                     (force-shifted u)
 *   f_i* = f_i - (f_i - f_i^eq(n,u))/tau + F_i (Guo, T = 2uF)
 *                                        (eqs. lbm, omega_i, f_eq, GuoForcing)
 *   f_i(x + xi_i, t+1) = f_i*(x)                                 (streaming)
 * G' = G for LB_G_LITERAL (the force written without c_s^2, the library's
 * default) or G c_s^2 = G/3 for LB_G_TIMES_CS2 (eq. sc_f as printed).
 *
 * Conventions shared by every call
 *   - Fields are x-fastest: index s = (z*ny + y)*nx + x.  2D lattices have
 *     nz = 1.  Vector fields are component-major: [D][N].
 *   - Populations ("state") are component-major [Q][N] float64, f_i(x) at
 *     integer time after streaming.  Velocity order, D2Q9:
 *       0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1)
 *       7 (-1,-1) 8 (1,-1)
 *     D3Q19:
 *       0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0) 5 (0,0,1)
 *       6 (0,0,-1) 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
 *       11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1)
 *       16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *   - Host pointers are caller-owned and only read/written during the call.
 *     Device memory is owned by the context until lb_destroy.
 *   - Every call returns an lb_status; no C++ exception crosses the ABI.
 *     A context is not thread-safe: use one context per host thread.
 *   - Precision LB_FP64 follows the exact rounding order documented below,
 *     so results equal a reference that evaluates the same expressions
 *     in IEEE binary64 (round to nearest, no FMA contraction) bit for bit.
 *     LB_FP32_SHIFTED stores g_i = f_i - w_i rho0 in binary32 and computes
 *     in binary32 (density within 1e-5 relative of binary64 over 100 steps
 *     on the tested workloads).
 *
 * FP64 rounding order (a reading of the model; every binary64 operation
 * below is rounded to nearest):
 *   n = ((f_0 + f_1) + f_2) + ...;  psi = RN(exp(RN(-1/n))), exp correctly
 *   rounded;  acc^mu += (W_a*(psi(x+e_a) - psi(x-e_a))) * e_a^mu over the
 *   canonical (e,-e) pairs of lb_expand_stencil;  F = (-G'*psi(x))*acc;
 *   j^mu = sum_i f_i xi_i^mu in table order;  u = (j + 0.5*F)/n;
 *   uu = u.u, uF = u.F, cu = xi.u, cF = xi.F summed x, y, z;
 *   f_eq = (w_i*n)*(((1 + 3*cu) + 4.5*(cu*cu)) - 1.5*uu);
 *   S = ((1 - 1/(2 tau))*w_i)*((3*cF + 9*(cu*cF)) - 3*uF);
 *   f* = (f - (1/tau)*(f - f_eq)) + S.
 */
#ifndef SCLBM_H
#define SCLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lb_status {
    LB_OK = 0,
    LB_EINVAL = 1,        /* bad argument or parameter */
    LB_ENOMEM = 2,        /* device or host allocation failed */
    LB_ECUDA = 3,         /* a CUDA runtime call failed (see lb_last_cuda_error) */
    LB_EUNSTABLE = 4,     /* a node had n <= 0 or NaN (see lb_obs.error_step) */
    LB_EUNSUPPORTED = 5,  /* valid request the library does not cover */
    LB_ESTATE = 6         /* call out of order, e.g. lb_step before lb_set_stencil */
} lb_status;

enum { LB_D2Q9 = 0, LB_D3Q19 = 1 };
enum { LB_FP64 = 0, LB_FP32_SHIFTED = 1 };
enum { LB_G_LITERAL = 0, LB_G_TIMES_CS2 = 1 };
/* Pseudopotential: LB_PSI_EXP psi = exp(-1/n) (Sec. IV B); LB_PSI_EPS
 * psi_eps = (n/(eps+n))^(1/eps) (eq. psieps, Sec. IV B / V C, e.g.
 * eps = 14/29 with e4 = 4/5), evaluated in binary64 as
 * RN(RN(n/RN(eps+n))^RN(1/eps)) with a correctly rounded power.  The
 * shifted-binary32 paths (two-kernel, fused D3Q19 and D2Q9, batches) all form
 * psi_eps as exp2f(RN(1/eps) * log2f(n / (eps + n))) in binary32 (the base
 * lies in (0, 1); about 2e-7 relative to the exact power), so every FP32 path uses
 * the same psi; a batch may mix both kinds. */
enum { LB_PSI_EXP = 0, LB_PSI_EPS = 1 };

/* Largest number of (e,-e) pairs and largest |component| of a stencil vector. */
#define LB_MAX_PAIRS 160
#define LB_MAX_RADIUS 4

typedef struct lb_params {
    int lattice;        /* LB_D2Q9 or LB_D3Q19 */
    int nx, ny, nz;     /* periodic lattice size; nz = 1 for D2Q9; each >= 1 */
    int precision;      /* LB_FP64 or LB_FP32_SHIFTED */
    double tau;         /* BGK relaxation time, > 1/2 */
    double G;           /* coupling constant (G < 0 separates phases) */
    int g_convention;   /* LB_G_LITERAL or LB_G_TIMES_CS2 */
    int psi_kind;       /* LB_PSI_EXP (default) or LB_PSI_EPS */
    double psi_eps;     /* eps of LB_PSI_EPS (> 0); ignored for LB_PSI_EXP */
    double rho0_shift;  /* rho0 of the FP32 shift g_i = f_i - w_i rho0 (default 0.5) */
    double forcing_A;   /* F^2 forcing variant: the tensor of eq. GuoForcing is
                           T = 2 u F - (A/tau) F F (Sec. VI); 0 (default) is
                           Guo's T = 2 u F.  Every path serves nonzero A. */
} lb_params;

typedef struct lb_stencil_info {
    int n_groups;       /* symmetry groups */
    int n_pairs;        /* (e,-e) pairs = n_vectors / 2 */
    int n_vectors;      /* N_e of the paper's tables */
    int radius;         /* max |component| */
    double e2, e4, e6, e8;   /* <x^2>, <x^2y^2>, <x^4y^2>/3, <x^4y^4>/9 */
    double iso_residual[4];  /* max |M_2k - e_2k Delta_2k| for 2k = 4,6,8,10 */
} lb_stencil_info;

typedef struct lb_obs {
    double mass;        /* sum_x n */
    double mom[3];      /* sum_x (j + F/2) */
    double umax;        /* max_x |u| */
    double rho_min, rho_max;
    long long step;     /* steps taken since lb_create */
    long long error_step;    /* first step whose density check failed, -1 if none */
    long long exp_ambiguous; /* FP64 exp evaluations flagged as too close to a
                                rounding boundary to certify (expected 0) */
} lb_obs;

/* One interface of a flat periodic slab (gradients along x), from the
 * binary64 profiles of n, P_N = P^xx and P_T = P^yy averaged over y (and z).
 * The window runs half way to the neighbouring interfaces; site x is the
 * cell [x - 1/2, x + 1/2]; n_l, n_g are the profile's values at the
 * window's liquid and gas ends. */
typedef struct lb_flat_obs {
    double sigma;       /* sum over the window of P_N - P_T (eq. sigma0pnpt) */
    double z_s;         /* first moment of P_N - P_T (surface of tension, eq. ZSDef) */
    double z_e;         /* equimolar surface, Gamma(z_e) = 0 */
    double delta;       /* Tolman length z_e - z_s, x oriented liquid -> gas (eq. zemzs) */
    double delta_ads;   /* Gamma(z_s) / (n_l - n_g) (eq. deltaads) */
    double n_l, n_g;    /* bulk densities at the window's ends */
    int window_lo, window_hi;  /* inclusive x range (may extend past 0 or nx-1: periodic) */
    int rising;         /* 1: gas -> liquid along +x, 0: liquid -> gas */
} lb_flat_obs;

/* A droplet or bubble at rest, in binary64 (Sec. III B, Sec. V B). */
typedef struct lb_curved_obs {
    double n_in;        /* density at the centre (linear interpolation) */
    double n_out;       /* density at the corner site (0, 0, 0) */
    double P_in, P_out; /* bulk pressures n c_s^2 + (G' e2 / 2) psi(n)^2 */
    double dP;          /* P_in - P_out (> 0 for droplets and bubbles alike) */
    double R_e;         /* equimolar radius from the total mass */
    double R_s;         /* surface of tension: d sigma[R] / dR = 0 */
    double sigma_s;     /* sigma[R_s] = dP R_s / (d - 1) (eq. ExactLaplace) */
    int bubble;         /* 1 if n_in < n_out (b = 1 of the (-1)^b sign) */
} lb_curved_obs;

typedef struct lb_ctx lb_ctx;

/* Human-readable name of a status code (static storage). */
const char *lb_status_str(lb_status s);

/* Last CUDA error string seen by this thread's failing call ("" if none). */
const char *lb_last_cuda_error(void);

/* Fill *p with defaults: D2Q9 64x64x1, FP64, tau 1, G -5, literal G,
 * psi = exp(-1/n), rho0_shift 0.5 (the shift keeps binary32 rounding of
 * both gas, n ~ 0.1-0.6, and liquid, n ~ 1.7-5.5, populations small; it
 * measured 2-5x more accurate than 1.0 on Shan-Chen droplets). */
lb_status lb_params_default(lb_params *p);

/* Expand symmetry groups into the canonical (e,-e) pair list (host only, no
 * GPU needed).  Each group is one base vector (dim ints, row-major in
 * base_vectors) whose orbit under coordinate permutations and sign flips is
 * the group (Sec. III A); W[g] is its weight W(|e|^2).  Pair order: groups by
 * |e|^2, ties by the sorted absolute base components in descending
 * lexicographic order; inside a group the representatives (first non-zero
 * component positive) in descending lexicographic order of (e_x,e_y,e_z).
 * Writes up to max_pairs pairs to pair_vec [3 per pair, z = 0 in 2D] and
 * pair_w, the count to *n_pairs, and moments to *info (either may be NULL).
 * LB_EINVAL: dim not 2/3, n_groups < 1, a zero or repeated group, a
 * component beyond LB_MAX_RADIUS, or more than max_pairs pairs. */
lb_status lb_expand_stencil(int dim, int n_groups, const int *base_vectors,
                            const double *W, int max_pairs, int *pair_vec,
                            double *pair_w, int *n_pairs, lb_stencil_info *info);

/* Create a context: allocate device state and set f_i = f_i^eq(rho, u)
 * (u = 0 if u_init is NULL) on every node (reading: the paper does not state
 * the initial condition; equilibrium at rest is used).  rho_init: host [N]
 * float64; u_init: host [D][N] float64 or NULL.  cuda_stream: a
 * cudaStream_t all work of the context is ordered on, or NULL for a stream
 * the context creates.  On success *out owns device memory until
 * lb_destroy.  LB_EINVAL for bad parameters (checked on the host) or an
 * initial density that is not positive and finite (checked on the device
 * after the upload; nothing is left allocated), LB_ENOMEM, LB_ECUDA. */
lb_status lb_create(const lb_params *p, const double *rho_init,
                    const double *u_init, void *cuda_stream, lb_ctx **out);

/* Free the context's device memory (synchronizes its stream).  NULL is a
 * no-op. */
lb_status lb_destroy(lb_ctx *ctx);

/* Set the forcing stencil (eq. sc_f): groups as in lb_expand_stencil.
 * Weights are used as given (no renormalisation).  *info may be NULL.
 * LB_EINVAL for the lb_expand_stencil errors or a radius larger than the
 * lattice allows (each dimension must be >= 1; any radius wraps
 * periodically).  Must be called before lb_step. */
lb_status lb_set_stencil(lb_ctx *ctx, int n_groups, const int *base_vectors,
                         const double *W, lb_stencil_info *info);

/* Advance nsteps >= 0 steps.  Asynchronous on the context's stream: returns
 * once the work is enqueued.  Density checks (n > 0, not NaN) run inside the
 * kernels; a failure is reported by lb_sync / lb_observables as
 * LB_EUNSTABLE with the first failing step in lb_obs.error_step.
 * LB_ESTATE if no stencil is set. */
lb_status lb_step(lb_ctx *ctx, int nsteps);

/* Wait for the context's stream.  LB_EUNSTABLE if a density check failed
 * since lb_create, else LB_OK (or LB_ECUDA). */
lb_status lb_sync(lb_ctx *ctx);

/* Observables of the current state, one fused pass over the populations
 * with binary64 warp-shuffle reductions (compensated double-double sums in a
 * fixed order, rounded once): mass, momentum sum(j + F/2), max |u|, min/max
 * n.  Binary64 lattices: every node quantity in binary64.  Shifted-binary32
 * lattices: the mass from each node's widened density (to 2^-47 relative),
 * F, u and j + F/2 in binary32 (the step's precision), the sums in binary64.
 * Shifted-binary32 D3Q19 lattices on the TMA step kernel are measured by
 * that kernel's measuring instantiation (one read of the populations, psi
 * never stored; the node sums compensated in binary32 pairs before the
 * binary64 reduction; min/max n are the step's binary32 densities); the
 * others by a generic pass that reads psi from a halo'd copy (min/max n
 * widened).  Synchronous; allocates nothing (the per-block records go to
 * the idle population buffer or the context's reduction buffer).  Returns
 * LB_EUNSTABLE (with *out filled) if a density check failed, LB_ECUDA if a
 * bounded wait of the measuring pass gave up. */
lb_status lb_observables(lb_ctx *ctx, lb_obs *out);

/* Lattice pressure tensor (Appendices E and F) including the ideal part
 * n c_s^2 delta, evaluated in binary64 from the current state.  out: host
 * [C][N] float64, C = 3 (xx, xy, yy) in 2D or 6 (xx, xy, xz, yy, yz, zz) in
 * 3D.  Groups covered: regular (k,0[,0]), (k,k[,0]), (k,k,k) for k <= 4 and
 * the irregular (2,1[,0]), (2,1,1), (2,2,1); others give LB_EUNSUPPORTED.
 * Synchronous. */
lb_status lb_pressure_tensor(lb_ctx *ctx, double *out);

/* Interfaces of a flat periodic slab with gradients along x (Sec. III B,
 * Sec. IV): the line integrals of the binary64 lattice pressure tensor over
 * each interface's window -- sigma_0 (eq. sigma0pnpt), z_s (eq. ZSDef), z_e
 * and the Tolman length delta = z_e - z_s (eq. zemzs), and Gamma(z_s) /
 * (n_l - n_g) (eq. deltaads) -- computed on the device.  An interface lies
 * between x and x + 1 where the y(z)-averaged density crosses
 * (n_max + n_min) / 2.  out: host array of max_interfaces entries (filled in
 * increasing x); *n_found: interfaces found (may exceed max_interfaces).
 * Synchronous; allocates nothing (staging in the context's idle population
 * buffer).  LB_EUNSUPPORTED for stencil groups outside Appendices E/F,
 * LB_EINVAL for bad arguments or a lattice too narrow to stage the
 * profiles. */
lb_status lb_flat_interfaces(lb_ctx *ctx, int max_interfaces, lb_flat_obs *out,
                             int *n_found);

/* One droplet or bubble at rest centred at center (x, y[, z]; host, 2 or 3
 * doubles, any real coordinates inside the box) (Sec. III B, Sec. V B):
 * n_in at the centre, n_out at the corner site, their bulk pressures, the
 * equimolar radius R_e (pi R_e^2 n_in + (L^2 - pi R_e^2) n_out = M, or the
 * 3D analogue), and the surface of tension: along the x axis through the
 * centre, with P_T = P^yy linear between the site samples on each ray (+x
 * and -x, averaged) from r = 0 to L/2, the generalized surface tension
 * sigma[R] = R^(1-d) int r^(d-1) (P_J(r; R) - P_T(r)) dr equals
 * C R^(1-d) + dP R / d; its stationary point is R_s^d = d (d-1) C / dP with
 * sigma_s = dP R_s / (d - 1).  All in binary64 on the device.  Synchronous;
 * allocates nothing.  LB_EUNSUPPORTED for stencil groups outside
 * Appendices E/F; LB_EINVAL for bad arguments. */
lb_status lb_curved_interface(lb_ctx *ctx, const double *center, lb_curved_obs *out);

/* The Laplace law over droplets and bubbles (Sec. V B): least-squares line
 * through ((-1)^b / R_e, (-1)^b dP) of n results; *sigma = slope / (d - 1),
 * *intercept its intercept.  Host arithmetic; LB_EINVAL for n < 2. */
lb_status lb_fit_laplace(const lb_curved_obs *runs, int n, int dim, double *sigma,
                         double *intercept);

/* The Tolman length from droplets and bubbles (Sec. III B): least-squares
 * line through ((-1)^b / R_s, dP R_s / ((d - 1) sigma0)) whose slope is
 * -(d - 1) delta; writes *delta and the line's intercept (1 for an exact
 * first-order expansion).  Host arithmetic; LB_EINVAL for n < 2. */
lb_status lb_fit_tolman(const lb_curved_obs *runs, int n, int dim, double sigma0,
                        double *delta, double *intercept);

/* Density [N] and velocity u = (j + F/2)/n [D][N] of the current state
 * (either pointer may be NULL).  Synchronous. */
lb_status lb_get_fields(lb_ctx *ctx, double *rho, double *u);

/* Current populations f_i(x) as float64 [Q][N] (FP32 states are widened and
 * the shift w_i rho0 added back).  Synchronous. */
lb_status lb_get_state(lb_ctx *ctx, double *f);

/* Replace the populations with f [Q][N] float64 (rounded to binary32 after
 * removing the shift in FP32 mode).  Synchronous. */
lb_status lb_set_state(lb_ctx *ctx, const double *f);

/* Diagnostic: y[k] = RN(exp(x[k])) for k < n, evaluated on the GPU by the
 * same correctly rounded binary64 exp the FP64 step uses.  Host arrays.
 * Synchronous.  *n_ambiguous (may be NULL) receives the number of inputs
 * whose rounding could not be certified. */
lb_status lb_exp_cr(const double *x, double *y, long long n,
                    long long *n_ambiguous);

/* Diagnostic: psi[k] = psi(n_in[k]) for k < n in binary64, by the step's own
 * device code (psi_kind as in lb_params; n_in[k] > 0).  Host arrays.
 * Synchronous.  *n_ambiguous (may be NULL): roundings not certified. */
lb_status lb_psi_eval(int psi_kind, double psi_eps, const double *n_in, double *psi,
                      long long n, long long *n_ambiguous);

/* Number of kernels this context has launched (for launch accounting). */
long long lb_kernel_launches(const lb_ctx *ctx);

/* Raw device counters of the context, read after the stream's work is done
 * (synchronous), without judging them: out[0] the first step whose density
 * check failed (-1: none), out[1] the steps the device has completed (the
 * last block of each step advances it, also in a step whose waits gave up),
 * out[2] binary64 roundings of psi that were not certified, out[3] blocks
 * counted in the current fused step (0 between steps), out[4] mbarrier
 * waits of the TMA kernel that gave up (sticky: every later lb_sync and
 * lb_observables reports LB_ECUDA).  Diagnostics; LB_EINVAL for NULL. */
lb_status lb_device_counters(lb_ctx *ctx, long long out[5]);

/* Options of lb_set_option. */
enum {
    LB_OPT_FUSED = 1,   /* 1 (default): shifted-FP32 steps use the fused
                           single-pass kernels: D3Q19 when the stencil's
                           groups are among the E8 groups and each dimension
                           is >= 8, D2Q9 when they are among the 2D groups
                           up to (2,2) and each dimension is >= 4 (either
                           pseudopotential, either forcing variant);
                           0: always the two-kernel path */
    LB_OPT_ZCHUNK = 2,  /* z planes marched by one CTA of the fused kernel
                           (default 28) */
    LB_OPT_TMA = 3,     /* 1 (default): on lattices with nx % 32 == 0,
                           ny % 8 == 0, nz >= 8 the fused kernel stages planes
                           with TMA; 0: with per-thread cp.async */
    LB_OPT_WAIT_POLLS = 5 /* bound on the tries of each mbarrier wait of the
                           TMA kernel (default 2^26, range 0 .. 2^40).  A
                           block whose wait runs out records it, lets its
                           copies land and skips the rest of the step; the
                           next lb_sync returns LB_ECUDA.  0 makes every
                           wait give up at once (for testing that path); the
                           state after such a step is not meaningful */
};

/* Set an option of the context.  LB_EINVAL for an unknown option or value. */
lb_status lb_set_option(lb_ctx *ctx, int option, long long value);

/* 0 if lb_step runs the two-kernel path, 1 the fused single-pass D3Q19
 * kernel with cp.async staging, 2 the fused D3Q19 kernel with TMA staging,
 * 3 the fused single-pass D2Q9 kernel (shifted FP32, stencils on the 2D
 * groups up to (2,2)). */
int lb_fused_active(const lb_ctx *ctx);

/* Kernel kinds of the step, for lb_timing_read. */
enum { LB_KERNEL_PSI = 0, LB_KERNEL_COLLIDE = 1, LB_KERNEL_FUSED = 2, LB_KERNEL_OTHER = 3,
       LB_KERNEL_KINDS = 4 };

/* Per-kernel timing: enable = 1 resets the accumulators and brackets every
 * subsequent step kernel with CUDA events recorded on the context's stream;
 * enable = 0 stops recording (accumulators are kept). */
lb_status lb_timing(lb_ctx *ctx, int enable);

/* Wait for the stream and return, per kernel kind, the summed device time
 * in milliseconds (ms[LB_KERNEL_KINDS]) and the number of launches timed
 * (launches[LB_KERNEL_KINDS]); either pointer may be NULL. */
lb_status lb_timing_read(lb_ctx *ctx, double *ms, long long *launches);

/* ---- batches of independent 2D lattices ------------------------------------
 *
 * The droplet and bubble runs of a Laplace / Tolman fit (Sec. V B) are many
 * independent lattices of uneven size.  A batch steps them together: one
 * launch per step covers every tile of every member (a grid of resident CTAs
 * walking one tile table), and lb_batch_step replays a CUDA graph of 64 such
 * launches.  Results are those of lb_step on each member (the same fused
 * D2Q9 kernel), whatever the tile shape.
 *
 * Members are contexts created by lb_create: D2Q9, LB_FP32_SHIFTED, stencil
 * set, every group among (1,0), (1,1), (2,0), (2,1), (2,2) (E4, E6, E8 and
 * their tuned variants), either pseudopotential and either forcing variant
 * (a batch whose members differ in these runs a kernel that picks per
 * member, slower than the one a uniform batch runs); LB_EUNSUPPORTED
 * otherwise, LB_ESTATE if a stencil is missing, LB_EINVAL for a repeated or
 * NULL member.  The batch borrows
 * the members (their buffers, counters and host step counts advance with
 * lb_batch_step); destroy the batch before any member.  A member may still
 * be used on its own between batch calls: lb_batch_step orders itself after
 * the work already queued on every member's stream, and the members' later
 * work after it.  cuda_stream (NULL: a stream of the batch's own) carries the
 * batch's launches. */
typedef struct lb_batch lb_batch;

lb_status lb_batch_create(lb_ctx *const *ctxs, int n, void *cuda_stream, lb_batch **out);
lb_status lb_batch_destroy(lb_batch *batch);

/* Advance every member by nsteps (asynchronous). */
lb_status lb_batch_step(lb_batch *batch, int nsteps);

/* Wait for the batch and check every member as lb_sync does; returns the
 * first member status that is not LB_OK. */
lb_status lb_batch_sync(lb_batch *batch);

/* Kernel launches lb_batch_step has issued (one per step). */
long long lb_batch_launches(const lb_batch *batch);

/* Tile shapes: lb_batch_tile_count() candidates, index -> (tx, ty) nodes. */
int lb_batch_tile_count(void);
lb_status lb_batch_tile_shape(int index, int *tx, int *ty);
lb_status lb_batch_set_tile(lb_batch *batch, int index);
int lb_batch_get_tile(const lb_batch *batch);

/* Autotuner: time steps_per_trial steps (rounded down to even, >= 2) with
 * every tile shape, keep the fastest.  The members' states and counters are
 * saved first and restored after each trial, so tuning does not advance the
 * simulation.  ms_out (NULL or lb_batch_tile_count() doubles) receives the
 * trial times.  Synchronous; allocates a copy of every member's state. */
lb_status lb_batch_tune(lb_batch *batch, int steps_per_trial, double *ms_out);

/* ---- adjoint: gradients of the surface tension ------------------------------
 *
 * The discrete adjoint of lb_step in binary64 (eqs. lbm, omega_i, f_eq,
 * GuoForcing, sc_f read backwards), for gradients of the flat-interface
 * surface tension sigma_0 (Sec. V A; the Appendix E pressure tensor summed
 * over the lattice is (G'/2) sum_x psi(x) sum_e W(e) psi(x+e)(e_x^2 - e_y^2))
 * or of any loss whose gradient with respect to the state the caller
 * supplies.  An adjoint belongs to one context (any lattice, precision,
 * pseudopotential and forcing: Guo's, or the F^2 variant, whose extra source
 * -cw_i (A/tau)(4.5 (xi.F)^2 - 1.5 F.F) adds -cw_i (A/tau)(9 (xi.F) xi - 3 F)
 * to dS_i/dF); its adjoint variable lam = dL/d(state) has the layout of
 * lb_get_state.
 *
 * Typical use, with checkpoints every K steps (a checkpoint is lb_get_state
 * / lb_set_state):  step forward saving checkpoints; lb_adjoint_seed_sigma
 * (or lb_adjoint_set) at the final state; then for each segment, last first:
 * lb_set_state(checkpoint); lb_adjoint_run(K).  lb_adjoint_run recomputes
 * the segment's forward steps with the context's own step (the context ends
 * K steps later), records the states in binary64 (K [Q][N] arrays of device
 * memory) and carries lam back to the checkpoint, adding the segment's terms
 * to the gradients.  lb_adjoint_gradient returns dL/dW for each stencil group
 * (the order of lb_set_stencil) and dL/dG; sums are in a fixed order, so
 * results are reproducible. */
typedef struct lb_adjoint lb_adjoint;

lb_status lb_adjoint_create(lb_ctx *ctx, lb_adjoint **out);
lb_status lb_adjoint_destroy(lb_adjoint *adj);
/* lam := host array [Q][N] (NULL: zero). */
lb_status lb_adjoint_set(lb_adjoint *adj, const double *lam);
lb_status lb_adjoint_get(lb_adjoint *adj, double *lam);
/* Clear the accumulated parameter gradients. */
lb_status lb_adjoint_zero_grad(lb_adjoint *adj);
/* sigma_0 of the context's current state (a flat slab with gradients along
 * x and n_interfaces interfaces): writes *sigma (may be NULL), sets lam =
 * dsigma/d(state) and adds sigma's explicit dependence on W and G to the
 * gradients. */
lb_status lb_adjoint_seed_sigma(lb_adjoint *adj, int n_interfaces, double *sigma);
/* Add the gradient of L_m = sum_x m(x) (P_xx - P_yy)(x) to lam, for site
 * weights m (host array [N], the layout of one field of lb_get_fields): the
 * normal minus a tangential component of the lattice pressure tensor of a
 * slab with gradients along x (Appendices E/F; the ideal part cancels).
 * Writes *value = L_m (may be NULL) and adds L_m's explicit dependence on W
 * and G to the gradients.  Used with lb_adjoint_set for losses built from
 * the density and the tensor together, e.g. the Tolman length
 * z_e - z_s of a flat interface.  LB_EUNSUPPORTED for stencil groups
 * outside Appendices E/F. */
lb_status lb_adjoint_seed_pt(lb_adjoint *adj, const double *m, double *value);
/* Quantities of a flat slab (gradients along x) for lb_adjoint_seed_flat. */
enum {
    LB_FLAT_SIGMA = 0,  /* sigma_0: sum over the line of P_N - P_T / #interfaces (eq. sigma0pnpt) */
    LB_FLAT_DELTA = 1,  /* Tolman length z_e - z_s, mean over the interfaces (eqs. zemzs, SCTolmanFlat) */
    LB_FLAT_WIDTH = 2,  /* 6 sum_x (n - n_g)(n_l - n) / (n_l - n_g)^2 / #interfaces (n: y(z)-mean
                           profile; equals w for a tanh profile of width w); params: n_l, n_g,
                           #interfaces (<= 0: the number found) */
    LB_FLAT_RATIO = 3   /* n(x_l) / n(x_g) of the profile; params: x_l, x_g (columns) */
};

/* Add weight * dQ/d(state) to lam, and weight * Q's explicit dependence on W
 * and G to the gradients, for one quantity Q of the current state of a flat
 * slab: the profiles of n and P_N - P_T (y(z) means, binary64 lattice
 * pressure tensor, Appendices E/F), the interface windows and Q and its
 * per-column derivatives are formed on the device (the windows and
 * integrals of lb_flat_interfaces).  The density part seeds lam through
 * n = sum_i f_i, the tensor part through the adjoint of the per-site
 * tensor (as lb_adjoint_seed_pt).  Seeds add up, so several quantities
 * with weights g_k give the gradient of sum_k g_k Q_k in one lb_adjoint_run
 * sweep.  *value (may be NULL) receives Q (not weighted).  params: host
 * doubles as listed above (may be NULL for SIGMA, DELTA).  LB_EINVAL for a
 * bad quantity or parameters or a state without an interface;
 * LB_EUNSUPPORTED for stencil groups outside Appendices E/F. */
lb_status lb_adjoint_seed_flat(lb_adjoint *adj, int quantity, const double *params, double weight,
                               double *value);
/* Carry lam back over the next nsteps steps of the context (see above). */
lb_status lb_adjoint_run(lb_adjoint *adj, int nsteps);
/* dL/dW per stencil group (n_groups doubles, may be NULL) and dL/dG. */
lb_status lb_adjoint_gradient(lb_adjoint *adj, double *dW, double *dG);

/* Largest lattice (nodes) lb_step_fp64_static accepts: 2^20, i.e. a fixed
 * 8 MiB of device memory (plus 64 bytes of counters) per GPU. */
#define LB_STATIC_MAX_NODES (1LL << 20)

/* One binary64 step that allocates nothing.  This entry point has no
 * counterpart in the paper; it exists for callers that cannot allocate device
 * memory where they step a lattice -- code running under another framework's
 * memory pool that forbids direct cudaMalloc, latency-critical loops where an
 * allocation or the synchronisation it can imply is not acceptable, or
 * embeddings that may only use buffers they already own.
 *
 * The caller owns both population buffers: f_in and f_out are device arrays
 * [Q][N] float64 in the state layout of lb_get_state (post-streaming
 * populations, x fastest); f_out receives the populations one step later.
 * They must not overlap.  The stencil is given as the canonical pair list of
 * lb_expand_stencil (n_pairs vectors of 3 ints in pair_vec and their weights
 * in pair_w, host arrays).  lattice, nx, ny, nz, tau, G and g_convention mean
 * what they mean in lb_params.  The arithmetic and rounding order are those
 * of lb_step in LB_FP64 mode, so results are identical bit for bit.  Work is
 * enqueued on cuda_stream (NULL: the legacy default stream) and the call
 * returns without waiting.  Nothing is reported back: neither the density
 * check (n <= 0 or NaN) nor the count of binary64 exp roundings the step
 * could not certify (which lb_observables reports as exp_ambiguous for a
 * context); a caller that needs either steps a context with lb_step.
 *
 * The only scratch, the lattice's psi field and a few counters, lives in one
 * array of fixed size compiled into the library (LB_STATIC_MAX_NODES nodes):
 * every GPU that loads the library holds it until the process exits.  The
 * first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that tears down and recreates the
 * device's primary context) the kept address is stale, so do not call this
 * entry point again in that process.  All calls on a device share the array and it keeps the last
 * call's contents: each call clears its counters and overwrites psi before
 * use, but two calls that overlap on the GPU (different streams, or
 * concurrent host threads) race on it and must be serialised by the caller.
 *
 * LB_EINVAL for bad arguments, for f_in == f_out, or for more than
 * LB_STATIC_MAX_NODES nodes (with a message in lb_last_cuda_error);
 * LB_ECUDA if a CUDA call fails. */
lb_status lb_step_fp64_static(int lattice, int nx, int ny, int nz, double tau, double G,
                              int g_convention, int n_pairs, const int *pair_vec,
                              const double *pair_w, const double *f_in, double *f_out,
                              void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SCLBM_H */
