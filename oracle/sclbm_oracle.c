/*
 * sclbm_oracle.c -- plain, slow FP64 CPU oracle of the Shan-Chen
 * lattice-Boltzmann step with an extended forcing stencil
 * (Lulli & Ching, "Higher-order Tuning of Interface Physics in Multiphase
 * Lattice Boltzmann").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline / reference leg may load this code.  It shares no
 * source with the CUDA library and must never be called from the product.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math: IEEE
 * round-to-nearest, no contraction of a*b+c into an FMA).
 *
 * One step, for every node x of a fully periodic nx*ny*nz lattice, follows
 * the paper's model statement in its order:
 *   1. n = sum_i f_i                                  (Sec. II, density)
 *   2. psi = psi(n), psi = exp(-1/n)                   (Sec. IV B, eq. psieps)
 *   3. F = -G' psi(x) sum_a W_a psi(x+e_a) e_a         (eq. sc_f)
 *   4. j = sum_i f_i xi_i;  u = (j + F/2)/n            (Sec. II, shifted u)
 *   5. f_eq from the 2nd-order Hermite expansion       (eq. f_eq)
 *   6. S_i Guo forcing, T = 2 u F                      (eq. GuoForcing)
 *      or, with the F^2 variant, T = 2 u F - (A/tau) F F    (Sec. VI, Appendix
 *      on eps and e4: the tensor of eq. GuoForcing with an F F term)
 *   7. f*_i = f_i - (f_i - f_eq_i)/tau + S_i           (eqs. lbm, omega_i)
 *   8. f_i(x + xi_i) <- f*_i(x)                        (eq. lbm, streaming)
 * G' = G (literal convention, force without c_s^2) or G/3 (the paper's
 * eq. sc_f with c_s^2 = 1/3).  c_s^2 = 1/3 enters as the exact constants
 * 1/c_s^2 = 3, 1/(2c_s^4) = 9/2, c_s^2/(2c_s^4) = 3/2, 1/c_s^4 = 9.
 *
 * Rounding order (a reading the paper leaves open; the CUDA path follows
 * the same order so FP64 results agree bit for bit):
 *   - sums over i run in the velocity-table order below, left to right;
 *   - the symmetric stencil sum is taken over (e, -e) pairs in the
 *     canonical order supplied by the caller:  acc += (W*(psi(x+e) -
 *     psi(x-e))) * e^mu;  F^mu = (-G' * psi(x)) * acc^mu;
 *   - psi = RN(exp(RN(-1/n))) with exp correctly rounded (evaluated in
 *     binary128 and rounded once to binary64);
 *   - 1/tau and (1 - 1/(2 tau)) w_i are formed once; the collision is
 *     f* = (f - (1/tau)*(f - f_eq)) + S.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 and D3Q19 velocity tables (Sec. II, "DdQq"); index order is part of
 * the state layout. */
static const int C9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const int C19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
    int D, Q, nx, ny, nz;
    long N;
    const int (*c)[3];
    double w[19];
} grid_t;

static int make_grid(grid_t *g, int D, int Q, int nx, int ny, int nz) {
    if (!((D == 2 && Q == 9 && nz == 1) || (D == 3 && Q == 19))) return -1;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    g->D = D; g->Q = Q; g->nx = nx; g->ny = ny; g->nz = nz;
    g->N = (long)nx * ny * nz;
    if (Q == 9) {
        g->c = C9;
        g->w[0] = 4.0 / 9.0;
        for (int i = 1; i <= 4; i++) g->w[i] = 1.0 / 9.0;
        for (int i = 5; i <= 8; i++) g->w[i] = 1.0 / 36.0;
    } else {
        g->c = C19;
        g->w[0] = 1.0 / 3.0;
        for (int i = 1; i <= 6; i++) g->w[i] = 1.0 / 18.0;
        for (int i = 7; i <= 18; i++) g->w[i] = 1.0 / 36.0;
    }
    return 0;
}

static long wrap(long a, long n) { long r = a % n; return r < 0 ? r + n : r; }

static long site(const grid_t *g, long x, long y, long z) {
    return (wrap(z, g->nz) * g->ny + wrap(y, g->ny)) * g->nx + wrap(x, g->nx);
}

/* Pseudopotential.  kind 0: psi = exp(-1/n) (Sec. IV B, e4 = 1/3 case).
 * kind 1: psi_eps = (n/(eps+n))^(1/eps) (eq. psieps), read as
 * RN(RN(n/RN(eps+n)) ^ RN(1/eps)) with a correctly rounded power. */
double or_psi(double n, int kind, double eps) {
    if (kind == 0) {
        double a = -1.0 / n;
        return (double)expf128((_Float128)a);
    }
    double r = n / (eps + n);
    double e = 1.0 / eps;
    return (double)powf128((_Float128)r, (_Float128)e);
}

double or_exp_cr(double a) { return (double)expf128((_Float128)a); }

/* n(x) = sum_i f_i(x), in table order. */
static void density(const grid_t *g, const double *f, double *n) {
    for (long s = 0; s < g->N; s++) {
        double acc = f[s];
        for (int i = 1; i < g->Q; i++) acc = acc + f[(long)i * g->N + s];
        n[s] = acc;
    }
}

/* F^mu(x) = (-G' psi(x)) * sum_pairs (W (psi(x+e) - psi(x-e))) e^mu. */
static void force_at(const grid_t *g, const double *psi, long x, long y, long z,
                     int npairs, const int *vec, const double *w, double mGp,
                     double F[3]) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < npairs; a++) {
        const int *e = vec + 3 * a;
        double pp = psi[site(g, x + e[0], y + e[1], z + e[2])];
        double pm = psi[site(g, x - e[0], y - e[1], z - e[2])];
        double t = w[a] * (pp - pm);
        for (int mu = 0; mu < g->D; mu++) acc[mu] = acc[mu] + t * (double)e[mu];
    }
    double pre = mGp * psi[site(g, x, y, z)];
    for (int mu = 0; mu < 3; mu++) F[mu] = (mu < g->D) ? pre * acc[mu] : 0.0;
}

/* Collision of one node: populations fi[Q] (post-streaming), density nn,
 * force F -> post-collision fo[Q].  Also returns j + F/2 and u if asked. */
/* kA = A/tau of the F^2 variant (0: Guo's T = 2 u F).  The source is
 * S_i = cw_i [xi.F/cs2 + (xi xi - cs2 1):T/(2 cs2^2)] with cs2 = 1/3:
 *   T = 2uF:        cw_i ((3 cF + 9 cu cF) - 3 u.F)
 *   - (A/tau) F F:  - cw_i kA (4.5 cF^2 - 1.5 F.F)                         */
static void collide_node(const grid_t *g, const double *fi, double nn,
                         const double F[3], double omega, const double *cw, double kA,
                         double *fo, double *mom, double *uout) {
    double j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < g->Q; i++)
        for (int mu = 0; mu < g->D; mu++)
            j[mu] = j[mu] + fi[i] * (double)g->c[i][mu];
    double u[3] = {0.0, 0.0, 0.0};
    for (int mu = 0; mu < g->D; mu++) {
        double m = j[mu] + 0.5 * F[mu];
        if (mom) mom[mu] = m;
        u[mu] = m / nn;
        if (uout) uout[mu] = u[mu];
    }
    double uu = u[0] * u[0];
    double uF = u[0] * F[0];
    double FF = F[0] * F[0];
    for (int mu = 1; mu < g->D; mu++) {
        uu = uu + u[mu] * u[mu];
        uF = uF + u[mu] * F[mu];
        FF = FF + F[mu] * F[mu];
    }
    for (int i = 0; i < g->Q; i++) {
        double cu = (double)g->c[i][0] * u[0];
        double cF = (double)g->c[i][0] * F[0];
        for (int mu = 1; mu < g->D; mu++) {
            cu = cu + (double)g->c[i][mu] * u[mu];
            cF = cF + (double)g->c[i][mu] * F[mu];
        }
        double feq = (g->w[i] * nn) * (((1.0 + 3.0 * cu) + 4.5 * (cu * cu)) - 1.5 * uu);
        double S = kA != 0.0
            ? cw[i] * (((3.0 * cF + 9.0 * (cu * cF)) - 3.0 * uF) - kA * (4.5 * (cF * cF) - 1.5 * FF))
            : cw[i] * ((3.0 * cF + 9.0 * (cu * cF)) - 3.0 * uF);
        fo[i] = (fi[i] - omega * (fi[i] - feq)) + S;
    }
}

static void constants(const grid_t *g, double tau, double *omega, double *cw) {
    *omega = 1.0 / tau;
    double pref = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < g->Q; i++) cw[i] = pref * g->w[i];
}

/* f: [Q][N] post-streaming populations, advanced nsteps in place.
 * Returns 0, or -1 on bad arguments, -2 on allocation failure, or
 * 1 + (first step) at which a node had n <= 0 or NaN (the step still runs). */
int or_step(int D, int Q, int nx, int ny, int nz, double *f, int npairs,
            const int *vec, const double *w, double tau, double Gp,
            int psi_kind, double psi_eps, int nsteps, double forcing_A) {
    grid_t g;
    if (make_grid(&g, D, Q, nx, ny, nz)) return -1;
    double *n = malloc(sizeof(double) * g.N);
    double *psi = malloc(sizeof(double) * g.N);
    double *fn = malloc(sizeof(double) * g.N * g.Q);
    if (!n || !psi || !fn) { free(n); free(psi); free(fn); return -2; }
    double omega, cw[19];
    constants(&g, tau, &omega, cw);
    const double kA = forcing_A / tau;
    double mGp = -Gp;
    int bad = 0;
    for (int t = 0; t < nsteps; t++) {
        density(&g, f, n);
        for (long s = 0; s < g.N; s++) {
            if (!(n[s] > 0.0) && !bad) bad = 1 + t;
            psi[s] = or_psi(n[s], psi_kind, psi_eps);
        }
        for (long z = 0; z < nz; z++)
            for (long y = 0; y < ny; y++)
                for (long x = 0; x < nx; x++) {
                    long s = site(&g, x, y, z);
                    double F[3], fi[19], fo[19];
                    force_at(&g, psi, x, y, z, npairs, vec, w, mGp, F);
                    for (int i = 0; i < g.Q; i++) fi[i] = f[(long)i * g.N + s];
                    collide_node(&g, fi, n[s], F, omega, cw, kA, fo, NULL, NULL);
                    for (int i = 0; i < g.Q; i++) {
                        long d = site(&g, x + g.c[i][0], y + g.c[i][1], z + g.c[i][2]);
                        fn[(long)i * g.N + d] = fo[i];
                    }
                }
        memcpy(f, fn, sizeof(double) * g.N * g.Q);
    }
    free(n); free(psi); free(fn);
    return bad;
}

/* Fields of the current state: n, psi, F [D][N], j + F/2 [D][N], u [D][N]. */
int or_fields(int D, int Q, int nx, int ny, int nz, const double *f, int npairs,
              const int *vec, const double *w, double Gp, int psi_kind,
              double psi_eps, double *n, double *psi, double *F, double *mom,
              double *u) {
    grid_t g;
    if (make_grid(&g, D, Q, nx, ny, nz)) return -1;
    density(&g, f, n);
    for (long s = 0; s < g.N; s++) psi[s] = or_psi(n[s], psi_kind, psi_eps);
    double omega, cw[19];
    constants(&g, 1.0, &omega, cw);
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long s = site(&g, x, y, z);
                double Fs[3], fi[19], fo[19], m[3], us[3];
                force_at(&g, psi, x, y, z, npairs, vec, w, -Gp, Fs);
                for (int i = 0; i < g.Q; i++) fi[i] = f[(long)i * g.N + s];
                collide_node(&g, fi, n[s], Fs, omega, cw, 0.0, fo, m, us);
                for (int mu = 0; mu < D; mu++) {
                    F[(long)mu * g.N + s] = Fs[mu];
                    mom[(long)mu * g.N + s] = m[mu];
                    u[(long)mu * g.N + s] = us[mu];
                }
            }
    return 0;
}

/* Post-collision populations of one node (x,y,z), computed from the full
 * post-streaming field f with psi evaluated on the fly where needed.  Used
 * to check sampled nodes of a large lattice one by one. */
int or_node_post(int D, int Q, int nx, int ny, int nz, const double *f, long x,
                 long y, long z, int npairs, const int *vec, const double *w,
                 double tau, double Gp, int psi_kind, double psi_eps,
                 double *out, double forcing_A) {
    grid_t g;
    if (make_grid(&g, D, Q, nx, ny, nz)) return -1;
    double omega, cw[19];
    constants(&g, tau, &omega, cw);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < npairs; a++) {
        const int *e = vec + 3 * a;
        long sp = site(&g, x + e[0], y + e[1], z + e[2]);
        long sm = site(&g, x - e[0], y - e[1], z - e[2]);
        double np = f[sp], nm = f[sm];
        for (int i = 1; i < Q; i++) {
            np = np + f[(long)i * g.N + sp];
            nm = nm + f[(long)i * g.N + sm];
        }
        double t = w[a] * (or_psi(np, psi_kind, psi_eps) - or_psi(nm, psi_kind, psi_eps));
        for (int mu = 0; mu < D; mu++) acc[mu] = acc[mu] + t * (double)e[mu];
    }
    long s = site(&g, x, y, z);
    double fi[19];
    for (int i = 0; i < Q; i++) fi[i] = f[(long)i * g.N + s];
    double nn = fi[0];
    for (int i = 1; i < Q; i++) nn = nn + fi[i];
    double pre = (-Gp) * or_psi(nn, psi_kind, psi_eps);
    double F[3] = {0.0, 0.0, 0.0};
    for (int mu = 0; mu < D; mu++) F[mu] = pre * acc[mu];
    collide_node(&g, fi, nn, F, omega, cw, forcing_A / tau, out, NULL, NULL);
    return 0;
}

/* Equilibrium initial state: f_i = f_eq_i(rho, u) (u may be NULL = 0). */
int or_init_feq(int D, int Q, int nx, int ny, int nz, const double *rho,
                const double *u, double *f) {
    grid_t g;
    if (make_grid(&g, D, Q, nx, ny, nz)) return -1;
    for (long s = 0; s < g.N; s++) {
        double us[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int mu = 0; mu < D; mu++) us[mu] = u[(long)mu * g.N + s];
        double uu = us[0] * us[0];
        for (int mu = 1; mu < D; mu++) uu = uu + us[mu] * us[mu];
        for (int i = 0; i < Q; i++) {
            double cu = (double)g.c[i][0] * us[0];
            for (int mu = 1; mu < D; mu++) cu = cu + (double)g.c[i][mu] * us[mu];
            f[(long)i * g.N + s] =
                (g.w[i] * rho[s]) * (((1.0 + 3.0 * cu) + 4.5 * (cu * cu)) - 1.5 * uu);
        }
    }
    return 0;
}

static long igcd(long a, long b) {
    a = labs(a); b = labs(b);
    while (b) { long t = a % b; a = b; b = t; }
    return a;
}

/* Lattice pressure tensor (Appendices E and F), with the ideal part
 * n c_s^2 delta = (n/3) delta.  Components: 2D xx,xy,yy; 3D xx,xy,xz,yy,yz,zz.
 *
 * Restatement of the appendices' group formulas, one rule per group kind
 * (reading; every printed term of both appendices is of this form, with the
 * (2,2,-1) line of Appendix F read with psi_{1,1,0} in place of the printed
 * psi_{-1,1,0}, the only factor whose offset does not match its vector):
 *   - regular groups (all non-zero components of e equal in size: (k,0,0),
 *     (k,k,0), (k,k,k)), e = m * ehat with ehat primitive: the link
 *     (y, y+e) gives G' W psi(y)psi(y+e) e e, shared as 1/(2m) to each end
 *     and 1/m to each of the m-1 interior sites;
 *   - irregular groups (2,1,0), (2,1,1), (2,2,1) (m = 1): 1/4 to each end
 *     and 1/(2 k) to each of the k = 2^(odd components) sites nearest the
 *     link's midpoint.
 * Per pair e (with -e): s = W * (kA*psi(x)(psi(x+e)+psi(x-e)) + kB*B),
 * B the sum of the interior / midpoint link products in the order
 * j = 1..m-1 (regular) or midpoint offsets +1/2 before -1/2 per odd
 * component, axis by axis (irregular); kA = G'/(2m) or G'/4,
 * kB = G'/m or G'/(2k); then P^{mu nu} += s * e^mu e^nu.
 * Returns 0, -1 on bad grid, -3 for a group the appendices do not cover. */
int or_pressure_tensor(int D, int nx, int ny, int nz, const double *n,
                       const double *psi, int npairs, const int *vec,
                       const double *w, double Gp, double *P) {
    grid_t g;
    if (make_grid(&g, D, D == 2 ? 9 : 19, nx, ny, nz)) return -1;
    int nc = D == 2 ? 3 : 6;
    int cmu[6], cnu[6];
    if (D == 2) { int a[3] = {0, 0, 1}, b[3] = {0, 1, 1}; for (int k = 0; k < 3; k++) { cmu[k] = a[k]; cnu[k] = b[k]; } }
    else { int a[6] = {0, 0, 0, 1, 1, 2}, b[6] = {0, 1, 2, 1, 2, 2}; for (int k = 0; k < 6; k++) { cmu[k] = a[k]; cnu[k] = b[k]; } }
    /* classify pairs */
    for (int a = 0; a < npairs; a++) {
        const int *e = vec + 3 * a;
        int mags[3] = {abs(e[0]), abs(e[1]), abs(e[2])};
        int mx = 0, nzc = 0, alleq = 1, ref = -1;
        for (int k = 0; k < 3; k++) {
            if (mags[k]) { nzc++; if (ref < 0) ref = mags[k]; else if (mags[k] != ref) alleq = 0; }
            if (mags[k] > mx) mx = mags[k];
        }
        if (alleq) { if (mx > 4) return -3; continue; }
        /* irregular: must be a permutation of (2,1,0), (2,1,1), (2,2,1) */
        int s2 = 0, s1 = 0, s0 = 0;
        for (int k = 0; k < 3; k++) { if (mags[k] == 2) s2++; else if (mags[k] == 1) s1++; else if (mags[k] == 0) s0++; }
        if (!((s2 == 1 && s1 == 1 && s0 == 1) || (s2 == 1 && s1 == 2) || (s2 == 2 && s1 == 1))) return -3;
    }
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                long s = site(&g, x, y, z);
                double Ps[6];
                for (int k = 0; k < nc; k++) Ps[k] = (cmu[k] == cnu[k]) ? n[s] / 3.0 : 0.0;
                double p0 = psi[s];
                for (int a = 0; a < npairs; a++) {
                    const int *e = vec + 3 * a;
                    int mags[3] = {abs(e[0]), abs(e[1]), abs(e[2])};
                    int ref = 0, alleq = 1;
                    for (int k = 0; k < 3; k++)
                        if (mags[k]) { if (!ref) ref = mags[k]; else if (mags[k] != ref) alleq = 0; }
                    double pp = psi[site(&g, x + e[0], y + e[1], z + e[2])];
                    double pm = psi[site(&g, x - e[0], y - e[1], z - e[2])];
                    double A = p0 * (pp + pm);
                    double B = 0.0, kA, kB;
                    if (alleq) {
                        long m = igcd(igcd(e[0], e[1]), e[2]);
                        long h[3] = {e[0] / m, e[1] / m, e[2] / m};
                        for (long j = 1; j < m; j++) {
                            double q1 = psi[site(&g, x - j * h[0], y - j * h[1], z - j * h[2])];
                            double q2 = psi[site(&g, x + (m - j) * h[0], y + (m - j) * h[1], z + (m - j) * h[2])];
                            B = B + q1 * q2;
                        }
                        kA = Gp / (2.0 * (double)m);
                        kB = Gp / (double)m;
                    } else {
                        int odd[3], nodd = 0;
                        for (int k = 0; k < 3; k++) if (mags[k] % 2) odd[nodd++] = k;
                        int nmid = 1 << nodd;
                        for (int b = 0; b < nmid; b++) {
                            long off[3];
                            for (int k = 0; k < 3; k++) off[k] = -e[k] / 2; /* even comps */
                            for (int q = 0; q < nodd; q++) {
                                int k = odd[q];
                                int sgn = ((b >> (nodd - 1 - q)) & 1) ? -1 : 1;
                                off[k] = (sgn - e[k]) / 2;
                            }
                            double q1 = psi[site(&g, x + off[0], y + off[1], z + off[2])];
                            double q2 = psi[site(&g, x + off[0] + e[0], y + off[1] + e[1], z + off[2] + e[2])];
                            B = B + q1 * q2;
                        }
                        kA = Gp / 4.0;
                        kB = Gp / (2.0 * (double)nmid);
                    }
                    double sc = w[a] * (kA * A + kB * B);
                    for (int k = 0; k < nc; k++)
                        Ps[k] = Ps[k] + sc * (double)(e[cmu[k]] * e[cnu[k]]);
                }
                for (int k = 0; k < nc; k++) P[(long)k * g.N + s] = Ps[k];
            }
    return 0;
}

/* Force field F [D][N] from a given psi field (eq. sc_f), for pins that set
 * psi directly. */
int or_force_field(int D, int nx, int ny, int nz, const double *psi, int npairs,
                   const int *vec, const double *w, double Gp, double *F) {
    grid_t g;
    if (make_grid(&g, D, D == 2 ? 9 : 19, nx, ny, nz)) return -1;
    for (long z = 0; z < nz; z++)
        for (long y = 0; y < ny; y++)
            for (long x = 0; x < nx; x++) {
                double Fs[3];
                force_at(&g, psi, x, y, z, npairs, vec, w, -Gp, Fs);
                long s = site(&g, x, y, z);
                for (int mu = 0; mu < D; mu++) F[(long)mu * g.N + s] = Fs[mu];
            }
    return 0;
}
