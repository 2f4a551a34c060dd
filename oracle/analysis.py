"""Oracle: post-processing of lattice fields into interface observables.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Restates, in plain numpy/scipy, the paper's definitions:

* bulk pressure P_b = n c_s^2 + (G' e2 / 2) psi^2          (Sec. III A)
* epsilon(e4) = (6 e4 - 2 e2) / (6 e4 + e2)                 (eq. eps_moments)
* Maxwell-like coexistence: int_{n_g}^{n_l} dn psi'/psi^(eps+1) (p0 - P_b) = 0
  with P_b(n_g) = P_b(n_l) = p0                              (eq. SCMaxwell)
* flat-interface profile slope (dpsi/dx)^2                 (eq. PSIProfile)
* second-order surface tension estimate                     (eq. scsigma)
* analytic SC Tolman length                                 (eq. SCTolmanFlat)
* flat sigma_0 = int (P_N - P_T) dx                         (eq. sigma0pnpt)
* z_s = first moment of P_N - P_T                           (eq. ZSDef)
* z_e from Gamma(z_e) = 0, delta = z_e - z_s                 (eq. zemzs)
* delta = Gamma(z_s) / (n_l - n_g)                          (eq. deltaads)
* equimolar radius R_e and the Laplace fit                  (Sec. V B, Laplace)
* generalized sigma[R], the surface of tension R_s, sigma_s (Sec. III B)
* curved Tolman length from Delta P R_s/((d-1) sigma0) vs 1/R_s (Sec. III B)

Readings where the paper is silent (each used identically by the package's
own post-processing):
* a flat periodic slab has several interfaces; the integrals are lattice sums
  over windows centred on each interface, window borders half way between
  neighbouring interfaces (in bulk);
* site x stands for the cell [x - 1/2, x + 1/2]; n_l and n_g are the measured
  densities at the liquid and gas ends of the window;
* the x axis of a window is oriented from liquid to gas when forming delta
  (the orientation that gives eq. SCTolmanFlat its sign);
* curved interfaces: P_T(r) is P^yy on the x axis through the centre, taken
  at the sites and linear between them (the paper interpolates without
  saying how), both rays (+x, -x) averaged, r from 0 to L/2; n_in is taken
  at the centre, n_out at a corner site; droplets and bubbles share one
  line in (-1)^b Delta P against the signed curvature (-1)^b / R.
"""
from __future__ import annotations

from math import exp

import numpy as np
from scipy import integrate, optimize

CS2 = 1.0 / 3.0


def psi_exp(n):
    return np.exp(-1.0 / np.asarray(n, dtype=np.float64))


def dpsi_exp(n):
    n = np.asarray(n, dtype=np.float64)
    return np.exp(-1.0 / n) / (n * n)


def psi_eps_fn(eps):
    def f(n):
        n = np.asarray(n, dtype=np.float64)
        return (n / (eps + n)) ** (1.0 / eps)

    def df(n):
        n = np.asarray(n, dtype=np.float64)
        return (n / (eps + n)) ** (1.0 / eps) / (n * (eps + n))
    return f, df


def epsilon_of_e4(e4, e2=1.0):
    """eq. ``eps_moments``."""
    return (6.0 * e4 - 2.0 * e2) / (6.0 * e4 + e2)


def bulk_pressure(n, Gp, e2=1.0, psi=psi_exp):
    """P_b = n c_s^2 + (G' e2 / 2) psi^2 (Sec. III A, with G' = G c_s^2 in the
    paper's convention or G in the literal one)."""
    n = np.asarray(n, dtype=np.float64)
    return n * CS2 + 0.5 * Gp * e2 * psi(n) ** 2


def critical_coupling(e2=1.0, psi=psi_exp, dpsi=dpsi_exp, n0=1.0):
    """(G'_c, n_c): where dP_b/dn = d^2P_b/dn^2 = 0 (found numerically)."""
    def eqs(v):
        G, n = v
        h = 1e-5
        p = lambda m: bulk_pressure(m, G, e2, psi)
        d1 = (p(n + h) - p(n - h)) / (2 * h)
        d2 = (p(n + h) - 2 * p(n) + p(n - h)) / (h * h)
        return [d1, d2]
    sol = optimize.fsolve(eqs, [-2.4, n0], xtol=1e-13)
    return float(sol[0]), float(sol[1])


def coexistence(Gp, eps=0.0, e2=1.0, psi=psi_exp, dpsi=dpsi_exp, guess=(0.2, 2.0)):
    """(n_g, n_l, p0) from eq. ``SCMaxwell``: equal pressure and a vanishing
    integral with measure dn psi'/psi^(eps+1).  Raises RuntimeError when the
    root finder stops short of a root (residuals above 1e-12) or falls onto
    the single-phase root n_g = n_l: the guess must lie in the basin of the
    two-phase root."""
    def P(n):
        return bulk_pressure(n, Gp, e2, psi)

    def integral(ng, nl, p0):
        fn = lambda m: dpsi(m) / psi(m) ** (eps + 1.0) * (p0 - P(m))
        return integrate.quad(fn, ng, nl, epsabs=1e-14, epsrel=1e-13, limit=400)[0]

    def eqs(v):
        ng, nl = v
        p0 = P(ng)
        return [P(nl) - p0, integral(ng, nl, p0)]
    ng, nl = optimize.fsolve(eqs, list(guess), xtol=1e-13)
    r = eqs([ng, nl])
    p0 = P(ng)
    if not (abs(r[0]) <= 1e-12 * max(1.0, abs(p0)) and abs(r[1]) <= 1e-12 and nl - ng > 1e-6):
        raise RuntimeError(f"coexistence: no two-phase root from guess {tuple(guess)} "
                           f"(n_g {ng:.6g}, n_l {nl:.6g}, residuals {r[0]:.2e}, {r[1]:.2e})")
    return float(ng), float(nl), float(p0)


def _profile_slope2(n, ng, p0, Gp, eps, e2, psi, dpsi):
    """(dpsi/dx)^2 at density n from eq. ``PSIProfile``."""
    fn = lambda m: dpsi(m) / psi(m) ** (eps + 1.0) * (p0 - bulk_pressure(m, Gp, e2, psi))
    I = integrate.quad(fn, ng, n, epsabs=1e-15, epsrel=1e-12, limit=400)[0]
    return 8.0 * (1.0 - eps) / (Gp * e2) * psi(n) ** eps * I


def sigma_second_order(Gp, e4, eps=0.0, e2=1.0, psi=psi_exp, dpsi=dpsi_exp, guess=(0.2, 2.0)):
    """eq. ``scsigma``: sigma0 ~ -(G' e4 / 2) int (dpsi/dx)^2 dx, with the
    integral over x rewritten over n through |dpsi/dx| dx = psi'(n) dn."""
    ng, nl, p0 = coexistence(Gp, eps, e2, psi, dpsi, guess)
    g = lambda m: dpsi(m) * np.sqrt(max(_profile_slope2(m, ng, p0, Gp, eps, e2, psi, dpsi), 0.0))
    I = integrate.quad(g, ng, nl, epsabs=1e-14, epsrel=1e-10, limit=400)[0]
    return -0.5 * Gp * e4 * I


def tolman_sc(Gp, sigma0, delta0_hat, ng, nl, psi=psi_exp):
    """eq. ``SCTolmanFlat``: delta ~ -(G'/(2 sigma0)) delta0_hat
    [psi^2(n_l) - psi^2(n_g)]."""
    return -(Gp / (2.0 * sigma0)) * delta0_hat * (float(psi(nl)) ** 2 - float(psi(ng)) ** 2)


# --- flat interfaces ------------------------------------------------------------
def _line_profiles(P, n, D):
    """Average over y (and z) to 1D profiles along x: n(x), P_N = P^xx,
    P_T = P^yy."""
    axes = (0, 1)
    nx_ = n.mean(axis=axes)
    PN = P[0].mean(axis=axes)
    PT = P[2 if D == 2 else 3].mean(axis=axes)
    return nx_, PN, PT


def interfaces(n1d):
    """Positions i where the profile crosses the mid density between i and
    i+1 (periodic), with +1 for rising (gas->liquid) and -1 for falling."""
    mid = 0.5 * (n1d.max() + n1d.min())
    s = np.sign(n1d - mid)
    out = []
    L = len(n1d)
    for i in range(L):
        a, b = s[i], s[(i + 1) % L]
        if a != b and a != 0 and b != 0:
            out.append((i, 1 if b > a else -1))
    return out


def flat_interface_windows(n1d):
    """Windows [a, b] (inclusive, may wrap) around each interface, bounded
    half way between neighbouring interfaces."""
    ifs = interfaces(n1d)
    L = len(n1d)
    k = len(ifs)
    wins = []
    for q in range(k):
        i, d = ifs[q]
        prev = ifs[q - 1][0]
        nxt = ifs[(q + 1) % k][0]
        gap_prev = (i - prev) % L if k > 1 else L
        gap_next = (nxt - i) % L if k > 1 else L
        a = i - gap_prev // 2 + 1
        b = i + gap_next // 2
        wins.append((a, b, d))
    return wins


def flat_observables(P, n, D=2):
    """sigma_0, z_s, z_e, delta (both definitions) per interface of a flat
    periodic slab (gradients along x)."""
    n1, PN, PT = _line_profiles(P, n, D)
    L = len(n1)
    res = []
    for a, b, d in flat_interface_windows(n1):
        xs = np.arange(a, b + 1)
        idx = xs % L
        dP = PN[idx] - PT[idx]
        sig = float(np.sum(dP))
        zs = float(np.sum(xs * dP) / sig)
        nn = n1[idx]
        if d > 0:   # gas -> liquid along +x
            ng, nl = nn[0], nn[-1]
            ze = (b + 0.5) - float(np.sum((nn - ng) / (nl - ng)))
        else:       # liquid -> gas along +x
            nl, ng = nn[0], nn[-1]
            ze = (a - 0.5) + float(np.sum((nn - ng) / (nl - ng)))
        orient = -d   # +1 when x runs from liquid to gas
        delta = orient * (ze - zs)
        # Gamma(z_s) with the same bulk values, x oriented liquid -> gas
        M = float(np.sum(nn))
        if d > 0:
            gamma = M - ng * (zs - (a - 0.5)) - nl * ((b + 0.5) - zs)
        else:
            gamma = M - nl * (zs - (a - 0.5)) - ng * ((b + 0.5) - zs)
        delta_ads = gamma / (nl - ng)
        res.append({"sigma": sig, "z_s": zs, "z_e": ze, "delta": delta,
                    "delta_ads": delta_ads, "n_l": float(nl), "n_g": float(ng),
                    "window": (a, b), "rising": d > 0})
    return res


def flat_sigma(P, n, D=2):
    """sigma_0 = (sum over the periodic line of P_N - P_T) / #interfaces."""
    n1, PN, PT = _line_profiles(P, n, D)
    k = len(interfaces(n1))
    if k == 0:
        return float("nan")
    return float(np.sum(PN - PT)) / k


# --- curved interfaces ----------------------------------------------------------
def equimolar_radius(n, n_in, n_out):
    """Equimolar radius R_e (Sec. V B, Laplace paragraph): the radius of the
    sharp disc (d = 2) or sphere (d = 3) of density n_in in a background
    n_out holding the lattice's total mass M:
    pi R^2 n_in + (L^2 - pi R^2) n_out = M, or with 4/3 pi R^3 and L^3.
    n_in is the inside density (liquid for a droplet, gas for a bubble);
    the dimension is read from n's shape (nz, ny, nx): nz == 1 is 2D."""
    if not n_in != n_out:
        raise ValueError("equimolar_radius: n_in equals n_out (no interface)")
    M = float(np.sum(n))
    V = n.size
    if n.shape[0] == 1:
        return float(np.sqrt((M - V * n_out) / (np.pi * (n_in - n_out))))
    return float(np.cbrt((M - V * n_out) / (4.0 / 3.0 * np.pi * (n_in - n_out))))


def laplace_fit(inv_R, dP):
    """Least-squares slope and intercept of dP vs 1/R (d-1 = 1 in 2D)."""
    A = np.vstack([np.asarray(inv_R), np.ones(len(inv_R))]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, np.asarray(dP), rcond=None)
    return float(slope), float(icpt)


def _sample_line(field, center, D):
    """Values of a site field (nz, ny, nx) along the x axis through `center`
    (x, y[, z]), at the sites x = 0 .. nx-1: linear interpolation between the
    neighbouring rows (and planes) when the centre's y (z) is not a site
    coordinate.  Returns the x coordinates and the values."""
    nz, ny, nx = field.shape
    cy = float(center[1])
    cz = float(center[2]) if D == 3 else 0.0
    y0, z0 = int(np.floor(cy)), int(np.floor(cz))
    ty, tz = cy - y0, cz - z0
    line = np.zeros(nx)
    for dz, wz in ((0, 1.0 - tz), (1, tz)):
        if wz == 0.0:
            continue
        for dy, wy in ((0, 1.0 - ty), (1, ty)):
            if wy == 0.0:
                continue
            line += wz * wy * field[(z0 + dz) % nz, (y0 + dy) % ny, :]
    return np.arange(nx, dtype=np.float64), line


def radial_profile(field, center, D):
    """A site field along the ray from the centre in +x and in -x, r from 0
    to L/2, as (r, value) for each ray: the field at sites, linearly
    interpolated in x where the centre lies between sites (periodic)."""
    xs, line = _sample_line(field, center, D)
    nx = len(xs)
    cx = float(center[0])
    r_max = nx / 2.0
    rays = []
    for sgn in (1.0, -1.0):
        # sample points: the centre, every site at 0 < r < L/2, and r = L/2
        pts = [0.0]
        k = np.arange(-nx, 2 * nx)
        r_sites = sgn * (k - cx)
        pts += sorted(r for r in r_sites if 0.0 < r < r_max)
        pts.append(r_max)
        r = np.array(pts)
        x = cx + sgn * r
        vals = np.interp(np.mod(x, nx), np.append(xs, nx), np.append(line, line[0]))
        rays.append((r, vals))
    return rays


def generalized_sigma(R, r, PT, P_in, P_out, D):
    """sigma[R] = int_0^{r_max} dr (r/R)^(d-1) [P_J(r; R) - P_T(r)] with
    P_J = P_in for r < R and P_out beyond (Sec. III B, generalized surface
    tension), for P_T given at the points r (0 .. r_max) and linear between
    them: each piece's integral of r^(d-1) (a + b r) is taken in closed form,
    the piece holding R split there."""
    total = 0.0
    for k in range(len(r) - 1):
        ra, rb = float(r[k]), float(r[k + 1])
        pa, pb = float(PT[k]), float(PT[k + 1])
        b = (pb - pa) / (rb - ra)
        a = pa - b * ra
        cuts = [ra] + ([R] if ra < R < rb else []) + [rb]
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            PJ = P_in if 0.5 * (lo + hi) < R else P_out
            # int r^(d-1) (PJ - a - b r) dr from lo to hi
            F = lambda t: (PJ - a) * t ** D / D - b * t ** (D + 1) / (D + 1)
            total += F(hi) - F(lo)
    return total / R ** (D - 1)


def golden_min(fun, lo, hi, tol=1e-12, maxit=400):
    """Minimum of a unimodal function on [lo, hi] by golden-section search."""
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = fun(c), fun(d)
    for _ in range(maxit):
        if b - a <= tol * max(1.0, abs(a) + abs(b)):
            break
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = fun(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = fun(d)
    x = 0.5 * (a + b)
    return x, fun(x)


def curved_observables(P, n, center, D, Gp, e2=1.0, psi=psi_exp, corner=(0, 0, 0)):
    """Observables of one droplet or bubble at rest (Sec. III B, Sec. V B):

    * n_in at the centre (linear interpolation), n_out at a corner site;
      P_in, P_out their bulk pressures, Delta P = P_in - P_out;
    * R_e, the equimolar radius;
    * sigma[R] along the x axis through the centre with P_T = P^yy (both rays
      averaged), its stationary point R_s (the surface of tension, where
      d sigma[R]/dR = 0: a minimum, for droplets and bubbles alike, since
      the inside pressure exceeds the outside one in both) and
      sigma_s = sigma[R_s], by golden-section search over 0 < R < L/2.
    P is the lattice pressure tensor (components of oracle.pressure_tensor,
    (xx, xy, yy) in 2D, (xx, xy, xz, yy, yz, zz) in 3D)."""
    nz, ny, nx = n.shape
    cxyz = tuple(float(c) for c in center) + ((0.0,) if D == 2 else ())
    _, nline = _sample_line(n, cxyz, D)
    n_in = float(np.interp(cxyz[0], np.arange(nx + 1), np.append(nline, nline[0])))
    n_out = float(n[corner[2] if D == 3 else 0, corner[1], corner[0]])
    P_in = float(bulk_pressure(n_in, Gp, e2, psi))
    P_out = float(bulk_pressure(n_out, Gp, e2, psi))
    bubble = n_in < n_out   # b = 1
    Pyy = P[2] if D == 2 else P[3]
    rays = radial_profile(Pyy, cxyz, D)

    def sigma(R):
        return 0.5 * sum(generalized_sigma(R, r, v, P_in, P_out, D) for r, v in rays)
    Rs, _ = golden_min(sigma, 0.5, nx / 2.0 - 0.5)
    return {"n_in": n_in, "n_out": n_out, "P_in": P_in, "P_out": P_out,
            "dP": P_in - P_out, "R_e": equimolar_radius(n, n_in, n_out),
            "R_s": Rs, "sigma_s": sigma(Rs), "bubble": bool(bubble), "sigma_fn": sigma}


def tolman_curved_fit(results, sigma0, D):
    """The Tolman length from droplets and bubbles (Sec. III B): by eqs.
    ExactLaplace and SigmaCExpansion, Delta P R_s / ((d-1) sigma0) =
    1 - (d-1) delta / R_s with R_s counted negative for a bubble (b = 1);
    a straight line through those points against (-1)^b / R_s has slope
    -(d-1) delta.  Returns (delta, intercept)."""
    x, y = [], []
    for r in results:
        s = -1.0 if r["bubble"] else 1.0
        x.append(s / r["R_s"])
        y.append(r["dP"] * r["R_s"] / ((D - 1) * sigma0))
    slope, icpt = laplace_fit(x, y)
    return -slope / (D - 1), icpt


def laplace_sigma(results, D):
    """sigma from the Laplace law over droplets and bubbles (Sec. V B): the
    inside pressure exceeds the outside one for both (Delta P > 0); with the
    factor (-1)^b on the pressure difference and on the curvature (b = 1 for
    a bubble) both kinds lie on one line (-1)^b Delta P = (d-1) sigma
    (-1)^b / R_e.  Returns (sigma, intercept)."""
    x, y = [], []
    for r in results:
        s = -1.0 if r["bubble"] else 1.0
        x.append(s / r["R_e"])
        y.append(s * r["dP"])
    slope, icpt = laplace_fit(x, y)
    return slope / (D - 1), icpt
