"""Discrete adjoint of the oracle's step, in plain numpy (TEST INFRASTRUCTURE
ONLY: used by tests/ to check the GPU adjoint; never by the library).

The step (Sec. II, eqs. lbm, omega_i, f_eq, GuoForcing, sc_f), per node x,
from the post-streaming populations g (the state):
    n = sum_i g_i,  psi = psi(n),
    acc = sum_pairs W_a (psi(x + e_a) - psi(x - e_a)) e_a,  F = -G' psi acc,
    j = sum_i g_i xi_i,  u = (j + F/2) / n,
    B_i = g_i - omega (g_i - f_eq_i(n, u)) + S_i(u, F),
    next state g'_i(x + xi_i) = B_i(x),
where S_i = cw_i (3 xi.F + 9 (xi.u)(xi.F) - 3 u.F) with Guo's forcing, and
the F^2 variant (Sec. VI, A = forcing_A, kA = A/tau) subtracts
cw_i kA (4.5 (xi.F)^2 - 1.5 F.F), so that dS_i/dF gains
-cw_i kA (9 (xi.F) xi - 3 F).
With lam' = dL/dg' (same layout as the state), the adjoint gives
dL/dg, dL/dW (per group) and dL/dG' by the chain rule through each line
above, read backwards:
    lamB_i(x) = lam'_i(x + xi_i)
    lam_u = sum_i lamB_i (omega df_eq_i/du + dS_i/du),  lam_n|u = omega sum_i lamB_i df_eq_i/dn
    lam_F|u = sum_i lamB_i dS_i/dF
    u = (j + F/2)/n:  lam_j = lam_u / n,  lam_F = lam_F|u + lam_u / (2n),
                      lam_n = lam_n|u - lam_u . u / n
    F = -G' psi acc:  lam_psi(x) += -G' lam_F . acc,  lam_acc = -G' psi lam_F,
                      dL/dG' += -psi acc . lam_F
    acc:              dL/dW_a += (psi(x+e_a) - psi(x-e_a)) e_a . lam_acc(x),
                      lam_psi(y) += W_a e_a . (lam_acc(y - e_a) - lam_acc(y + e_a))
    psi(n):           lam_n += psi'(n) lam_psi
    g:                lam_i = (1 - omega) lamB_i + lam_n + xi_i . lam_j
Surface tension of a flat periodic slab: summed over the lattice, the
pressure tensor of Appendix E gives
    sum_x (P_N - P_T) = (G'/2) sum_x psi(x) sum_e W(e) psi(x + e) (e_x^2 - e_y^2)
(every vector e of the stencil, both signs); sigma_0 is that sum over the
number of interfaces (eq. for sigma_0 in Sec. V A).
"""
import numpy as np

from . import C9, C19


def _lattice(Q):
    if Q == 9:
        C = np.zeros((9, 3), dtype=int)
        C[:, :2] = C9
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    else:
        C = np.asarray(C19, dtype=int)
        w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return C, w


def _shift(a, e):
    """b(x) = a(x + e) on the periodic lattice (arrays indexed [z, y, x])."""
    return np.roll(a, shift=(-e[2], -e[1], -e[0]), axis=(0, 1, 2))


def _psi(n, kind, eps):
    if kind == 0:
        p = np.exp(-1.0 / n)
        return p, p / (n * n)
    p = (n / (eps + n)) ** (1.0 / eps)
    return p, p / (n * (eps + n))


def _pair_groups(o):
    """Group index (position in o.groups) of each canonical pair of o.vec."""
    keys = [tuple(sorted(abs(int(c)) for c in (tuple(b) + (0,) * (3 - len(b))))) for b, _ in o.groups]
    return np.array([keys.index(tuple(sorted(abs(int(c)) for c in v))) for v in o.vec])


def step_forward(o, g):
    """The oracle's step on state g [Q, nz, ny, nx] in numpy (same model as
    the C oracle; used here to have the intermediates of the adjoint)."""
    Q = g.shape[0]
    C, w = _lattice(Q)
    D = o.D
    n = g.sum(axis=0)
    psi, _ = _psi(n, o.psi_kind, o.psi_eps)
    acc = np.zeros((3,) + n.shape)
    for e, Wa in zip(o.vec, o.w):
        d = _shift(psi, e) - _shift(psi, -e)
        for a in range(D):
            acc[a] += Wa * d * e[a]
    F = -o.Gp * psi * acc
    j = np.einsum("ia,i...->a...", C.astype(float), g)
    u = (j + 0.5 * F) / n
    om = 1.0 / o.tau
    cwf = (1.0 - 0.5 * om) * w
    kA = getattr(o, "forcing_A", 0.0) / o.tau
    uu = (u * u).sum(axis=0)
    uF = (u * F).sum(axis=0)
    FF = (F * F).sum(axis=0)
    out = np.empty_like(g)
    for i in range(Q):
        cu = sum(C[i, a] * u[a] for a in range(D))
        cF = sum(C[i, a] * F[a] for a in range(D))
        feq = w[i] * n * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
        S = cwf[i] * (3 * cF + 9 * cu * cF - 3 * uF - kA * (4.5 * cF * cF - 1.5 * FF))
        B = g[i] - om * (g[i] - feq) + S
        out[i] = _shift(B, -C[i])          # g'_i(x + xi_i) = B_i(x)
    return out


def step_adjoint(o, g, lam_next):
    """dL/dg, dL/dW (per group of o.groups) and dL/dG' for one step from
    state g, given lam_next = dL/d(next state)."""
    Q = g.shape[0]
    C, w = _lattice(Q)
    D = o.D
    n = g.sum(axis=0)
    psi, dpsi = _psi(n, o.psi_kind, o.psi_eps)
    acc = np.zeros((3,) + n.shape)
    for e, Wa in zip(o.vec, o.w):
        d = _shift(psi, e) - _shift(psi, -e)
        for a in range(D):
            acc[a] += Wa * d * e[a]
    F = -o.Gp * psi * acc
    j = np.einsum("ia,i...->a...", C.astype(float), g)
    u = (j + 0.5 * F) / n
    om = 1.0 / o.tau
    cwf = (1.0 - 0.5 * om) * w
    kA = getattr(o, "forcing_A", 0.0) / o.tau
    lamB = np.stack([_shift(lam_next[i], C[i]) for i in range(Q)])
    lam_u = np.zeros((3,) + n.shape)
    lam_Fu = np.zeros((3,) + n.shape)
    lam_nu = np.zeros(n.shape)
    uu = (u * u).sum(axis=0)
    for i in range(Q):
        cu = sum(C[i, a] * u[a] for a in range(D))
        cF = sum(C[i, a] * F[a] for a in range(D))
        lam_nu += lamB[i] * om * w[i] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
        for a in range(D):
            dfeq = w[i] * n * (3 * C[i, a] + 9 * cu * C[i, a] - 3 * u[a])
            dSu = cwf[i] * (9 * cF * C[i, a] - 3 * F[a])
            dSF = cwf[i] * (3 * C[i, a] + 9 * cu * C[i, a] - 3 * u[a]
                            - kA * (9 * cF * C[i, a] - 3 * F[a]))
            lam_u[a] += lamB[i] * (om * dfeq + dSu)
            lam_Fu[a] += lamB[i] * dSF
    lam_j = lam_u / n
    lam_F = lam_Fu + lam_u / (2 * n)
    lam_n = lam_nu - (lam_u * u).sum(axis=0) / n
    lam_psi = -o.Gp * (lam_F * acc).sum(axis=0)
    lam_acc = -o.Gp * psi * lam_F
    dGp = float(np.sum(-psi * (acc * lam_F).sum(axis=0)))
    pg = _pair_groups(o)
    dW = np.zeros(len(o.groups))
    for e, Wa, q in zip(o.vec, o.w, pg):
        ela = sum(e[a] * lam_acc[a] for a in range(D))
        dW[q] += float(np.sum((_shift(psi, e) - _shift(psi, -e)) * ela))
        lam_psi += Wa * (_shift(ela, -e) - _shift(ela, e))
    lam_n = lam_n + dpsi * lam_psi
    lam = np.stack([(1 - om) * lamB[i] + lam_n + sum(C[i, a] * lam_j[a] for a in range(D))
                    for i in range(Q)])
    return lam, dW, dGp


def sigma_flat(o, g, n_interfaces):
    """sigma_0 of a flat slab (gradients along x) from state g, with its
    gradient: (sigma, dsigma/dg, dsigma/dW per group, dsigma/dG')."""
    n = g.sum(axis=0)
    psi, dpsi = _psi(n, o.psi_kind, o.psi_eps)
    pg = _pair_groups(o)
    dW = np.zeros(len(o.groups))
    tot = 0.0
    h = np.zeros(n.shape)                 # sum_e W(e) psi(x + e) (e_x^2 - e_y^2)
    for e, Wa, q in zip(o.vec, o.w, pg):
        k = float(e[0] * e[0] - e[1] * e[1])
        if k == 0.0:
            continue
        s = (_shift(psi, e) + _shift(psi, -e)) * k      # e and -e
        h += Wa * s
        dW[q] += 0.5 * o.Gp / n_interfaces * float(np.sum(psi * s))
    tot = float(np.sum(psi * h))
    sigma = 0.5 * o.Gp * tot / n_interfaces
    lam_n = dpsi * (o.Gp / n_interfaces) * h
    lam = np.broadcast_to(lam_n, g.shape).copy()
    return sigma, lam, dW, sigma / o.Gp


def gradient(o, g0, steps, n_interfaces):
    """sigma after `steps` steps from g0 and its gradient with respect to the
    initial state, the group weights and G' (forward in numpy, then the
    adjoint steps backwards)."""
    states = [g0]
    for _ in range(steps):
        states.append(step_forward(o, states[-1]))
    sigma, lam, dW, dGp = sigma_flat(o, states[-1], n_interfaces)
    for s in range(steps - 1, -1, -1):
        lam, w_s, g_s = step_adjoint(o, states[s], lam)
        dW += w_s
        dGp += g_s
    return sigma, lam, dW, dGp


def gradient_of_density_functional(o, g0, steps, fn):
    """A loss fn(n) -> (L, dL/dn) of the density after `steps` steps from g0
    and its gradient (forward in numpy, then the adjoint steps backwards):
    returns (L, dL/dg0, dL/dW per group, dL/dG')."""
    states = [g0]
    for _ in range(steps):
        states.append(step_forward(o, states[-1]))
    value, dn = fn(states[-1].sum(axis=0))
    lam = np.broadcast_to(dn, states[-1].shape).copy()
    dW = np.zeros(len(o.groups))
    dGp = 0.0
    for s in range(steps - 1, -1, -1):
        lam, w_s, g_s = step_adjoint(o, states[s], lam)
        dW += w_s
        dGp += g_s
    return value, lam, dW, dGp
