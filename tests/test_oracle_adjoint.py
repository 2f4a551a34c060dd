"""Pin of the oracle's adjoint (oracle/adjoint.py) to the oracle's forward step:
its numpy forward reproduces the C oracle, and the gradient of the flat-slab
surface tension sigma_0 (Sec. V A, from the Appendix E pressure tensor summed
over the lattice) with respect to the stencil group weights, G and the
initial populations equals central finite differences of the C oracle run
(h = 1e-6 relative for the parameters, 1e-4 for the populations)."""
import numpy as np
import pytest

import lbinputs as L
import oracle
from oracle import adjoint as AD

CASES = [
    ("D2Q9", (1, 5, 24), L.E8_2D, 1.0, -3.0, "literal", 12),
    ("D3Q19", (3, 4, 20), L.E4_3D, 0.8, -4.0, "literal", 8),
    ("D2Q9", (1, 4, 22), L.E6_2D, 1.3, -9.0, "paper", 10),
]


def _setup(lattice, shape, st, tau, G, conv, A=0.0):
    nz, ny, nx = shape
    rho = L.tanh_slab(nx, ny, nz, nx // 4, 3 * nx // 4, 0.456, 2.25, 2.0)
    o = oracle.Oracle(lattice, shape, st.groups, tau=tau, G=G, convention=conv, forcing_A=A)
    o.init_equilibrium(rho)
    return o


def _sigma_after(lattice, shape, groups, tau, G, conv, g0, steps, A=0.0):
    o = oracle.Oracle(lattice, shape, groups, tau=tau, G=G, convention=conv, forcing_A=A)
    o.f = g0.copy()
    o.step(steps)
    return AD.sigma_flat(o, o.f, 2)[0]


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,steps", CASES)
def test_numpy_forward_matches_c_oracle(lattice, shape, st, tau, G, conv, steps):
    o = _setup(lattice, shape, st, tau, G, conv)
    g = o.f.copy()
    for _ in range(3):
        g = AD.step_forward(o, g)
    o.step(3)
    assert np.max(np.abs(g - o.f)) < 1e-14


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,steps", CASES)
def test_sigma_formula_matches_pressure_tensor(lattice, shape, st, tau, G, conv, steps):
    o = _setup(lattice, shape, st, tau, G, conv)
    o.step(steps)
    s = AD.sigma_flat(o, o.f, 2)[0]
    P = o.pressure_tensor()
    PT = P[2] if o.D == 2 else P[3]
    assert abs(s - float(np.sum(P[0] - PT)) / 2) < 1e-12 * abs(s)


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,steps", CASES)
def test_adjoint_gradient_matches_finite_differences(lattice, shape, st, tau, G, conv, steps):
    o = _setup(lattice, shape, st, tau, G, conv)
    g0 = o.f.copy()
    sigma, lam, dW, dGp = AD.gradient(o, g0, steps, 2)
    assert abs(sigma - _sigma_after(lattice, shape, st.groups, tau, G, conv, g0, steps)) < 1e-13
    # group weights
    for q, (b, wq) in enumerate(st.groups):
        h = 1e-6 * float(wq)
        gp = [(bb, float(ww) + (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        gm = [(bb, float(ww) - (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        fd = (_sigma_after(lattice, shape, gp, tau, G, conv, g0, steps) -
              _sigma_after(lattice, shape, gm, tau, G, conv, g0, steps)) / (2 * h)
        assert abs(dW[q] - fd) < 1e-6 * max(abs(fd), 1e-3 * abs(sigma) / float(wq)), (q, dW[q], fd)
    # coupling (G' = G or G/3)
    h = 1e-6 * abs(G)
    fd = (_sigma_after(lattice, shape, st.groups, tau, G + h, conv, g0, steps) -
          _sigma_after(lattice, shape, st.groups, tau, G - h, conv, g0, steps)) / (2 * h)
    dG = dGp * (1.0 / 3.0 if conv == "paper" else 1.0)
    assert abs(dG - fd) < 1e-6 * abs(fd), (dG, fd)
    # initial populations, a few entries
    rng = np.random.default_rng(1)
    for _ in range(4):
        idx = tuple(int(rng.integers(0, s)) for s in g0.shape)
        h = 1e-4 * abs(g0[idx])      # sigma ~ 0.2: FD rounding 1e-16 sigma / h stays below 1e-11
        gp, gm = g0.copy(), g0.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (_sigma_after(lattice, shape, st.groups, tau, G, conv, gp, steps) -
              _sigma_after(lattice, shape, st.groups, tau, G, conv, gm, steps)) / (2 * h)
        assert abs(lam[idx] - fd) < 1e-6 * abs(fd) + 1e-10, (idx, lam[idx], fd)


def _ratio_fn(xl, xg):
    """n_l / n_g of the column averages at xl (liquid) and xg (gas)."""
    def fn(n):
        cols = n.shape[0] * n.shape[1]
        nl, ng = n[..., xl].mean(), n[..., xg].mean()
        d = np.zeros_like(n)
        d[..., xl] = 1.0 / (ng * cols)
        d[..., xg] = -nl / (ng * ng * cols)
        return nl / ng, d
    return fn


def _n_after(lattice, shape, groups, tau, G, conv, g0, steps):
    o = oracle.Oracle(lattice, shape, groups, tau=tau, G=G, convention=conv)
    o.f = g0.copy()
    o.step(steps)
    return o.fields()["n"]


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,steps", CASES[:2])
def test_density_functional_gradient_matches_finite_differences(lattice, shape, st, tau, G, conv, steps):
    """The same adjoint seeded by a loss on the density (the ratio of the
    liquid to the gas column density) against central differences."""
    o = _setup(lattice, shape, st, tau, G, conv)
    g0 = o.f.copy()
    nx = shape[2]
    fn = _ratio_fn(nx // 2, 1)
    val, lam, dW, dGp = AD.gradient_of_density_functional(o, g0, steps, fn)
    assert abs(val - fn(_n_after(lattice, shape, st.groups, tau, G, conv, g0, steps))[0]) < 1e-12
    for q, (b, wq) in enumerate(st.groups):
        h = 1e-6 * float(wq)
        gp = [(bb, float(ww) + (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        gm = [(bb, float(ww) - (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        fd = (fn(_n_after(lattice, shape, gp, tau, G, conv, g0, steps))[0] -
              fn(_n_after(lattice, shape, gm, tau, G, conv, g0, steps))[0]) / (2 * h)
        assert abs(dW[q] - fd) < 1e-6 * abs(fd) + 1e-9, (q, dW[q], fd)
    h = 1e-6 * abs(G)
    fd = (fn(_n_after(lattice, shape, st.groups, tau, G + h, conv, g0, steps))[0] -
          fn(_n_after(lattice, shape, st.groups, tau, G - h, conv, g0, steps))[0]) / (2 * h)
    assert abs(dGp - fd) < 1e-6 * abs(fd) + 1e-9


# the F^2 forcing variant (Sec. VI): the source term gains
# -cw_i (A/tau) (4.5 (xi.F)^2 - 1.5 F.F); A = 0.25 and 0.6
CASES_F2 = [
    ("D2Q9", (1, 5, 24), L.E8_2D, 1.0, -3.0, "literal", 10, 0.25),
    ("D3Q19", (3, 4, 20), L.E4_3D, 0.8, -4.0, "literal", 6, 0.6),
]


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,steps,A", CASES_F2)
def test_f2_numpy_forward_matches_c_oracle(lattice, shape, st, tau, G, conv, steps, A):
    o = _setup(lattice, shape, st, tau, G, conv, A)
    g = o.f.copy()
    for _ in range(3):
        g = AD.step_forward(o, g)
    o.step(3)
    assert np.max(np.abs(g - o.f)) < 1e-14
    # the variant changes the step (a dropped term would pass the first check
    # only if the F^2 source vanished)
    o0 = _setup(lattice, shape, st, tau, G, conv, 0.0)
    o0.step(3)
    assert np.max(np.abs(o0.f - o.f)) > 1e-8


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,steps,A", CASES_F2)
def test_f2_adjoint_gradient_matches_finite_differences(lattice, shape, st, tau, G, conv, steps, A):
    o = _setup(lattice, shape, st, tau, G, conv, A)
    g0 = o.f.copy()
    sigma, lam, dW, dGp = AD.gradient(o, g0, steps, 2)
    assert abs(sigma - _sigma_after(lattice, shape, st.groups, tau, G, conv, g0, steps, A)) < 1e-13
    for q, (b, wq) in enumerate(st.groups):
        h = 1e-6 * float(wq)
        gp = [(bb, float(ww) + (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        gm = [(bb, float(ww) - (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        fd = (_sigma_after(lattice, shape, gp, tau, G, conv, g0, steps, A) -
              _sigma_after(lattice, shape, gm, tau, G, conv, g0, steps, A)) / (2 * h)
        assert abs(dW[q] - fd) < 1e-6 * max(abs(fd), 1e-3 * abs(sigma) / float(wq)), (q, dW[q], fd)
    h = 1e-6 * abs(G)
    fd = (_sigma_after(lattice, shape, st.groups, tau, G + h, conv, g0, steps, A) -
          _sigma_after(lattice, shape, st.groups, tau, G - h, conv, g0, steps, A)) / (2 * h)
    assert abs(dGp - fd) < 1e-6 * abs(fd), (dGp, fd)
    rng = np.random.default_rng(7)
    for _ in range(4):
        idx = tuple(int(rng.integers(0, s)) for s in g0.shape)
        h = 1e-4 * abs(g0[idx])
        gp, gm = g0.copy(), g0.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (_sigma_after(lattice, shape, st.groups, tau, G, conv, gp, steps, A) -
              _sigma_after(lattice, shape, st.groups, tau, G, conv, gm, steps, A)) / (2 * h)
        assert abs(lam[idx] - fd) < 1e-6 * abs(fd) + 1e-10, (idx, lam[idx], fd)
