"""The pseudopotential psi_eps = (n/(eps+n))^(1/eps) (eq. psieps) on the GPU.

* the binary64 power the step uses equals the oracle's (a correctly rounded
  power of the same rounded base and exponent) bit for bit;
* binary64 steps with psi_eps match the oracle bit for bit after 100 steps
  (D2Q9 E8 with eps = 10/31, the eps of its e4 = 4/7; D3Q19 E8 with the
  paper's eps = 14/29);
* shifted binary32 steps with psi_eps stay within 1e-5 of the oracle's
  density on every binary32 path: the fused D2Q9 strip march, the fused
  D3Q19 kernel with cp.async or TMA staging, and the two-kernel path, which
  also agree with each other;
* a batch that mixes psi_eps and psi = exp(-1/n) lattices, with and without
  the F^2 forcing variant, matches the oracle per member and equals each
  member stepped on its own, bit for bit.
"""
import numpy as np
import pytest

import lbinputs as L
import oracle
from oracle import analysis as A

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")


def _inputs():
    rng = np.random.default_rng(31)
    ns = list(0.02 + 6.0 * rng.random(3000)) + list(np.exp(rng.uniform(np.log(1e-3), np.log(50.0), 1000)))
    return np.array(ns + [0.15, 1.9, 1.0, 0.456, 2.25, 1e-3, 50.0, 1e-300, 1e300, 1e-310, 4e-320])


@pytest.mark.parametrize("eps", [14.0 / 29.0, 10.0 / 31.0, 0.25, 2.0])
def test_power_matches_oracle_bitwise(eps):
    n = _inputs()
    got, amb = P.lb_psi_eval(n, eps)
    want = np.array([oracle.psi(v, 1, eps) for v in n])
    assert amb == 0
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(n[i], got[i], want[i]) for i in bad[:5]]


def test_exp_kind_matches_oracle_bitwise():
    n = _inputs()
    got, amb = P.lb_psi_eval(n)
    want = np.array([oracle.psi(v) for v in n])
    assert amb == 0 and np.array_equal(got, want)


@pytest.mark.parametrize("eps", [14.0 / 29.0, 10.0 / 31.0, 0.25, 2.0])
def test_eps_kind_many_densities_bitwise(eps):
    """60,000 seeded densities per eps: the binary64 psi_eps (a power of the
    rounded base) equals the oracle's correctly rounded power bit for bit,
    whichever phase of the library's power answered."""
    rng = np.random.default_rng(77)
    n = np.concatenate([rng.uniform(0.02, 6.0, 40_000),
                        np.exp(rng.uniform(np.log(1e-3), np.log(1e3), 20_000))])
    got, amb = P.lb_psi_eval(n, eps)
    want = np.array([oracle.psi(v, 1, eps) for v in n])
    assert amb == 0
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(n[i], got[i], want[i]) for i in bad[:5]]


def test_exp_kind_many_densities_bitwise():
    """300,000 seeded densities over the range the steps see (and beyond,
    where exp(-1/n) leaves the table-driven first phase): the binary64 psi
    equals the oracle's binary128 exp rounded once, bit for bit, whichever
    phase of the library's exp answered."""
    rng = np.random.default_rng(2024)
    n = np.concatenate([rng.uniform(0.02, 6.0, 200_000),
                        np.exp(rng.uniform(np.log(1e-3), np.log(1e4), 100_000))])
    got, amb = P.lb_psi_eval(n)
    want = np.array([oracle.psi(v) for v in n])
    assert amb == 0
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(n[i], got[i], want[i]) for i in bad[:5]]


def _coupling(eps):
    f, df = A.psi_eps_fn(eps)
    Gc, _ = A.critical_coupling(psi=f, dpsi=df)
    Gp = 1.1 * Gc
    ng, nl, _ = A.coexistence(Gp, eps, psi=f, dpsi=df, guess=(0.4, 1.4))
    return Gp, ng, nl


CASES = [
    ("D2Q9", (61, 47), L.E8_2D, 10.0 / 31.0, 0.8),
    ("D3Q19", (24, 20, 18), L.E8_3D, 14.0 / 29.0, 1.0),
]


def _run(lattice, shape, st, eps, tau, precision, steps=100):
    Gp, ng, nl = _coupling(eps)
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    rho = L.tanh_sphere(nx, ny, nz, 0.3 * min(nx, ny), nl, ng, 2.0)
    lat = P.Lattice(lattice, shape, rho, st.bases, st.weights, precision=precision, tau=tau, G=Gp,
                    convention="literal", psi_eps=eps)
    lat.step(steps)
    assert lat.sync() == P.LB_OK
    o = oracle.Oracle(lattice, (nz, ny, nx), st.groups, tau=tau, G=Gp, convention="literal",
                      psi_kind=1, psi_eps=eps)
    o.init_equilibrium(rho)
    o.step(steps)
    return lat, o


@pytest.mark.parametrize("lattice,shape,st,eps,tau", CASES)
def test_fp64_steps_bitwise(lattice, shape, st, eps, tau):
    lat, o = _run(lattice, shape, st, eps, tau, "fp64")
    assert P.lb_fused_active(lat.ctx) == 0
    f = lat.state().reshape(o.f.shape)
    assert np.array_equal(f, o.f)
    assert lat.observables()["exp_ambiguous"] == 0
    lat.close()


@pytest.mark.parametrize("lattice,shape,st,eps,tau", CASES)
def test_fp32_density(lattice, shape, st, eps, tau):
    lat, o = _run(lattice, shape, st, eps, tau, "fp32")
    # D2Q9: the fused strip march; D3Q19 24 x 20 x 18: the fused kernel with
    # cp.async staging (nx is not a multiple of 32)
    assert P.lb_fused_active(lat.ctx) == (3 if lattice == "D2Q9" else 1)
    n, _ = lat.fields()
    ref = o.fields()["n"]
    assert np.max(np.abs(n - ref) / ref) < 1e-5
    lat.close()


# every binary32 path with psi_eps: (lattice, shape, stencil, eps, options,
# expected lb_fused_active)
PATHS = [
    ("D2Q9", (61, 47), L.E8_2D, 10.0 / 31.0, "fused", 3),
    ("D2Q9", (61, 47), L.E8_2D, 10.0 / 31.0, "two-kernel", 0),
    ("D3Q19", (64, 32, 24), L.E8_3D, 14.0 / 29.0, "tma", 2),
    ("D3Q19", (64, 32, 24), L.E8_3D, 14.0 / 29.0, "cpasync", 1),
    ("D3Q19", (64, 32, 24), L.E8_3D, 14.0 / 29.0, "two-kernel", 0),
]


def _fp32_run(lattice, shape, st, eps, mode, steps):
    Gp, ng, nl = _coupling(eps)
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    rho = L.tanh_sphere(nx, ny, nz, 0.3 * min(nx, ny), nl, ng, 2.0)
    lat = P.Lattice(lattice, shape, rho, st.bases, st.weights, precision="fp32", tau=1.0, G=Gp,
                    convention="literal", psi_eps=eps)
    P.lb_set_option(lat.ctx, P.LB_OPT_FUSED, mode != "two-kernel")
    if lattice == "D3Q19":
        P.lb_set_option(lat.ctx, P.LB_OPT_TMA, mode == "tma")
    active = P.lb_fused_active(lat.ctx)
    lat.step(steps)
    assert lat.sync() == P.LB_OK
    n = lat.fields()[0]
    lat.close()
    return rho, Gp, active, n


@pytest.fixture(scope="module")
def path_runs():
    out = {}
    for lattice, shape, st, eps, mode, want in PATHS:
        out[(lattice, mode)] = _fp32_run(lattice, shape, st, eps, mode, 100)
    return out


@pytest.mark.parametrize("lattice,shape,st,eps,mode,want", PATHS)
def test_every_fp32_path_matches_oracle(path_runs, lattice, shape, st, eps, mode, want):
    rho, Gp, active, n = path_runs[(lattice, mode)]
    assert active == want
    nz = shape[2] if len(shape) > 2 else 1
    o = oracle.Oracle(lattice, (nz, shape[1], shape[0]), st.groups, tau=1.0, G=Gp,
                      convention="literal", psi_kind=1, psi_eps=eps)
    o.init_equilibrium(rho)
    o.step(100)
    ref = o.fields()["n"]
    assert np.max(np.abs(n - ref) / ref) < 1e-5


def test_fused_and_two_kernel_paths_agree(path_runs):
    for lattice, modes in (("D2Q9", ("fused", "two-kernel")),
                           ("D3Q19", ("tma", "cpasync", "two-kernel"))):
        base = path_runs[(lattice, modes[0])][3]
        for m in modes[1:]:
            other = path_runs[(lattice, m)][3]
            assert np.max(np.abs(other - base) / base) < 2e-6, (lattice, m)


# (nx, ny, stencil, radius, droplet, eps or None, F^2 A)
MIXED = [
    (64, 64, L.E8_2D, 14.0, True, 10.0 / 31.0, 0.0),
    (96, 64, L.E6_2D, 18.0, False, None, 0.0),
    (50, 70, L.E8_2D, 12.0, False, 14.0 / 29.0, 0.0),
    (40, 36, L.E4_2D, 9.0, True, None, 0.3),
    (48, 40, L.E8_2D, 10.0, True, 10.0 / 31.0, 0.3),
]


def _mixed_member(nx, ny, st, r, droplet, eps, A):
    if eps is None:
        Gp, ng, nl = -3.0, 0.456, 2.25
    else:
        Gp, ng, nl = _coupling(eps)
    rin, rout = (nl, ng) if droplet else (ng, nl)
    rho = L.tanh_sphere(nx, ny, 1, r, rin, rout, 2.0)
    lat = P.Lattice("D2Q9", (nx, ny), rho, st.bases, st.weights, precision="fp32", tau=1.0,
                    G=Gp, convention="literal", psi_eps=eps, forcing_A=A)
    return lat, rho, Gp


def test_mixed_psi_batch_matches_oracle_and_single_steps():
    made = [_mixed_member(*m) for m in MIXED]
    lats = [m[0] for m in made]
    b = P.Batch(lats)
    b.step(100)
    assert b.sync() == P.LB_OK
    got = [l.state() for l in lats]
    for (lat, rho, Gp), (nx, ny, st, r, drop, eps, A) in zip(made, MIXED):
        o = oracle.Oracle("D2Q9", (1, ny, nx), st.groups, tau=1.0, G=Gp, convention="literal",
                          psi_kind=0 if eps is None else 1, psi_eps=eps or 0.0, forcing_A=A)
        o.init_equilibrium(rho)
        o.step(100)
        ref = o.fields()["n"]
        n = lat.fields()[0]
        assert np.max(np.abs(n - ref) / ref) < 1e-5, (nx, ny, eps)
    b.close()
    for l in lats:
        l.close()
    # the same members stepped one by one: the batch changes no node's arithmetic
    for k, m in enumerate(MIXED):
        lat, _, _ = _mixed_member(*m)
        assert P.lb_fused_active(lat.ctx) == 3
        lat.step(100)
        assert lat.sync() == P.LB_OK
        assert np.array_equal(lat.state(), got[k])
        lat.close()
