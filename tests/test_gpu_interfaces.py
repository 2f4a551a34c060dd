"""The library's own interface observables (lb_flat_interfaces,
lb_curved_interface, lb_fit_laplace, lb_fit_tolman: binary64 line
integrals of the pressure tensor on the device) against the oracle's
analysis of the oracle's run (Sec. III B, Sec. IV, Sec. V B).

* binary64 lattices reach the oracle's state bit for bit, so the two
  analyses of the same state must agree to rounding: sigma_0, z_s, z_e,
  delta and delta_ads of a slab to 1e-11; n_in, n_out, Delta P, R_e to
  1e-12; the surface of tension R_s and sigma_s, which the library takes in
  closed form and the oracle by a minimum search, to 1e-7 (the search's
  resolution in binary64); in 2D and 3D, centres on and between sites;
* shifted binary32 lattices: the fitted quantities within 1e-3 relative of
  the oracle's -- the flat slab's sigma_0 and Tolman length, and over
  droplets and bubbles (G' = -4, E8, R = 8, 12, 16 in boxes of side 4R) the
  Laplace-law sigma, the curved Tolman length and each run's R_s and
  sigma_s.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import lbinputs as L
import oracle
from oracle import analysis as A

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

GP = -4.0
RADII = (8, 12, 16)
STEPS = 2000


def _coex():
    ng, nl, _ = A.coexistence(GP, guess=(0.2, 3.0))
    return ng, nl


def _rel(a, b):
    return abs(a - b) / abs(b)


# --- flat slab --------------------------------------------------------------------
def _slab(ng, nl, nx=128, ny=4, steps=3000):
    return L.tanh_slab(nx, ny, 1, nx // 4, 3 * nx // 4, ng, nl, 2.0), (nx, ny), steps


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-3)])
def test_flat_interfaces_match_oracle(precision, tol):
    ng, nl = _coex()
    rho, shape, steps = _slab(ng, nl)
    lat = P.Lattice("D2Q9", shape, rho, L.E8_2D.bases, L.E8_2D.weights, precision=precision,
                    G=GP)
    lat.step(steps)
    assert lat.sync() == P.LB_OK
    got = lat.flat_interfaces()
    lat.close()
    o = oracle.Oracle("D2Q9", (1, shape[1], shape[0]), L.E8_2D.groups, tau=1.0, G=GP)
    o.init_equilibrium(rho)
    o.step(steps)
    want = A.flat_observables(o.pressure_tensor(), o.fields()["n"], D=2)
    assert len(got) == len(want) == 2
    for g, w in zip(got, want):
        assert (g["window_lo"], g["window_hi"]) == w["window"]
        assert bool(g["rising"]) == w["rising"]
        for k in ("sigma", "z_s", "z_e", "delta", "delta_ads", "n_l", "n_g"):
            assert _rel(g[k], w[k]) < tol, (k, g[k], w[k])


def test_flat_interfaces_3d_slab_fp64():
    ng, nl = _coex()
    nx, ny, nz = 48, 3, 2
    rho = L.tanh_slab(nx, ny, nz, 12, 36, ng, nl, 2.0)
    lat = P.Lattice("D3Q19", (nx, ny, nz), rho, L.E4_3D.bases, L.E4_3D.weights,
                    precision="fp64", G=GP)
    lat.step(200)
    got = lat.flat_interfaces()
    lat.close()
    o = oracle.Oracle("D3Q19", (nz, ny, nx), L.E4_3D.groups, tau=1.0, G=GP)
    o.init_equilibrium(rho)
    o.step(200)
    want = A.flat_observables(o.pressure_tensor(), o.fields()["n"], D=3)
    assert len(got) == len(want) == 2
    for g, w in zip(got, want):
        for k in ("sigma", "z_s", "z_e", "delta", "delta_ads"):
            assert _rel(g[k], w[k]) < 1e-11, (k, g[k], w[k])


# --- droplets and bubbles -----------------------------------------------------------
def _oracle_curved(args):
    R, bubble, ng, nl = args
    side = 4 * R
    c = (side / 2.0, side / 2.0)
    rin, rout = (ng, nl) if bubble else (nl, ng)
    rho = L.tanh_sphere(side, side, 1, R, rin, rout, 2.0, center=(c[0], c[1], 0.0))
    o = oracle.Oracle("D2Q9", (1, side, side), L.E8_2D.groups, tau=1.0, G=GP)
    o.init_equilibrium(rho)
    o.step(STEPS)
    r = A.curved_observables(o.pressure_tensor(), o.fields()["n"], c, 2, GP)
    r.pop("sigma_fn")
    return r


@pytest.fixture(scope="module")
def curved():
    ng, nl = _coex()
    jobs = [(R, b, ng, nl) for R in RADII for b in (False, True)]
    with mp.get_context("spawn").Pool(max(1, min(len(jobs), os.cpu_count() or 1))) as pool:
        want = pool.map(_oracle_curved, jobs)
    got = {"fp64": [], "fp32": []}
    for prec in got:
        for R, b, _, _ in jobs:
            side = 4 * R
            rin, rout = (ng, nl) if b else (nl, ng)
            rho = L.tanh_sphere(side, side, 1, R, rin, rout, 2.0,
                                center=(side / 2.0, side / 2.0, 0.0))
            lat = P.Lattice("D2Q9", (side, side), rho, L.E8_2D.bases, L.E8_2D.weights,
                            precision=prec, G=GP)
            lat.step(STEPS)
            assert lat.sync() == P.LB_OK
            got[prec].append(lat.curved_interface((side / 2.0, side / 2.0)))
            lat.close()
    # the flat sigma_0 of the same model (oracle)
    rho, shape, steps = _slab(ng, nl, steps=6000)
    o = oracle.Oracle("D2Q9", (1, shape[1], shape[0]), L.E8_2D.groups, tau=1.0, G=GP)
    o.init_equilibrium(rho)
    o.step(steps)
    sigma0 = float(np.mean([w["sigma"] for w in
                            A.flat_observables(o.pressure_tensor(), o.fields()["n"], D=2)]))
    return got, want, sigma0


def test_curved_fp64_matches_oracle_analysis(curved):
    got, want, _ = curved
    for g, w in zip(got["fp64"], want):
        assert g["bubble"] == w["bubble"]
        for k in ("n_in", "n_out", "P_in", "P_out", "dP", "R_e"):
            assert _rel(g[k], w[k]) < 1e-12, (k, g[k], w[k])
        for k in ("R_s", "sigma_s"):
            assert _rel(g[k], w[k]) < 1e-7, (k, g[k], w[k])


def test_curved_fp32_fits_within_1e3_of_oracle(curved):
    got, want, sigma0 = curved
    for g, w in zip(got["fp32"], want):
        for k in ("R_e", "dP", "R_s", "sigma_s"):
            assert _rel(g[k], w[k]) < 1e-3, (k, g[k], w[k])
    s32, _ = P.lb_fit_laplace(got["fp32"], 2)
    s_or, _ = A.laplace_sigma(want, 2)
    assert _rel(s32, s_or) < 1e-3, (s32, s_or)
    d32, _ = P.lb_fit_tolman(got["fp32"], 2, sigma0)
    d_or, _ = A.tolman_curved_fit(want, sigma0, 2)
    assert _rel(d32, d_or) < 1e-3, (d32, d_or)
    # and the physics the oracle pins: Laplace sigma near the flat one
    assert abs(s32 / sigma0 - 1.0) < 0.02


@pytest.mark.parametrize("center", [(12.0, 12.0, 12.0), (11.5, 12.25, 12.75)])
def test_curved_3d_fp64_matches_oracle_analysis(center):
    ng, nl = _coex()
    n3 = 24
    rho = L.tanh_sphere(n3, n3, n3, 6.0, nl, ng, 2.0, center=center)
    lat = P.Lattice("D3Q19", (n3, n3, n3), rho, L.E4_3D.bases, L.E4_3D.weights,
                    precision="fp64", G=GP)
    lat.step(150)
    assert lat.sync() == P.LB_OK
    g = lat.curved_interface(center)
    lat.close()
    o = oracle.Oracle("D3Q19", (n3, n3, n3), L.E4_3D.groups, tau=1.0, G=GP)
    o.init_equilibrium(rho)
    o.step(150)
    w = A.curved_observables(o.pressure_tensor(), o.fields()["n"], center, 3, GP)
    for k in ("n_in", "n_out", "P_in", "P_out", "dP", "R_e"):
        assert _rel(g[k], w[k]) < 1e-12, (k, g[k], w[k])
    for k in ("R_s", "sigma_s"):
        assert _rel(g[k], w[k]) < 1e-7, (k, g[k], w[k])


def test_interface_calls_allocate_nothing_and_leave_the_state():
    """The observables stage in the idle population buffer: the state and
    the next steps are unchanged by them."""
    ng, nl = _coex()
    rho = L.tanh_sphere(40, 40, 1, 10.0, nl, ng, 2.0, center=(20.0, 20.0, 0.0))
    a = P.Lattice("D2Q9", (40, 40), rho, L.E8_2D.bases, L.E8_2D.weights, precision="fp64", G=GP)
    b = P.Lattice("D2Q9", (40, 40), rho, L.E8_2D.bases, L.E8_2D.weights, precision="fp64", G=GP)
    for k in range(3):
        a.step(7)
        b.step(7)
        a.observables()
        a.curved_interface((20.0, 20.0))
        a.flat_interfaces()
        a.pressure_tensor()
        a.fields()
    assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()
