"""Observables of shifted-binary32 D3Q19 lattices on the TMA path.

lb_observables measures such a lattice with the fused step kernel's
measuring instantiation (one read of the populations, the force from psi
planes in registers, no store).  Checked here against the binary64 oracle's
observables of the same state (the GPU state widened): the mass to 1e-12
relative (each node's density is the binary32 sum of its populations plus
that sum's rounding errors, summed with compensation); the momentum
sum_x (j + F/2) and max |u|, binary32 node values, within 2^-20 of the
scale of the terms they sum (_bounds); the density extrema, binary32
densities, to 2^-20 relative; against the generic observables
pass on the same state (the option that turns the TMA kernel off selects
it) to the same bounds; and the call leaves the state and the step counter
alone.  A measuring pass whose waits give up reports LB_ECUDA (its blocks
write a NaN mass) and does not count as a step.
"""
import numpy as np
import pytest

import lbinputs as L
import oracle
from oracle import analysis as A

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

CASES = [
    # shape, stencil, G, psi_eps, steps (nz not a multiple of the z chunk:
    # a ragged last chunk)
    ((64, 32, 36), L.E8_3D, -4.0, None, 40),
    ((96, 40, 37), L.E8_3D, -4.0, None, 25),
    ((64, 24, 20), L.E4_3D, -4.0, None, 30),
    ((64, 32, 30), L.E8_3D, None, "psi_eps", 30),
]


def _lattice(shape, st, G, eps_kind):
    if eps_kind:
        pe = L.PSI_EPS_BUBBLE
        rho = L.tanh_sphere(*shape, 0.25 * min(shape), pe["n_gas"], pe["n_liquid"], 2.0)
        lat = P.Lattice("D3Q19", shape, rho, st.bases, st.weights, precision="fp32", tau=1.0,
                        G=pe["Gp"], psi_eps=pe["eps"])
        o = oracle.Oracle("D3Q19", shape[::-1], st.groups, tau=1.0, G=pe["Gp"], psi_kind=1,
                          psi_eps=pe["eps"])
    else:
        # a drop started from the coexistence pair of G' = G (eq. SCMaxwell)
        ng, nl, _ = A.coexistence(G, guess=(0.2, 3.0))
        rho = L.tanh_sphere(*shape, 0.25 * min(shape), nl, ng, 2.0)
        lat = P.Lattice("D3Q19", shape, rho, st.bases, st.weights, precision="fp32", tau=1.0, G=G)
        o = oracle.Oracle("D3Q19", shape[::-1], st.groups, tau=1.0, G=G)
    return lat, o


def _bounds(o, st):
    """Rounding scales of the binary32 node values: j sums populations of
    size ~ w_i n, F sums terms G' w psi(x) psi(x +- e) e; s(x) = n(x) +
    |G'| psi(x) sum_e w |e|_1 psi(x + e) bounds both, and a binary32
    evaluation errs by a few units of 2^-24 of it.  Returns the momentum
    bound 2^-20 sum_x s, the max |u| bound 2^-20 max_x s / n and n itself."""
    fl = o.fields()
    n, ps = fl["n"], fl["psi"]
    vec, w = oracle.pair_arrays(st.groups, 3)
    acc = np.zeros_like(ps)
    for (ex, ey, ez), wt in zip(vec, w):
        l1 = abs(ex) + abs(ey) + abs(ez)
        for sg in (1, -1):
            acc += wt * l1 * np.roll(ps, shift=(-sg * ez, -sg * ey, -sg * ex), axis=(0, 1, 2))
    s = n + abs(o.Gp) * ps * acc
    return 2.0 ** -20 * float(np.sum(s)), 2.0 ** -20 * float(np.max(s / n))


def _check(ob, ref, bnd):
    tol_mom, tol_u = bnd
    assert abs(ob["mass"] - ref["mass"]) <= 1e-12 * ref["mass"], (ob["mass"], ref["mass"])
    for k in range(3):
        assert abs(ob["mom"][k] - ref["mom"][k]) <= tol_mom, (k, ob["mom"], ref["mom"], tol_mom)
    assert abs(ob["umax"] - ref["umax"]) <= tol_u, (ob["umax"], ref["umax"], tol_u)
    for k in ("rho_min", "rho_max"):
        assert abs(ob[k] - ref[k]) <= 2.0 ** -20 * ref[k], (k, ob[k], ref[k])


@pytest.mark.parametrize("shape,st,G,eps_kind,steps", CASES)
def test_measuring_pass_matches_oracle_and_generic_pass(shape, st, G, eps_kind, steps):
    lat, o = _lattice(shape, st, G, eps_kind)
    assert P.lb_fused_active(lat.ctx) == 2
    lat.step(steps)
    assert lat.sync() == P.LB_OK
    f = lat.state()
    ob = lat.observables()
    assert ob["status"] == P.LB_OK and ob["step"] == steps
    o.f = f
    ref = o.observables()
    bnd = _bounds(o, st)
    _check(ob, ref, bnd)
    # the generic pass on the same state
    P.lb_set_option(lat.ctx, P.LB_OPT_TMA, 0)
    assert P.lb_fused_active(lat.ctx) == 1
    og = lat.observables()
    assert og["status"] == P.LB_OK
    _check(og, ref, bnd)
    assert abs(ob["mass"] - og["mass"]) <= 1e-12 * og["mass"]
    assert np.array_equal(lat.state(), f)
    lat.close()


def test_measuring_pass_leaves_state_and_step():
    shape = (64, 32, 36)
    a, _ = _lattice(shape, L.E8_3D, -4.0, None)
    b, _ = _lattice(shape, L.E8_3D, -4.0, None)
    for _ in range(3):
        a.step(5)
        b.step(5)
        for _ in range(2):
            assert a.observables()["status"] == P.LB_OK
    assert np.array_equal(a.state(), b.state())
    ca, cb = P.lb_device_counters(a.ctx), P.lb_device_counters(b.ctx)
    assert ca["device_step"] == cb["device_step"] == 15
    assert ca["blocks_done"] == 0
    a.close()
    b.close()


def test_measuring_pass_wait_that_gives_up():
    shape = (64, 32, 36)
    lat, _ = _lattice(shape, L.E8_3D, -4.0, None)
    P.lb_set_option(lat.ctx, P.LB_OPT_ZCHUNK, 18)
    lat.step(2)
    assert lat.sync() == P.LB_OK
    P.lb_set_option(lat.ctx, P.LB_OPT_WAIT_POLLS, 0)
    with pytest.raises(P.LbError) as ei:
        lat.observables()
    assert ei.value.status == P.LB_ECUDA
    c = P.lb_device_counters(lat.ctx)
    assert c["timeouts"] == (64 // 32) * (32 // 8) * 2
    assert c["device_step"] == 2 and c["blocks_done"] == 0
    lat.close()
