"""The adjoint tuning configuration as written, on the GPU.

D2Q9 with the E8 stencil (groups (1,0), (1,1), (2,0), (2,1), (2,2)), G' =
-3 from its eq. SCMaxwell pair (0.456, 2.25).  A flat 512 x 4 slab,
shifted-binary32 forward, 4,000 steps, checkpoint every 100 steps, binary64
adjoint: Newton steps on the five group weights and G (minimum-norm, six
unknowns for four targets; the gradient solve replacing the hand tuning of
Sec. V) take its (sigma_0, delta) to 1.2 x and 0.5 x their untuned values
while the interface width and the density ratio stay at theirs -- all four
within 1e-3 relative.  The companion droplet (512 x 512, R = 64, binary32)
is measured with the untuned and the tuned stencil by the library's
curved-interface observables after 40,000 steps (at the configuration's
4,000 steps its Laplace pressure is a third of its equilibrium value and the
surface of tension is not yet defined).  The untuned droplet has its
surface of tension inside the equimolar radius (a positive curvature
correction, like the flat Tolman length) and sigma_s within 10 % of the
flat sigma_0; the tuned one stays stable with a positive Laplace pressure.
What the tuned droplet does is recorded, not pinned: moving the five
weights freely breaks the stencil's isotropy (the paper's tables keep it
by construction), and the droplet's Laplace estimate Delta P R_e falls
(0.84 x) where the slab's sigma_0 rose 1.2 x; solving within the isotropic
table tab:e4e6e8_tuning_6_2d instead reaches the same slab targets with
knobs whose droplet is unstable.
"""
import numpy as np
import pytest

import lbinputs as L

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")
AD = pytest.importorskip("paper_2505_23647_gb300.adjoint")

N_GAS, N_LIQ = 0.4558015024901948, 2.249571904134268
NX, NY, STEPS, K = 512, 4, 4000, 100


def _weights_of(k):
    return [float(v) for v in k]


BASES = L.E8_2D.bases


def _slab(W, G):
    rho = L.tanh_slab(NX, NY, 1, NX // 4, 3 * NX // 4, N_GAS, N_LIQ, 2.0)
    return P.Lattice("D2Q9", (NX, NY), rho, BASES, W, precision="fp32", G=G)


def _droplet(W, G, steps=40000):
    n = 512
    rho = L.tanh_sphere(n, n, 1, 64.0, N_LIQ, N_GAS, 2.0, center=(n / 2.0, n / 2.0, 0.0))
    lat = P.Lattice("D2Q9", (n, n), rho, BASES, W, precision="fp32", G=G)
    lat.step(steps)
    assert lat.sync() == P.LB_OK
    r = lat.curved_interface((n / 2.0, n / 2.0))
    lat.close()
    return r


@pytest.fixture(scope="module")
def solve():
    knobs0, G0 = np.array([float(w) for w in L.E8_2D.weights]), -3.0
    v0, _, _ = AD.slab_observables(lambda: _slab(_weights_of(knobs0), G0), STEPS, NX // 2, 0,
                                   N_LIQ, N_GAS, K)
    targets = v0 * np.array([1.2, 0.5, 1.0, 1.0])
    knobs, G, vals, hist = AD.tune_slab(_slab, _weights_of, knobs0, G0, targets, STEPS, NX // 2, 0,
                                        N_LIQ, N_GAS, K, rtol=1e-3, max_iter=12)
    return knobs0, G0, v0, targets, knobs, G, vals, hist


def test_gradient_solve_hits_targets(solve):
    knobs0, G0, v0, targets, knobs, G, vals, hist = solve
    assert v0[0] > 0 and v0[1] > 0 and v0[3] > 1.0
    assert np.max(np.abs(vals / targets - 1.0)) < 1e-3, (knobs, G, vals, targets, hist)


def test_droplet_companion_before_and_after(solve):
    knobs0, G0, v0, targets, knobs, G, vals, hist = solve
    before = _droplet(_weights_of(knobs0), G0)
    after = _droplet(_weights_of(knobs), G)
    for r in (before, after):
        assert not r["bubble"] and r["dP"] > 0
        assert 0.8 * 64 < r["R_e"] < 1.2 * 64
    assert before["R_s"] < before["R_e"]
    assert abs(before["sigma_s"] / v0[0] - 1.0) < 0.1, (before, v0)
