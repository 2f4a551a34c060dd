"""Interface observables of the shifted-binary32 path against binary64.

The accuracy the FP32 path has to deliver is stated on the quantities the
method is run for: surface tension and Tolman length within 1e-3 relative
of the binary64 result.

Coupling G' = -3 (below the critical -e^2/3 of psi = exp(-1/n)), runs
started from the coexistence densities of eq. SCMaxwell (0.456, 2.25).

* Flat slab (Sec. V A set-up, D2Q9 E8): sigma_0 and delta = z_e - z_s from
  the lattice pressure tensor (Appendix E, eqs. SCTolmanFlat / deltaads)
  after 4000 steps, GPU FP32 against the FP64 oracle itself.
* Droplets (Laplace law, Sec. V B): the slope of Delta P against 1/R_e over
  four radii, GPU FP32 against the GPU's binary64 path (which matches the
  oracle bit for bit, tests/test_gpu_parity.py).
"""
import numpy as np
import pytest

import lbinputs as L
import oracle
from oracle import analysis as A

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

G, CONV = -3.0, "literal"
GP = G
N_GAS, N_LIQ = 0.456, 2.25
REL = 1e-3


def _rel(a, b):
    return abs(a - b) / abs(b)


def test_flat_slab_sigma_and_tolman_fp32_vs_oracle():
    nx, ny, steps = 256, 4, 4000
    st = L.E8_2D
    rho = L.tanh_slab(nx, ny, 1, 64, 192, N_GAS, N_LIQ, 2.0)
    lat = P.Lattice("D2Q9", (nx, ny), rho, st.bases, st.weights, precision="fp32", G=G,
                    convention=CONV)
    lat.step(steps)
    assert lat.sync() == P.LB_OK
    n32, _ = lat.fields()
    obs32 = A.flat_observables(lat.pressure_tensor(), n32, D=2)
    lat.close()

    o = oracle.Oracle("D2Q9", (1, ny, nx), st.groups, tau=1.0, G=G, convention=CONV)
    o.init_equilibrium(rho)
    o.step(steps)
    obs64 = A.flat_observables(o.pressure_tensor(), o.fields()["n"], D=2)

    assert len(obs32) == len(obs64) == 2
    for a, b in zip(obs32, obs64):
        assert a["window"] == b["window"]
        assert _rel(a["sigma"], b["sigma"]) < REL, (a["sigma"], b["sigma"])
        assert _rel(a["delta"], b["delta"]) < REL, (a["delta"], b["delta"])
        assert _rel(a["delta_ads"], b["delta_ads"]) < REL
        assert _rel(a["n_l"], b["n_l"]) < 1e-5 and _rel(a["n_g"], b["n_g"]) < 1e-5
    # the slab is a physical one: two interfaces, positive tension
    assert obs64[0]["sigma"] > 0 and obs64[1]["sigma"] > 0


def _laplace_sigma(precision, radii, side=96, steps=6000):
    st = L.E8_2D
    inv_r, dp = [], []
    for R in radii:
        rho = L.tanh_sphere(side, side, 1, R, N_LIQ, N_GAS, 2.0)
        lat = P.Lattice("D2Q9", (side, side), rho, st.bases, st.weights, precision=precision,
                        G=G, convention=CONV)
        lat.step(steps)
        assert lat.sync() == P.LB_OK
        n, _ = lat.fields()
        lat.close()
        n2 = n[0]
        n_in, n_out = float(n2[side // 2, side // 2]), float(n2[0, 0])
        inv_r.append(1.0 / A.equimolar_radius(n, n_in, n_out))
        dp.append(A.bulk_pressure(n_in, GP) - A.bulk_pressure(n_out, GP))
    slope, _ = A.laplace_fit(inv_r, dp)
    return slope, np.array(inv_r), np.array(dp)


def test_droplet_laplace_sigma_fp32_vs_fp64():
    radii = (12, 16, 20, 24)
    s32, ir32, dp32 = _laplace_sigma("fp32", radii)
    s64, ir64, dp64 = _laplace_sigma("fp64", radii)
    assert s64 > 0
    assert _rel(s32, s64) < REL, (s32, s64)
    assert np.max(np.abs(ir32 - ir64) / ir64) < REL
    assert np.max(np.abs(dp32 - dp64) / dp64) < REL
