"""Binary32 steps move no mass systematically (eqs. lbm, omega_i, f_eq: the
collision conserves n exactly, so the lattice mass is constant).

Each binary32 constant rounded on its own (the weights, keep = 1 - omega,
omega w per velocity class) makes the density coefficient of a step miss 1
by a few 1e-8, the same way at every node and step: at tau = 0.8 the mass
of a D2Q9 lattice drifted by about 5.6e-8 of (n - rho0) per step.  The
library picks the binary32 constants so that the coefficient is exactly 1
(a few ulps of nudging).  What remains is the rounding of the binary32
sums themselves: the nodes of a bulk phase hold nearly the same populations,
so the rounding of n = sum_i g_i is the same at each of them and repeats
every step, and the mass changes by (1 - keep) times it per bulk node and
step.  That depends on the bulk values (measured 0.3e-9 to 2.6e-9 of the
mass per step over these cases, at tau = 1 too) and is not a property of
the constants.  The bound below is 5e-9 per step, 11 times under the
removed bias at tau = 0.8; the runs are deterministic.  Checked on every
binary32 path at relaxation times on both sides of 1, on the lattice mass
(binary64 sum of the densities).
"""
import numpy as np
import pytest

import lbinputs as L

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

G, N_GAS, N_LIQ = -3.0, 0.456, 2.25      # coexistence at G' = -3 (stable two-phase runs)

CASES = []
for tau in (0.6, 0.8, 1.7):
    for mode in ("fused", "two-kernel"):
        CASES.append(("D2Q9", (256, 256), L.E8_2D, tau, mode, 2000))
for tau in (0.8, 1.3):
    for mode in ("tma", "cpasync", "two-kernel"):
        CASES.append(("D3Q19", (64, 64, 32), L.E8_3D, tau, mode, 400))


@pytest.mark.parametrize("lattice,shape,st,tau,mode,steps", CASES)
def test_mass_is_conserved(lattice, shape, st, tau, mode, steps):
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    rho = L.tanh_sphere(nx, ny, nz, 0.3 * min(nx, ny), N_LIQ, N_GAS, 2.0)
    lat = P.Lattice(lattice, shape, rho, st.bases, st.weights, precision="fp32", tau=tau, G=G)
    P.lb_set_option(lat.ctx, P.LB_OPT_FUSED, mode != "two-kernel")
    if lattice == "D3Q19":
        P.lb_set_option(lat.ctx, P.LB_OPT_TMA, mode == "tma")
    want = {"fused": 3, "tma": 2, "cpasync": 1, "two-kernel": 0}[mode]
    assert P.lb_fused_active(lat.ctx) == want
    m0 = lat.observables()["mass"]
    lat.step(steps)
    ob = lat.observables()
    lat.close()
    assert ob["status"] == P.LB_OK
    drift = abs(ob["mass"] - m0) / m0
    assert drift < 5e-9 * steps, drift
