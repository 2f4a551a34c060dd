"""Degenerate and ragged lattices on every path, against the oracle.

Periodic lattices smaller than the stencil (1 x 1, 1 x 1 x 1, 2 x 3, 3 x 2 x 2,
a single row or column) make every neighbour an image of the node itself or
of a few nodes: binary64 must still match the oracle bit for bit, binary32
within its tolerance; a uniform state is a fixed point to rounding; a
zero-step call changes nothing; an initial density that is not positive
and finite is rejected by lb_create."""
import numpy as np
import pytest

import lbinputs as L
import oracle

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

SHAPES = [
    ("D2Q9", (1, 1), L.E8_2D),
    ("D2Q9", (2, 3), L.E8_2D),
    ("D2Q9", (1, 17), L.E4_2D),
    ("D2Q9", (19, 1), L.E6_2D),
    ("D3Q19", (1, 1, 1), L.E8_3D),
    ("D3Q19", (3, 2, 2), L.E8_3D),
    ("D3Q19", (1, 5, 7), L.E4_3D),
    ("D3Q19", (9, 1, 1), L.E8_3D),
]


def _rho(shape, seed):
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    rng = np.random.default_rng(seed)
    return 0.8 + 0.6 * rng.random((nz, ny, nx))


@pytest.mark.parametrize("lattice,shape,st", SHAPES)
def test_tiny_lattices_fp64_bitwise(lattice, shape, st):
    rho = _rho(shape, 3)
    lat = P.Lattice(lattice, shape, rho, st.bases, st.weights, precision="fp64", tau=0.9, G=-2.0)
    lat.step(20)
    assert lat.sync() == P.LB_OK
    nz = shape[2] if len(shape) > 2 else 1
    o = oracle.Oracle(lattice, (nz, shape[1], shape[0]), st.groups, tau=0.9, G=-2.0)
    o.init_equilibrium(rho)
    o.step(20)
    assert np.array_equal(lat.state().reshape(o.f.shape), o.f)
    lat.close()


@pytest.mark.parametrize("lattice,shape,st", SHAPES)
def test_tiny_lattices_fp32(lattice, shape, st):
    rho = _rho(shape, 4)
    lat = P.Lattice(lattice, shape, rho, st.bases, st.weights, precision="fp32", tau=0.9, G=-2.0)
    lat.step(20)
    assert lat.sync() == P.LB_OK
    nz = shape[2] if len(shape) > 2 else 1
    o = oracle.Oracle(lattice, (nz, shape[1], shape[0]), st.groups, tau=0.9, G=-2.0)
    o.init_equilibrium(rho)
    o.step(20)
    n, _ = lat.fields()
    ref = o.fields()["n"]
    assert np.max(np.abs(n - ref) / ref) < 1e-5
    lat.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("lattice,shape,st", [("D2Q9", (37, 29), L.E8_2D),
                                              ("D3Q19", (64, 32, 16), L.E8_3D)])
def test_uniform_state_is_a_fixed_point(lattice, shape, st, precision):
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    rho = np.full((nz, ny, nx), 1.3)
    lat = P.Lattice(lattice, shape, rho, st.bases, st.weights, precision=precision, G=-4.0)
    f0 = lat.state()
    lat.step(25)
    assert lat.sync() == P.LB_OK
    f1 = lat.state()
    # f_eq of the rounded n is not exactly the initial f: rounding-level drift
    # (the oracle's own fixed point is held to 8 ulp)
    tol = 8 * np.finfo(float).eps if precision == "fp64" else 1e-6
    assert np.max(np.abs(f1 - f0)) <= tol * np.max(np.abs(f0))
    lat.step(0)
    assert np.array_equal(lat.state(), f1)
    lat.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_initial_density_not_positive_and_finite_is_rejected(precision, bad):
    """lb_create checks the uploaded densities on the device: LB_EINVAL, and
    a valid creation afterwards still works (nothing left behind)."""
    p = P.make_params("D3Q19", (32, 8, 9), precision)
    rho = np.ones(32 * 8 * 9)
    rho[123] = bad
    with pytest.raises(P.LbError) as ei:
        P.lb_create(p, rho)
    assert ei.value.status == P.LB_EINVAL
    ctx = P.lb_create(p, np.ones(32 * 8 * 9))
    P.lb_destroy(ctx)
