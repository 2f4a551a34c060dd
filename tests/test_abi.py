"""C ABI checks that need no GPU: the library builds, loads, exports every
function include/sclbm.h declares, expands stencils in the same canonical
pair order as the oracle, reports stencil moments, and rejects invalid
parameters before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import lbinputs as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2505_23647_gb300 as pkg
    return pkg


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(P):
    lib = ctypes.CDLL(P.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(P.EXPORTED) <= set(names)


@pytest.mark.parametrize("stencil", [L.E4_2D, L.E6_2D, L.E8_2D, L.E4_3D, L.E8_3D,
                                     L.stencil_e4e6_tuning_8(3, -0.3, 0.1),
                                     L.stencil_e4e6e8_tuning_6(2, -0.4, 0.18, 0.3)])
def test_pair_order_matches_oracle(P, stencil):
    import oracle
    v, w, info = P.lb_expand_stencil(stencil.dim, stencil.bases, stencil.weights)
    ov, ow = oracle.pair_arrays(stencil.groups, stencil.dim)
    assert np.array_equal(v, ov)
    assert np.array_equal(w, ow)
    assert info.n_vectors == 2 * len(ov)


def test_stencil_moments(P):
    from oracle import stencil as st
    for s in (L.E8_2D, L.E8_3D):
        _, _, info = P.lb_expand_stencil(s.dim, s.bases, s.weights)
        e2, e4, e6, e8 = st.isotropy_coeffs(s.groups, s.dim)
        for got, want in ((info.e2, e2), (info.e4, e4), (info.e6, e6), (info.e8, e8)):
            assert abs(got - float(want)) < 1e-14
        assert max(info.iso_residual[:3]) < 1e-14      # isotropic through 8th order
        assert info.radius == 2
    _, _, info = P.lb_expand_stencil(2, L.E4_2D.bases, L.E4_2D.weights)
    assert info.iso_residual[0] < 1e-15 and info.iso_residual[1] > 0.1


@pytest.mark.parametrize("bases,weights", [
    ([[1, 0], [1, 0]], [0.1, 0.2]),        # repeated group
    ([[0, 0]], [1.0]),                     # zero vector
    ([[5, 0]], [1.0]),                     # beyond LB_MAX_RADIUS
    ([[1, 0]], [float("nan")]),
])
def test_invalid_stencils_rejected(P, bases, weights):
    with pytest.raises(P.LbError) as ei:
        P.lb_expand_stencil(2, bases, weights)
    assert ei.value.status == P.LB_EINVAL


@pytest.mark.parametrize("field,value", [("tau", 0.5), ("tau", float("nan")), ("nx", 0),
                                         ("lattice", 7), ("precision", 9),
                                         ("g_convention", 3), ("nz", 2)])
def test_invalid_params_rejected_on_host(P, field, value):
    p = P.make_params("D2Q9", (8, 8))
    setattr(p, field, value)
    with pytest.raises(P.LbError) as ei:
        P.lb_create(p, np.ones(256))
    assert ei.value.status == P.LB_EINVAL


def test_laplace_and_tolman_fits_match_the_oracle_fits(P):
    """lb_fit_laplace / lb_fit_tolman are host arithmetic: the same lines as
    the oracle's laplace_sigma / tolman_curved_fit on made-up results."""
    from oracle import analysis as A
    rng = np.random.default_rng(7)
    runs = []
    for R in (8.0, 11.0, 15.0, 22.0):
        for b in (False, True):
            Re = R * (1 + 0.01 * rng.standard_normal())
            Rs = Re - (0.8 if not b else -0.5)
            dP = 0.18 / Re * (1 + 0.05 * rng.standard_normal())
            runs.append({"n_in": 0.3 if b else 3.8, "n_out": 3.8 if b else 0.3, "P_in": 0.1 + dP,
                         "P_out": 0.1, "dP": dP, "R_e": Re, "R_s": Rs, "sigma_s": dP * Rs,
                         "bubble": b})
    s, i = P.lb_fit_laplace(runs, 2)
    s0, i0 = A.laplace_sigma(runs, 2)
    assert s == pytest.approx(s0, rel=1e-12) and i == pytest.approx(i0, rel=1e-9, abs=1e-15)
    d, j = P.lb_fit_tolman(runs, 2, 0.18)
    d0, j0 = A.tolman_curved_fit(runs, 0.18, 2)
    assert d == pytest.approx(d0, rel=1e-12) and j == pytest.approx(j0, rel=1e-12)
    s3, _ = P.lb_fit_laplace(runs, 3)
    assert s3 == pytest.approx(s0 / 2, rel=1e-12)
    with pytest.raises(P.LbError):
        P.lb_fit_laplace(runs[:1], 2)
