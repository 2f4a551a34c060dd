"""lb_step replays a captured CUDA graph of 32 steps for long runs: the
state after one long call equals, bit for bit, the state after the same
number of single steps -- for the binary64 two-kernel path, the fused
binary32 D2Q9 and D3Q19 (TMA) kernels, odd remainders and a buffer parity
that changes between calls; and options set between calls are honoured."""
import numpy as np
import pytest

import lbinputs as L

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

CASES = [
    ("D2Q9", (61, 47), L.E8_2D, "fp64"),
    ("D2Q9", (64, 48), L.E8_2D, "fp32"),
    ("D3Q19", (64, 32, 16), L.E8_3D, "fp32"),
]


def _lat(lattice, shape, st, prec):
    # a droplet at G' = -3 from its coexistence densities (a stable run)
    ng, nl = 0.4558015024901948, 2.249571904134268
    rho = L.tanh_sphere(*shape, min(shape) / 4.0, nl, ng, 2.0) if len(shape) == 3 else \
        L.tanh_sphere(shape[0], shape[1], 1, min(shape) / 4.0, nl, ng, 2.0)
    return P.Lattice(lattice, shape, rho, st.bases, st.weights, precision=prec, G=-3.0)


@pytest.mark.parametrize("lattice,shape,st,prec", CASES)
def test_graph_replay_equals_single_steps(lattice, shape, st, prec):
    a = _lat(lattice, shape, st, prec)
    b = _lat(lattice, shape, st, prec)
    for n in (131, 7, 100, 97):
        l0 = a.launches()
        a.step(n)
        assert a.launches() > l0
        for _ in range(n):
            b.step(1)
        assert a.sync() == b.sync() == P.LB_OK
        assert np.array_equal(a.state(), b.state()), n
    assert a.observables()["step"] == b.observables()["step"] == 335
    a.close()
    b.close()


def test_options_set_between_long_runs_take_effect():
    shape = (64, 32, 16)
    a = _lat("D3Q19", shape, L.E8_3D, "fp32")
    b = _lat("D3Q19", shape, L.E8_3D, "fp32")
    a.step(100)
    b.step(100)
    P.lb_set_option(a.ctx, P.LB_OPT_FUSED, 0)     # two-kernel path from now on
    assert P.lb_fused_active(a.ctx) == 0
    a.step(100)
    P.lb_set_option(b.ctx, P.LB_OPT_FUSED, 0)
    for _ in range(100):
        b.step(1)
    assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()
