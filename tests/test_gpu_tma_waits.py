"""GPU test of the TMA fused D3Q19 kernel's bounded waits.

A wait that gives up is reported, not hidden: with the poll bound set to
zero every CTA's first mbarrier wait gives up at once (a bound that is never
met; no fault or hang is involved), the CTA lets its copies land and leaves;
lb_sync returns LB_ECUDA, every CTA is counted once, and the device step
counter still advances by one per step, also for the steps after it.
"""
import numpy as np
import pytest

import lbinputs as L

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")


def test_wait_that_gives_up_is_reported():
    shape = (64, 32, 36)
    rho = L.tanh_sphere(*shape, 8.0, 1.9, 0.15, 2.0)
    lat = P.Lattice("D3Q19", shape, rho, L.E8_3D.bases, L.E8_3D.weights, precision="fp32",
                    tau=1.0, G=-4.0)
    assert P.lb_fused_active(lat.ctx) == 2
    P.lb_set_option(lat.ctx, P.LB_OPT_ZCHUNK, 18)
    f0 = lat.state()
    lat.step(1)
    assert lat.sync() == P.LB_OK
    c = P.lb_device_counters(lat.ctx)
    assert c["device_step"] == 1 and c["timeouts"] == 0 and c["blocks_done"] == 0

    P.lb_set_option(lat.ctx, P.LB_OPT_WAIT_POLLS, 0)
    lat.step(1)
    with pytest.raises(P.LbError) as ei:
        lat.sync()
    assert ei.value.status == P.LB_ECUDA
    ctas = (64 // 32) * (32 // 8) * 2      # 36 planes in chunks of 18
    c = P.lb_device_counters(lat.ctx)
    assert c["timeouts"] == ctas
    assert c["blocks_done"] == 0
    assert c["device_step"] == 2

    # back to the default bound: the counters stay consistent, the timeout
    # stays reported
    P.lb_set_option(lat.ctx, P.LB_OPT_WAIT_POLLS, 1 << 26)
    lat.set_state(f0)
    lat.step(3)
    with pytest.raises(P.LbError) as ei:
        lat.sync()
    assert ei.value.status == P.LB_ECUDA
    c = P.lb_device_counters(lat.ctx)
    assert c["timeouts"] == ctas and c["blocks_done"] == 0 and c["device_step"] == 5
    assert np.all(np.isfinite(lat.state()))
    lat.close()


def test_wait_polls_option_range():
    shape = (64, 32, 16)
    rho = np.ones(shape[::-1])
    lat = P.Lattice("D3Q19", shape, rho, L.E4_3D.bases, L.E4_3D.weights, precision="fp32")
    with pytest.raises(P.LbError):
        P.lb_set_option(lat.ctx, P.LB_OPT_WAIT_POLLS, -1)
    with pytest.raises(P.LbError):
        P.lb_set_option(lat.ctx, P.LB_OPT_WAIT_POLLS, (1 << 40) + 1)
    lat.close()
