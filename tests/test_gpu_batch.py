"""Batched 2D lattices (lb_batch_*) and the fused D2Q9 kernel.

* a batch of uneven boxes (sizes that are not multiples of any tile, E4 /
  E6 / E8 stencils, droplets and bubbles) against the FP64 oracle per
  member, density within the binary32 tolerance after 100 steps;
* every tile shape, the graph replay and stepping each member on its own
  give the same populations bit for bit (the tiling never changes what a
  node computes);
* lb_batch_tune leaves the members' states and counters as they were;
* the many-instance workload (64 seeded instances, 4.55 M nodes, one
  launch per step in a CUDA graph): sampled nodes recomputed by the oracle
  from the GPU's own state, and per-member mass conservation;
* members that the batch cannot step are refused on the host.
"""
import numpy as np
import pytest

import lbinputs as L
import oracle

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")

G, CONV = -3.0, "literal"         # G' = -3: below the critical coupling, phases coexist
N_GAS, N_LIQ = 0.456, 2.25

MEMBERS = [
    # (nx, ny, stencil, radius, droplet)
    (64, 64, L.E8_2D, 14.0, True),
    (96, 64, L.E6_2D, 18.0, False),
    (40, 36, L.E4_2D, 9.0, True),
    (50, 70, L.E8_2D, 12.0, False),
    (128, 128, L.E8_2D, 30.0, True),
]


def _rho(nx, ny, radius, droplet):
    if droplet:
        return L.tanh_sphere(nx, ny, 1, radius, N_LIQ, N_GAS, 2.0)
    return L.tanh_sphere(nx, ny, 1, radius, N_GAS, N_LIQ, 2.0)


def _make(members=MEMBERS):
    lats = []
    for nx, ny, st, r, drop in members:
        lats.append(P.Lattice("D2Q9", (nx, ny), _rho(nx, ny, r, drop), st.bases, st.weights,
                              precision="fp32", G=G, convention=CONV))
    return lats


def _close(batch, lats):
    batch.close()
    for l in lats:
        l.close()


def test_fused2d_path_is_active():
    lats = _make(MEMBERS[:1])
    assert P.lb_fused_active(lats[0].ctx) == 3
    lats[0].close()


def test_batch_matches_oracle_per_member():
    lats = _make()
    b = P.Batch(lats)
    b.step(100)                       # one graph replay of 64 + 36 single launches
    assert b.sync() == P.LB_OK
    assert b.launches() == 100
    for lat, (nx, ny, st, r, drop) in zip(lats, MEMBERS):
        o = oracle.Oracle("D2Q9", (1, ny, nx), st.groups, tau=1.0, G=G, convention=CONV)
        o.init_equilibrium(_rho(nx, ny, r, drop))
        o.step(100)
        n_gpu, _ = lat.fields()
        n_ref = o.fields()["n"]
        err = np.max(np.abs(n_gpu - n_ref) / n_ref)
        assert err < 1e-5, (nx, ny, err)
        assert lat.observables()["step"] == 100
    _close(b, lats)


def test_tile_shapes_graph_and_single_steps_agree_bitwise():
    ref = None
    for shape in range(len(P.lb_batch_tile_shapes())):
        lats = _make()
        b = P.Batch(lats)
        b.set_tile(shape)
        b.step(70)
        assert b.sync() == P.LB_OK
        states = [l.state() for l in lats]
        _close(b, lats)
        if ref is None:
            ref = states
        else:
            for a, c in zip(states, ref):
                assert np.array_equal(a, c), shape
    # the same steps one launch at a time, and each member on its own
    lats = _make()
    b = P.Batch(lats)
    for _ in range(70):
        b.step(1)
    assert b.sync() == P.LB_OK
    for a, c in zip([l.state() for l in lats], ref):
        assert np.array_equal(a, c)
    _close(b, lats)
    lats = _make()
    for l, c in zip(lats, ref):
        l.step(70)
        assert l.sync() == P.LB_OK
        assert np.array_equal(l.state(), c)
        l.close()


def test_members_stepped_alone_between_batch_calls():
    lats = _make()
    b = P.Batch(lats)
    b.step(3)
    lats[1].step(1)                   # one member moves on its own
    b.step(4)
    assert b.sync() == P.LB_OK
    got = [l.state() for l in lats]
    _close(b, lats)
    lats = _make()
    for i, l in enumerate(lats):
        l.step(8 if i == 1 else 7)
        assert np.array_equal(l.state(), got[i])
        l.close()


def test_tune_restores_the_members():
    lats = _make()
    b = P.Batch(lats)
    b.step(5)
    before = [l.state() for l in lats]
    best, ms = b.tune(steps_per_trial=8)
    assert 0 <= best < len(ms) and np.all(ms > 0)
    assert b.tile() == best
    for l, s in zip(lats, before):
        assert np.array_equal(l.state(), s)
        assert l.observables()["step"] == 5
    b.step(5)
    assert b.sync() == P.LB_OK
    _close(b, lats)


def test_unsupported_members_are_refused():
    l2 = _make(MEMBERS[:1])[0]
    l64 = P.Lattice("D2Q9", (32, 32), np.full((1, 32, 32), 1.0), L.E8_2D.bases,
                    L.E8_2D.weights, precision="fp64")
    l3 = P.Lattice("D3Q19", (16, 16, 16), np.full((16, 16, 16), 1.0), L.E4_3D.bases,
                   L.E4_3D.weights, precision="fp32")
    for bad in ([l2, l64], [l3], [l2, l2]):
        with pytest.raises(P.LbError) as e:
            P.Batch(bad)
        assert e.value.status in (P.LB_EUNSUPPORTED, P.LB_EINVAL)
    for l in (l2, l64, l3):
        l.close()


@pytest.fixture(scope="module")
def many():
    """The many-instance workload: 64 seeded instances, FP32-shifted."""
    inst = L.batched_instances(64)
    lats, rhos = [], []
    for d in inst:
        s = d["side"]
        rho = (L.tanh_sphere(s, s, 1, d["radius"], N_GAS, N_LIQ, 2.0) if d["bubble"]
               else L.tanh_sphere(s, s, 1, d["radius"], N_LIQ, N_GAS, 2.0))
        st = d["stencil"]
        lats.append(P.Lattice("D2Q9", (s, s), rho, st.bases, st.weights, precision="fp32",
                              G=G, convention=CONV))
        rhos.append(rho)
    b = P.Batch(lats)
    b.tune(steps_per_trial=6)
    m0 = [l.observables()["mass"] for l in lats]
    b.step(131)
    assert b.sync() == P.LB_OK
    f_pre = [l.state() for l in lats]
    b.step(1)
    assert b.sync() == P.LB_OK
    f_post = [l.state() for l in lats]
    m1 = [l.observables()["mass"] for l in lats]
    out = dict(inst=inst, f_pre=f_pre, f_post=f_post, m0=m0, m1=m1,
               nodes=sum(d["side"] ** 2 for d in inst))
    _close(b, lats)
    return out


def test_64_instance_workload_sampled_nodes_match_oracle(many):
    assert many["nodes"] > 4_000_000
    rng = np.random.default_rng(0xC3)
    worst = 0.0
    for k in rng.choice(len(many["inst"]), size=12, replace=False):
        d = many["inst"][k]
        s = d["side"]
        o = oracle.Oracle("D2Q9", (1, s, s), d["stencil"].groups, tau=1.0, G=G, convention=CONV)
        o.f = many["f_pre"][k].reshape(9, -1).copy()
        pts = [(0, 0), (s - 1, s - 1), (s // 2, s // 2)]
        pts += [tuple(int(v) for v in rng.integers(0, s, 2)) for _ in range(6)]
        r = d["radius"]
        for a in rng.uniform(0, 2 * np.pi, 6):   # interface ring
            pts.append((int(round(s / 2 - 0.5 + r * np.cos(a))) % s,
                        int(round(s / 2 - 0.5 + r * np.sin(a))) % s))
        for x, y in pts:
            post = o.node_post(x, y)
            for i, c in enumerate(oracle.C9):
                g = many["f_post"][k][i, 0, (y + c[1]) % s, (x + c[0]) % s]
                worst = max(worst, abs(g - post[i]) / max(abs(post[i]), 1e-3))
    assert worst < 1e-5, worst


def test_64_instance_workload_conserves_mass(many):
    for m0, m1 in zip(many["m0"], many["m1"]):
        assert abs(m1 - m0) < 1e-6 * m0
