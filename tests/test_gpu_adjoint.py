"""The GPU adjoint (lb_adjoint_*, binary64) against the oracle's adjoint
(oracle/adjoint.py, itself pinned to central finite differences of the
oracle's forward step) and against finite differences of the GPU's own
forward runs; checkpointing changes nothing; the torch.autograd.Function
returns the same gradient; losses on the density (liquid/gas density ratio,
interface width) differentiate the same way; the F^2 forcing variant too; and a
gradient solve of the paper's surface tension knob (Table tab:e4_tuning_6,
sigma0_hat) hits a target sigma_0."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import lbinputs as L
import oracle
from oracle import adjoint as OAD

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2505_23647_gb300")
AD = pytest.importorskip("paper_2505_23647_gb300.adjoint")

N_GAS, N_LIQ = 0.456, 2.25

CASES = [
    ("D2Q9", (24, 5), L.E8_2D, 1.0, -3.0, "literal", None, 12),
    ("D3Q19", (20, 4, 3), L.E4_3D, 0.8, -4.0, "literal", None, 8),
    ("D2Q9", (22, 4), L.E6_2D, 1.3, -9.0, "paper", None, 10),
    ("D2Q9", (26, 4), L.E8_2D, 1.0, -2.7, "literal", 10.0 / 31.0, 10),
]


def _rho(shape):
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    return L.tanh_slab(nx, ny, nz, nx // 4, 3 * nx // 4, N_GAS, N_LIQ, 2.0)


def _lat(lattice, shape, st, tau, G, conv, eps, precision="fp64", weights=None):
    return P.Lattice(lattice, shape, _rho(shape), st.bases,
                     st.weights if weights is None else weights, precision=precision, tau=tau,
                     G=G, convention=conv, psi_eps=eps)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("lattice,shape,st,tau,G,conv,eps,steps", CASES)
def test_gpu_adjoint_matches_oracle_adjoint(lattice, shape, st, tau, G, conv, eps, steps):
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    g0 = lat.state()
    sigma, dW, dG, lam0 = AD.sigma_and_gradient(lat, steps, checkpoint_every=steps)
    lat.close()
    nz = shape[2] if len(shape) > 2 else 1
    o = oracle.Oracle(lattice, (nz, shape[1], shape[0]), st.groups, tau=tau, G=G, convention=conv,
                      psi_kind=0 if eps is None else 1, psi_eps=0.0 if eps is None else eps)
    s_o, lam_o, dW_o, dGp_o = OAD.gradient(o, g0.reshape((o.Q, nz, shape[1], shape[0])), steps, 2)
    dG_o = dGp_o / 3.0 if conv == "paper" else dGp_o
    assert abs(sigma - s_o) < 1e-12 * abs(s_o)
    assert _rel(dW, dW_o) < 1e-10, (dW, dW_o)
    assert abs(dG - dG_o) < 1e-10 * abs(dG_o)
    assert _rel(lam0.reshape(lam_o.shape), lam_o) < 1e-10


@pytest.mark.parametrize("lattice,shape,st,tau,G,steps,A,precision", [
    ("D2Q9", (24, 5), L.E8_2D, 1.0, -3.0, 12, 0.25, "fp64"),
    ("D3Q19", (20, 4, 3), L.E4_3D, 0.8, -4.0, 8, 0.6, "fp64"),
    ("D2Q9", (24, 5), L.E8_2D, 1.0, -3.0, 12, 0.25, "fp32"),
])
def test_f2_forcing_adjoint_matches_oracle_adjoint(lattice, shape, st, tau, G, steps, A, precision):
    """The F^2 variant (Sec. VI): the GPU adjoint against the oracle's (its
    F^2 terms pinned to finite differences of the C oracle on the CPU)."""
    lat = P.Lattice(lattice, shape, _rho(shape), st.bases, st.weights, precision=precision,
                    tau=tau, G=G, forcing_A=A)
    g0 = lat.state()
    sigma, dW, dG, lam0 = AD.sigma_and_gradient(lat, steps, checkpoint_every=4)
    lat.close()
    nz = shape[2] if len(shape) > 2 else 1
    o = oracle.Oracle(lattice, (nz, shape[1], shape[0]), st.groups, tau=tau, G=G, forcing_A=A)
    s_o, lam_o, dW_o, dGp_o = OAD.gradient(o, g0.reshape((o.Q, nz, shape[1], shape[0])), steps, 2)
    if precision == "fp64":
        assert abs(sigma - s_o) < 1e-12 * abs(s_o)
        assert _rel(dW, dW_o) < 1e-10, (dW, dW_o)
        assert abs(dG - dGp_o) < 1e-10 * abs(dGp_o)
        assert _rel(lam0.reshape(lam_o.shape), lam_o) < 1e-10
    else:   # binary32 forward states: the gradient to binary32 accuracy
        assert abs(sigma - s_o) < 1e-5 * abs(s_o)
        assert _rel(dW, dW_o) < 1e-3, (dW, dW_o)


def test_graph_replay_changes_nothing():
    """Segments after the first replay a captured graph of the run; with
    per-kernel timing on, every segment runs directly: the same bits."""
    lattice, shape, st, tau, G, conv, eps, _ = CASES[0]
    out = []
    for timing in (False, True):
        lat = _lat(lattice, shape, st, tau, G, conv, eps, precision="fp32")
        if timing:
            P.lb_timing(lat.ctx, 1)
        out.append(AD.sigma_and_gradient(lat, 24, checkpoint_every=6))
        f = lat.state()
        out[-1] = out[-1] + (f,)
        lat.close()
    (s0, w0, g0, l0, f0), (s1, w1, g1, l1, f1) = out
    assert s0 == s1 and g0 == g1
    assert np.array_equal(w0, w1) and np.array_equal(l0, l1) and np.array_equal(f0, f1)


def test_checkpointing_changes_nothing():
    lattice, shape, st, tau, G, conv, eps, _ = CASES[0]
    res = []
    for K in (60, 7, 1):
        lat = _lat(lattice, shape, st, tau, G, conv, eps)
        res.append(AD.sigma_and_gradient(lat, 60, checkpoint_every=K))
        lat.close()
    for r in res[1:]:
        assert r[0] == res[0][0]
        assert np.array_equal(r[1], res[0][1]) and r[2] == res[0][2]
        assert np.array_equal(r[3], res[0][3])


def test_gradient_matches_finite_differences_of_gpu_runs():
    lattice, shape, st, tau, G, conv, eps, _ = CASES[0]
    steps = 200
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    _, dW, dG, _ = AD.sigma_and_gradient(lat, steps, checkpoint_every=50)
    lat.close()

    def sigma_of(weights, Gv):
        l = _lat(lattice, shape, st, tau, Gv, conv, eps, weights=weights)
        l.step(steps)
        a = AD.Adjoint(l)
        s = a.seed_sigma(2)
        a.close()
        l.close()
        return s

    w0 = st.weights.copy()
    for q in range(len(w0)):
        h = 1e-6 * w0[q]
        wp, wm = w0.copy(), w0.copy()
        wp[q] += h
        wm[q] -= h
        fd = (sigma_of(wp, G) - sigma_of(wm, G)) / (2 * h)
        assert abs(dW[q] - fd) < 1e-6 * abs(fd) + 1e-9, (q, dW[q], fd)
    h = 1e-6 * abs(G)
    fd = (sigma_of(w0, G + h) - sigma_of(w0, G - h)) / (2 * h)
    assert abs(dG - fd) < 1e-6 * abs(fd)


def test_fp32_forward_gradient_close_to_fp64():
    lattice, shape, st, tau, G, conv, eps, _ = CASES[0]
    out = {}
    for prec in ("fp64", "fp32"):
        lat = _lat(lattice, (64, 4), st, tau, G, conv, eps, precision=prec)
        out[prec] = AD.sigma_and_gradient(lat, 500, checkpoint_every=100)
        lat.close()
    s64, w64, g64, _ = out["fp64"]
    s32, w32, g32, _ = out["fp32"]
    assert abs(s32 - s64) < 1e-4 * abs(s64)
    assert _rel(w32, w64) < 1e-3 and abs(g32 - g64) < 1e-3 * abs(g64)


def test_torch_autograd_function():
    """flat_slab: the four quantities in forward, one adjoint sweep for any
    combination of them in backward; equal to the per-quantity gradients of
    flat_quantity_and_gradient (and sigma_0 to the lattice-summed sigma of
    lb_adjoint_seed_sigma divided by the rows)."""
    torch = pytest.importorskip("torch")
    lattice, shape, st, tau, G, conv, eps, steps = CASES[0]
    nx, ny = shape
    spec = dict(lattice=lattice, shape=shape, rho=_rho(shape), bases=st.bases, steps=steps,
                tau=tau, convention=conv, checkpoint_every=5, n_liquid=N_LIQ, n_gas=N_GAS,
                x_liquid=nx // 2, x_gas=1)
    W = torch.tensor(st.weights, dtype=torch.float64, requires_grad=True)
    Gt = torch.tensor(G, dtype=torch.float64, requires_grad=True)
    q = AD.flat_slab(W, Gt, spec)
    wts = np.array([2.0, 3.0, -1.0, 0.5])
    (q * torch.tensor(wts)).sum().backward()
    specs = [(AD.LB_FLAT_SIGMA, None), (AD.LB_FLAT_DELTA, None),
             AD.interface_width(N_LIQ, N_GAS), AD.density_ratio(nx // 2, 1)]
    dW_sum, dG_sum = 0.0, 0.0
    for k, (qq, pp) in enumerate(specs):
        lat = _lat(lattice, shape, st, tau, G, conv, eps)
        v, dW, dG, _ = AD.flat_quantity_and_gradient(lat, steps, qq, pp, checkpoint_every=5)
        lat.close()
        assert abs(float(q[k].detach()) - v) <= 1e-13 * abs(v)
        dW_sum = dW_sum + wts[k] * dW
        dG_sum = dG_sum + wts[k] * dG
    assert _rel(W.grad.numpy(), dW_sum) < 1e-12
    assert abs(float(Gt.grad) - dG_sum) < 1e-12 * abs(dG_sum)
    # sigma_0 of the device seed against the pinned lattice-summed sigma
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    sig_sum, dW_s, dG_s, _ = AD.sigma_and_gradient(lat, steps, checkpoint_every=steps)
    lat.close()
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    sig, dW_q, dG_q, _ = AD.flat_quantity_and_gradient(lat, steps, AD.LB_FLAT_SIGMA)
    lat.close()
    assert abs(sig * ny - sig_sum) < 1e-12 * abs(sig_sum)
    assert _rel(dW_q * ny, dW_s) < 1e-10 and abs(dG_q * ny - dG_s) < 1e-10 * abs(dG_s)


def test_gradient_solve_hits_target_sigma():
    """Replace the hand tuning of Sec. V with a gradient solve: Newton on the
    knob sigma0_hat of Table tab:e4_tuning_6 (weights linear in the knob)
    until sigma_0 of a relaxed slab is 1.15 x its untuned value."""
    nx, ny, steps, G = 64, 4, 1500, -3.0
    rho = L.tanh_slab(nx, ny, 1, 16, 48, N_GAS, N_LIQ, 2.0)
    # d W / d knob of the table (groups (1,0), (1,1), (2,0), (2,2))
    slope = np.array([4 / 3, -1 / 6, -5 / 24, -1 / 48])

    def run(s0):
        st = L.stencil_e4_tuning_6(2, Fr(s0).limit_denominator(10 ** 12))
        lat = P.Lattice("D2Q9", (nx, ny), rho, st.bases, st.weights, G=G)
        sigma, dW, _, _ = AD.sigma_and_gradient(lat, steps, checkpoint_every=250)
        lat.close()
        return sigma, float(np.dot(dW, slope))

    s0 = 0.0
    sigma0, _ = run(s0)
    target = 1.15 * sigma0
    for _ in range(8):
        sigma, dsig = run(s0)
        if abs(sigma / target - 1.0) < 1e-3:
            break
        s0 -= (sigma - target) / dsig
    assert abs(sigma / target - 1.0) < 1e-3, (s0, sigma, target)


def _oracle_width(nl, ng):
    """6 sum (n - ng)(nl - n) / (nl - ng)^2 / 2 of the column-averaged profile."""
    def fn(n):
        cols = n.shape[0] * n.shape[1]
        prof = n.mean(axis=(0, 1))
        d2 = (nl - ng) ** 2
        val = 3.0 * float(np.sum((prof - ng) * (nl - prof))) / d2
        return val, np.broadcast_to(3.0 * (nl + ng - 2 * prof) / d2 / cols, n.shape).copy()
    return fn


def _oracle_ratio(xl, xg):
    """n_l / n_g of the column averages at xl (liquid) and xg (gas)."""
    def fn(n):
        cols = n.shape[0] * n.shape[1]
        nl, ng = n[..., xl].mean(), n[..., xg].mean()
        d = np.zeros_like(n)
        d[..., xl] = 1.0 / (ng * cols)
        d[..., xg] = -nl / (ng * ng * cols)
        return nl / ng, d
    return fn


@pytest.mark.parametrize("which", ["ratio", "width"])
def test_density_functionals_match_oracle_adjoint(which):
    lattice, shape, st, tau, G, conv, eps, steps = CASES[0]
    nx, ny = shape
    if which == "ratio":
        spec, fn_or = AD.density_ratio(nx // 2, 1), _oracle_ratio(nx // 2, 1)
    else:
        spec, fn_or = AD.interface_width(N_LIQ, N_GAS), _oracle_width(N_LIQ, N_GAS)
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    g0 = lat.state()
    val, dW, dG, lam0 = AD.flat_quantity_and_gradient(lat, steps, *spec, checkpoint_every=5)
    lat.close()
    o = oracle.Oracle(lattice, (1, ny, nx), st.groups, tau=tau, G=G, convention=conv)
    v_o, lam_o, dW_o, dGp_o = OAD.gradient_of_density_functional(o, g0.reshape((9, 1, ny, nx)), steps,
                                                                   fn_or)
    assert abs(val - v_o) < 1e-12 * abs(v_o)
    assert _rel(dW, dW_o) < 1e-10 and abs(dG - dGp_o) < 1e-10 * abs(dGp_o)
    assert _rel(lam0.reshape(lam_o.shape), lam_o) < 1e-10


def test_interface_width_gradient_matches_gpu_finite_differences():
    lattice, shape, st, tau, G, conv, eps, _ = CASES[0]
    steps = 150
    fn = _oracle_width(N_LIQ, N_GAS)
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    w, dW, dG, _ = AD.flat_quantity_and_gradient(lat, steps, *AD.interface_width(N_LIQ, N_GAS),
                                                 checkpoint_every=40)
    lat.close()
    assert 1.0 < w < 10.0

    def width_of(Gv):
        l = _lat(lattice, shape, st, tau, Gv, conv, eps)
        l.step(steps)
        n, _ = l.fields()
        l.close()
        return fn(n)[0]

    h = 1e-6 * abs(G)
    fd = (width_of(G + h) - width_of(G - h)) / (2 * h)
    assert abs(dG - fd) < 1e-6 * abs(fd) + 1e-9, (dG, fd)


def _oracle_delta(lattice, shape, groups, tau, G, conv, g0, steps):
    """Mean Tolman length of the oracle run, by the oracle's own analysis."""
    from oracle import analysis as OA
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) > 2 else 1
    o = oracle.Oracle(lattice, (nz, ny, nx), groups, tau=tau, G=G, convention=conv)
    o.f = g0.reshape((o.Q, nz, ny, nx)).copy()
    o.step(steps)
    obs = OA.flat_observables(o.pressure_tensor(), o.fields()["n"], D=o.D)
    return float(np.mean([r["delta"] for r in obs]))


@pytest.mark.parametrize("case", [0, 1])
def test_tolman_gradient_matches_oracle_finite_differences(case):
    """delta = z_e - z_s (eqs. zemzs, SCTolmanFlat) through the adjoint: its
    value equals the oracle's analysis of the oracle run, its gradient central
    differences of that (weights per group, G, initial populations)."""
    lattice, shape, st, tau, G, conv, eps, steps = CASES[case]
    lat = _lat(lattice, shape, st, tau, G, conv, eps)
    g0 = lat.state()
    delta, dW, dG, lam0 = AD.tolman_and_gradient(lat, steps, checkpoint_every=5)
    lat.close()
    ref = _oracle_delta(lattice, shape, st.groups, tau, G, conv, g0, steps)
    assert abs(delta - ref) < 1e-10 * abs(ref), (delta, ref)
    for q, (b, wq) in enumerate(st.groups):
        h = 1e-6 * float(wq)
        gp = [(bb, float(ww) + (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        gm = [(bb, float(ww) - (h if k == q else 0.0)) for k, (bb, ww) in enumerate(st.groups)]
        fd = (_oracle_delta(lattice, shape, gp, tau, G, conv, g0, steps) -
              _oracle_delta(lattice, shape, gm, tau, G, conv, g0, steps)) / (2 * h)
        assert abs(dW[q] - fd) < 1e-5 * abs(fd) + 1e-7, (q, dW[q], fd)
    h = 1e-6 * abs(G)
    fd = (_oracle_delta(lattice, shape, st.groups, tau, G + h, conv, g0, steps) -
          _oracle_delta(lattice, shape, st.groups, tau, G - h, conv, g0, steps)) / (2 * h)
    assert abs(dG - fd) < 1e-5 * abs(fd) + 1e-7, (dG, fd)
    rng = np.random.default_rng(2)
    lam = lam0.reshape(g0.shape)
    for _ in range(3):
        idx = tuple(int(rng.integers(0, s)) for s in g0.shape)
        h = 1e-4 * abs(g0[idx])
        gp, gm = g0.copy(), g0.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (_oracle_delta(lattice, shape, st.groups, tau, G, conv, gp, steps) -
              _oracle_delta(lattice, shape, st.groups, tau, G, conv, gm, steps)) / (2 * h)
        assert abs(lam[idx] - fd) < 1e-5 * abs(fd) + 1e-8, (idx, lam[idx], fd)


def test_gradient_solve_of_sigma_and_tolman_at_fixed_profile():
    """The tuning the paper does by hand (Sec. V) as a gradient solve: the
    knobs sigma0_hat, sigma1_hat, delta0_hat of Table tab:e4e6e8_tuning_6 and
    G move a relaxed slab to 1.1 x its sigma_0 and 0.5 x its Tolman length
    while its interface width and density ratio stay where they were, all
    four to 1e-3 relative."""
    nx, ny, steps, K = 64, 4, 1500, 250
    rho = L.tanh_slab(nx, ny, 1, 16, 48, N_GAS, N_LIQ, 2.0)
    st0 = L.stencil_e4e6e8_tuning_6(2, 0, 0, 0)

    def weights_of(k):
        s0, s1, d0 = (Fr(float(v)).limit_denominator(10 ** 15) for v in k)
        return L.stencil_e4e6e8_tuning_6(2, s0, s1, d0).weights

    def make(W, G):
        return P.Lattice("D2Q9", (nx, ny), rho, st0.bases, W, G=G)

    knobs0, G0 = np.array([-0.1, 0.0, 0.05]), -3.0
    v0, _, _ = AD.slab_observables(lambda: make(weights_of(knobs0), G0), steps, nx // 2, 0,
                                   N_LIQ, N_GAS, K)
    assert v0[0] > 0 and v0[3] > 1.0
    targets = v0 * np.array([1.1, 0.5, 1.0, 1.0])
    knobs, G, vals, hist = AD.tune_slab(make, weights_of, knobs0, G0, targets, steps, nx // 2, 0,
                                        N_LIQ, N_GAS, K, rtol=1e-3, max_iter=10)
    assert np.max(np.abs(vals / targets - 1.0)) < 1e-3, (knobs, G, vals, targets, hist)
