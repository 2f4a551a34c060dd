"""Gradients of the flat-interface surface tension through the step
(``lb_adjoint_*``), with checkpointed recomputation, and a
``torch.autograd.Function`` on top.

Every step, forward and backward, runs in the library's kernels; this module
only moves checkpoints (``lb_get_state`` / ``lb_set_state``) and arguments.
"""
import ctypes

import numpy as np

from . import LbError, Lattice, _check, _lib, _ptr, _vp


class Adjoint:
    """The adjoint of one :class:`Lattice` (see ``lb_adjoint_*`` in sclbm.h)."""

    def __init__(self, lattice):
        self.lat = lattice
        out = _vp()
        _check(_lib.lb_adjoint_create(_vp(lattice.ctx), ctypes.byref(out)), "lb_adjoint_create")
        self.a = out.value

    def set(self, lam=None):
        if lam is None:
            _check(_lib.lb_adjoint_set(_vp(self.a), None), "lb_adjoint_set")
        else:
            lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
            if lam.size != self.lat.Q * self.lat.N:
                raise ValueError("lam must have Q x N entries")
            _check(_lib.lb_adjoint_set(_vp(self.a), _ptr(lam)), "lb_adjoint_set")

    def get(self):
        lam = np.empty(self.lat.Q * self.lat.N)
        _check(_lib.lb_adjoint_get(_vp(self.a), _ptr(lam)), "lb_adjoint_get")
        return lam.reshape((self.lat.Q,) + self.lat.shape)

    def zero_grad(self):
        _check(_lib.lb_adjoint_zero_grad(_vp(self.a)), "lb_adjoint_zero_grad")

    def seed_sigma(self, n_interfaces=2):
        s = ctypes.c_double(0.0)
        _check(_lib.lb_adjoint_seed_sigma(_vp(self.a), int(n_interfaces), ctypes.byref(s)),
               "lb_adjoint_seed_sigma")
        return s.value

    def seed_pt(self, m):
        """Add the gradient of sum_x m(x) (P_xx - P_yy)(x) to lam; returns the sum."""
        m = np.ascontiguousarray(m, dtype=np.float64).reshape(-1)
        if m.size != self.lat.N:
            raise ValueError("m must have N entries")
        v = ctypes.c_double(0.0)
        _check(_lib.lb_adjoint_seed_pt(_vp(self.a), _ptr(m), ctypes.byref(v)), "lb_adjoint_seed_pt")
        return v.value

    def run(self, nsteps):
        _check(_lib.lb_adjoint_run(_vp(self.a), int(nsteps)), "lb_adjoint_run")

    def gradient(self):
        """(dL/dW per stencil group, dL/dG)."""
        dW = np.zeros(len(self.lat.stencil_weights))
        dG = ctypes.c_double(0.0)
        _check(_lib.lb_adjoint_gradient(_vp(self.a), _ptr(dW), ctypes.byref(dG)),
               "lb_adjoint_gradient")
        return dW, dG.value

    def close(self):
        if self.a:
            _lib.lb_adjoint_destroy(_vp(self.a))
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sigma_and_gradient(lattice, steps, checkpoint_every=100, n_interfaces=2):
    """sigma_0 after ``steps`` steps of ``lattice`` (a flat slab along x) and its
    gradient with respect to the stencil group weights, G and the initial
    state.  The forward run keeps a checkpoint every ``checkpoint_every``
    steps; the backward pass recomputes one segment at a time.  The lattice
    ends ``steps`` steps after its initial state.  Returns
    (sigma, dW [groups], dG, dsigma/d(initial state))."""
    K = max(1, int(checkpoint_every))
    ckpts = []
    done = 0
    while done < steps:
        ckpts.append((done, lattice.state()))
        k = min(K, steps - done)
        lattice.step(k)
        done += k
    adj = Adjoint(lattice)
    try:
        sigma = adj.seed_sigma(n_interfaces)
        for start, st in reversed(ckpts):
            lattice.set_state(st)
            adj.run(min(K, steps - start))
        dW, dG = adj.gradient()
        lam0 = adj.get()
    finally:
        adj.close()
    return sigma, dW, dG, lam0


def density_functional_and_gradient(lattice, steps, fn, checkpoint_every=100):
    """A loss L(n) of the density after ``steps`` steps and its gradient with
    respect to the stencil group weights, G and the initial state.  ``fn(n)``
    receives the final density (shape of ``lattice.shape``) and returns
    (L, dL/dn); since n = sum_i f_i, dL/df_i = dL/dn seeds the adjoint.
    Returns (L, dW [groups], dG, dL/d(initial state))."""
    K = max(1, int(checkpoint_every))
    ckpts = []
    done = 0
    while done < steps:
        ckpts.append((done, lattice.state()))
        k = min(K, steps - done)
        lattice.step(k)
        done += k
    n, _ = lattice.fields()
    value, dn = fn(n)
    adj = Adjoint(lattice)
    try:
        adj.set(np.broadcast_to(np.asarray(dn, dtype=np.float64), (lattice.Q,) + lattice.shape))
        for start, st in reversed(ckpts):
            lattice.set_state(st)
            adj.run(min(K, steps - start))
        dW, dG = adj.gradient()
        lam0 = adj.get()
    finally:
        adj.close()
    return value, dW, dG, lam0


def density_ratio(x_liquid, x_gas):
    """L(n) = n_l / n_g of a flat slab (gradients along x): the densities are
    the y (and z) averages of columns x_liquid and x_gas."""
    def fn(n):
        cols = n.shape[0] * n.shape[1]
        nl, ng = n[..., x_liquid].mean(), n[..., x_gas].mean()
        d = np.zeros_like(n)
        d[..., x_liquid] = 1.0 / (ng * cols)
        d[..., x_gas] = -nl / (ng * ng * cols)
        return nl / ng, d
    return fn


def interface_width(n_liquid, n_gas, n_interfaces=2):
    """Smooth width of the interfaces of a flat slab (gradients along x):
    L(n) = 6 sum_x (n(x) - n_g)(n_l - n(x)) / (n_l - n_g)^2 / #interfaces with
    n(x) the y (and z) average; for a tanh profile of width w it equals w."""
    def fn(n):
        cols = n.shape[0] * n.shape[1]
        prof = n.mean(axis=(0, 1))
        dl = n_liquid - n_gas
        val = 6.0 * float(np.sum((prof - n_gas) * (n_liquid - prof))) / (dl * dl) / n_interfaces
        dprof = 6.0 * (n_liquid + n_gas - 2.0 * prof) / (dl * dl) / n_interfaces
        return val, np.broadcast_to(dprof / cols, n.shape).copy()
    return fn


def _windows(prof):
    """Interface windows of a periodic profile: for each crossing of the mid
    density between x and x+1, the columns from half way to the previous
    crossing to half way to the next one; +1 for gas -> liquid along +x."""
    L = len(prof)
    mid = 0.5 * (prof.max() + prof.min())
    sg = np.sign(prof - mid)
    cross = [(i, 1 if sg[(i + 1) % L] > sg[i] else -1) for i in range(L)
             if sg[i] != sg[(i + 1) % L] and sg[i] != 0 and sg[(i + 1) % L] != 0]
    out = []
    k = len(cross)
    for q, (i, d) in enumerate(cross):
        gp = (i - cross[q - 1][0]) % L if k > 1 else L
        gn = (cross[(q + 1) % k][0] - i) % L if k > 1 else L
        out.append((i - gp // 2 + 1, i + gn // 2, d))
    return out


def tolman_and_gradient(lattice, steps, checkpoint_every=100):
    """Tolman length delta = z_e - z_s of a flat slab (gradients along x) after
    ``steps`` steps, averaged over its interfaces, and its gradient with
    respect to the stencil group weights, G and the initial state.

    Per interface window (columns a..b, site x the cell [x - 1/2, x + 1/2]):
    z_s = sum x (P_N - P_T) / sum (P_N - P_T) from the lattice pressure tensor
    (Appendices E/F), z_e the equimolar position from the window-end
    densities, delta oriented from liquid to gas (eqs. zemzs, SCTolmanFlat).
    The loss is a function of the column-averaged density and of
    P_N - P_T: its density part seeds lam, its tensor part enters through
    lb_adjoint_seed_pt.  Returns (delta, dW, dG, d delta/d(initial state))."""
    K = max(1, int(checkpoint_every))
    ckpts = []
    done = 0
    while done < steps:
        ckpts.append((done, lattice.state()))
        k = min(K, steps - done)
        lattice.step(k)
        done += k
    n, _ = lattice.fields()
    P = lattice.pressure_tensor()
    D = P[0] - (P[2] if lattice.D == 2 else P[3])
    cols = n.shape[0] * n.shape[1]
    prof, dprof = n.mean(axis=(0, 1)), D.mean(axis=(0, 1))
    L = len(prof)
    wins = _windows(prof)
    if not wins:
        raise ValueError("no interface in the final state")
    g_n = np.zeros(L)     # d delta / d profile
    g_d = np.zeros(L)     # d delta / d (P_N - P_T) profile
    delta = 0.0
    for a, b, d in wins:
        xs = np.arange(a, b + 1)
        idx = xs % L
        J = len(idx)
        S = float(np.sum(dprof[idx]))
        zs = float(np.sum(xs * dprof[idx])) / S
        nv = prof[idx]
        if d > 0:      # gas at a, liquid at b
            T = float(np.sum(nv)) - J * nv[0]
            Dl = nv[-1] - nv[0]
            ze = (b + 0.5) - T / Dl
            dT = np.ones(J)
            dT[0] -= J
            dD = np.zeros(J)
            dD[-1], dD[0] = 1.0, -1.0
            dze = -(dT * Dl - T * dD) / (Dl * Dl)
        else:          # liquid at a, gas at b
            T = float(np.sum(nv)) - J * nv[-1]
            Dl = nv[0] - nv[-1]
            ze = (a - 0.5) + T / Dl
            dT = np.ones(J)
            dT[-1] -= J
            dD = np.zeros(J)
            dD[0], dD[-1] = 1.0, -1.0
            dze = (dT * Dl - T * dD) / (Dl * Dl)
        orient = -d
        delta += orient * (ze - zs)
        np.add.at(g_n, idx, orient * dze)
        np.add.at(g_d, idx, -orient * (xs - zs) / S)
    nw = len(wins)
    delta /= nw
    g_n /= nw * cols
    g_d /= nw * cols
    adj = Adjoint(lattice)
    try:
        adj.set(np.broadcast_to(g_n, (lattice.Q,) + lattice.shape))
        adj.seed_pt(np.broadcast_to(g_d, lattice.shape))
        for start, st in reversed(ckpts):
            lattice.set_state(st)
            adj.run(min(K, steps - start))
        dW, dG = adj.gradient()
        lam0 = adj.get()
    finally:
        adj.close()
    return delta, dW, dG, lam0


def slab_observables(make_lattice, steps, x_liquid, x_gas, n_liquid, n_gas, checkpoint_every=100):
    """The four quantities the stencil tuning of Sec. V targets, for a flat
    slab (gradients along x), with their gradients: values (sigma_0, delta,
    interface width, density ratio n_l/n_g), dW [4, groups] and dG [4].
    ``make_lattice()`` returns a fresh lattice in the initial state (each
    quantity runs its own forward and adjoint pass)."""
    vals, dWs, dGs = [], [], []
    runs = [lambda lat: sigma_and_gradient(lat, steps, checkpoint_every),
            lambda lat: tolman_and_gradient(lat, steps, checkpoint_every),
            lambda lat: density_functional_and_gradient(lat, steps, interface_width(n_liquid, n_gas),
                                                        checkpoint_every),
            lambda lat: density_functional_and_gradient(lat, steps, density_ratio(x_liquid, x_gas),
                                                        checkpoint_every)]
    for run in runs:
        lat = make_lattice()
        try:
            v, dW, dG, _ = run(lat)
        finally:
            lat.close()
        vals.append(v)
        dWs.append(dW)
        dGs.append(dG)
    return np.array(vals), np.array(dWs), np.array(dGs)


def tune_slab(make_lattice, weights_of, knobs, G, targets, steps, x_liquid, x_gas, n_liquid, n_gas,
              checkpoint_every=100, rtol=1e-3, max_iter=10):
    """Gradient solve replacing the hand tuning of Sec. V: Newton steps on the
    stencil knobs and G until (sigma_0, delta, width, n_l/n_g) of a relaxed
    flat slab match ``targets`` to ``rtol`` (relative).

    ``weights_of(knobs)`` gives the group weights, linear in the knobs (the
    paper's tables are); ``make_lattice(weights, G)`` a fresh lattice in the
    initial state.  With as many knobs plus G as targets the Newton system is
    square; otherwise it is solved in the least-squares sense.  Returns
    (knobs, G, values, history of the relative errors)."""
    knobs = np.array(knobs, dtype=np.float64)
    targets = np.asarray(targets, dtype=np.float64)
    base = np.asarray(weights_of(np.zeros_like(knobs)), dtype=np.float64)
    slope = np.stack([np.asarray(weights_of(np.eye(len(knobs))[k]), dtype=np.float64) - base
                      for k in range(len(knobs))], axis=1)          # dW/dknob
    hist = []
    vals = None
    for _ in range(max_iter):
        W = np.asarray(weights_of(knobs), dtype=np.float64)
        vals, dW, dG = slab_observables(lambda: make_lattice(W, G), steps, x_liquid, x_gas,
                                        n_liquid, n_gas, checkpoint_every)
        rel = (vals - targets) / targets
        hist.append(rel)
        if np.max(np.abs(rel)) < rtol:
            break
        J = np.concatenate([dW @ slope, dG[:, None]], axis=1) / targets[:, None]
        dx = np.linalg.lstsq(J, -rel, rcond=None)[0]
        knobs = knobs + dx[:-1]
        G = G + dx[-1]
    return knobs, G, vals, hist


_FN = None


def _torch_function():
    global _FN
    if _FN is not None:
        return _FN
    import torch

    class FlatSigma(torch.autograd.Function):
        """sigma_0(W, G) of a flat slab after a fixed number of steps from a
        fixed initial density; backward by the adjoint (computed with the
        forward, checkpointed)."""

        @staticmethod
        def forward(ctx, W, G, spec):
            lat = Lattice(spec["lattice"], spec["shape"], spec["rho"], spec["bases"],
                          W.detach().cpu().numpy().astype(np.float64), precision=spec.get("precision", "fp64"),
                          tau=spec.get("tau", 1.0), G=float(G), convention=spec.get("convention", "literal"),
                          psi_eps=spec.get("psi_eps"))
            try:
                sigma, dW, dG, _ = sigma_and_gradient(lat, spec["steps"], spec.get("checkpoint_every", 100),
                                                      spec.get("n_interfaces", 2))
            finally:
                lat.close()
            ctx.save_for_backward(torch.as_tensor(dW, dtype=W.dtype), torch.as_tensor(dG, dtype=W.dtype))
            return W.new_tensor(sigma)

        @staticmethod
        def backward(ctx, g):
            dW, dG = ctx.saved_tensors
            return g * dW, g * dG, None

    _FN = FlatSigma
    return FlatSigma


def flat_sigma(W, G, spec):
    """Differentiable sigma_0 (torch): W a tensor of group weights (the order
    of spec['bases']), G a scalar tensor; spec holds lattice, shape, rho,
    bases, steps and optionally precision, tau, convention, psi_eps,
    checkpoint_every, n_interfaces."""
    return _torch_function().apply(W, G, spec)


__all__ = ["Adjoint", "sigma_and_gradient", "density_functional_and_gradient", "density_ratio",
           "interface_width", "tolman_and_gradient", "slab_observables", "tune_slab", "flat_sigma",
           "LbError"]
