"""Gradients of flat-interface quantities through the step (``lb_adjoint_*``),
with checkpointed recomputation, and a ``torch.autograd.Function`` on top.

Every step, forward and backward, runs in the library's kernels, and so does
the post-processing of the quantities (profiles, interface windows, sigma_0,
the Tolman length, the interface width, the density ratio and their seeds:
``lb_adjoint_seed_flat``, binary64 on the device); this module only moves
checkpoints (``lb_get_state`` / ``lb_set_state``) and arguments.
"""
import ctypes

import numpy as np

from . import LbError, Lattice, _check, _lib, _ptr, _vp

# quantities of lb_adjoint_seed_flat
LB_FLAT_SIGMA, LB_FLAT_DELTA, LB_FLAT_WIDTH, LB_FLAT_RATIO = range(4)


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

    def seed_flat(self, quantity, params=None, weight=1.0):
        """Add weight x the gradient of a flat-slab quantity (LB_FLAT_*) of the
        current state to lam; returns the quantity (computed on the device)."""
        v = ctypes.c_double(0.0)
        if params is None:
            pp = None
        else:
            arr = np.ascontiguousarray(np.asarray(params, dtype=np.float64).ravel())
            pp = _ptr(arr)
        _check(_lib.lb_adjoint_seed_flat(_vp(self.a), int(quantity), pp, float(weight),
                                         ctypes.byref(v)), "lb_adjoint_seed_flat")
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


def forward_with_checkpoints(lattice, steps, checkpoint_every=100):
    """Step ``lattice`` ``steps`` steps, keeping its state every
    ``checkpoint_every`` steps: [(step, state), ...]."""
    K = max(1, int(checkpoint_every))
    ckpts = []
    done = 0
    while done < steps:
        ckpts.append((done, lattice.state()))
        k = min(K, steps - done)
        lattice.step(k)
        done += k
    return ckpts


def backward_through(lattice, adj, ckpts, steps, checkpoint_every=100):
    """Carry the adjoint back to the initial state, one checkpointed segment
    at a time (each recomputed from its checkpoint by the library's step);
    returns (dW, dG, dL/d(initial state))."""
    K = max(1, int(checkpoint_every))
    for start, st in reversed(ckpts):
        lattice.set_state(st)
        adj.run(min(K, steps - start))
    dW, dG = adj.gradient()
    return dW, dG, adj.get()


def flat_quantity_and_gradient(lattice, steps, quantity, params=None, checkpoint_every=100):
    """A flat-slab quantity (LB_FLAT_SIGMA, _DELTA, _WIDTH with params
    (n_l, n_g, #interfaces), _RATIO with params (x_liquid, x_gas)) after
    ``steps`` steps of ``lattice`` and its gradient with respect to the
    stencil group weights, G and the initial state; the quantity and its
    seed are formed by the library (lb_adjoint_seed_flat).  Returns
    (value, dW [groups], dG, dvalue/d(initial state))."""
    ckpts = forward_with_checkpoints(lattice, steps, checkpoint_every)
    adj = Adjoint(lattice)
    try:
        value = adj.seed_flat(quantity, params)
        dW, dG, lam0 = backward_through(lattice, adj, ckpts, steps, checkpoint_every)
    finally:
        adj.close()
    return value, dW, dG, lam0


def density_ratio(x_liquid, x_gas):
    """Quantity spec of n_l / n_g of a flat slab (gradients along x): the y
    (and z) averages of columns x_liquid and x_gas."""
    return LB_FLAT_RATIO, (x_liquid, x_gas)


def interface_width(n_liquid, n_gas, n_interfaces=2):
    """Quantity spec of the smooth interface width of a flat slab:
    6 sum_x (n(x) - n_g)(n_l - n(x)) / (n_l - n_g)^2 / #interfaces with n(x)
    the y (and z) average; for a tanh profile of width w it equals w."""
    return LB_FLAT_WIDTH, (n_liquid, n_gas, n_interfaces)


def tolman_and_gradient(lattice, steps, checkpoint_every=100):
    """Tolman length delta = z_e - z_s of a flat slab (gradients along x)
    after ``steps`` steps, averaged over its interfaces, and its gradient
    with respect to the stencil group weights, G and the initial state
    (eqs. zemzs, SCTolmanFlat; z_s from the lattice pressure tensor of
    Appendices E/F, z_e from the window-end densities).  Returns
    (delta, dW, dG, d delta/d(initial state))."""
    return flat_quantity_and_gradient(lattice, steps, LB_FLAT_DELTA, None, checkpoint_every)


def slab_observables(make_lattice, steps, x_liquid, x_gas, n_liquid, n_gas, checkpoint_every=100):
    """The four quantities the stencil tuning of Sec. V targets, for a flat
    slab (gradients along x), with their gradients: values (sigma_0, delta,
    interface width, density ratio n_l/n_g), dW [4, groups] and dG [4].
    ``make_lattice()`` returns a fresh lattice in the initial state; one
    forward run with checkpoints serves the four adjoint sweeps."""
    specs = [(LB_FLAT_SIGMA, None), (LB_FLAT_DELTA, None),
             interface_width(n_liquid, n_gas), density_ratio(x_liquid, x_gas)]
    lat = make_lattice()
    vals, dWs, dGs = [], [], []
    try:
        ckpts = forward_with_checkpoints(lat, steps, checkpoint_every)
        final = lat.state()
        for q, params in specs:
            lat.set_state(final)
            adj = Adjoint(lat)
            try:
                vals.append(adj.seed_flat(q, params))
                dW, dG, _ = backward_through(lat, adj, ckpts, steps, checkpoint_every)
            finally:
                adj.close()
            dWs.append(dW)
            dGs.append(dG)
    finally:
        lat.close()
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

    class FlatSlab(torch.autograd.Function):
        """(sigma_0, delta, interface width, n_l/n_g) of a flat slab after a
        fixed number of steps from a fixed initial density, as a function of
        the stencil group weights W and G.  forward runs the steps (keeping
        checkpoints) and measures the four quantities on the device;
        backward seeds the adjoint with sum_k g_k dQ_k (one sweep back
        through the checkpoints, whatever the number of outputs used)."""

        @staticmethod
        def forward(ctx, W, G, spec):
            lat = _spec_lattice(spec, W.detach().cpu().numpy().astype(np.float64), float(G))
            try:
                ckpts = forward_with_checkpoints(lat, spec["steps"], spec.get("checkpoint_every", 100))
                final = lat.state()
                qs = _spec_quantities(spec)
                adj = Adjoint(lat)
                try:
                    vals = [adj.seed_flat(q, p, 0.0) for q, p in qs]   # values only
                finally:
                    adj.close()
            finally:
                lat.close()
            ctx.spec = spec
            ctx.ckpts = ckpts
            ctx.final = final
            ctx.save_for_backward(W, G)
            return W.new_tensor(vals)

        @staticmethod
        def backward(ctx, g):
            W, G = ctx.saved_tensors
            spec = ctx.spec
            lat = _spec_lattice(spec, W.detach().cpu().numpy().astype(np.float64), float(G))
            try:
                lat.set_state(ctx.final)
                adj = Adjoint(lat)
                try:
                    for (q, p), gk in zip(_spec_quantities(spec), g.detach().cpu().numpy()):
                        if gk != 0.0:
                            adj.seed_flat(q, p, float(gk))
                    dW, dG, _ = backward_through(lat, adj, ctx.ckpts, spec["steps"],
                                                 spec.get("checkpoint_every", 100))
                finally:
                    adj.close()
            finally:
                lat.close()
            return W.new_tensor(dW), G.new_tensor(dG), None

    _FN = FlatSlab
    return FlatSlab


def _spec_lattice(spec, W, G):
    return Lattice(spec["lattice"], spec["shape"], spec["rho"], spec["bases"], W,
                   precision=spec.get("precision", "fp64"), tau=spec.get("tau", 1.0), G=G,
                   convention=spec.get("convention", "literal"), psi_eps=spec.get("psi_eps"))


def _spec_quantities(spec):
    nx = spec["shape"][0]
    return [(LB_FLAT_SIGMA, None), (LB_FLAT_DELTA, None),
            interface_width(spec.get("n_liquid", 0.0), spec.get("n_gas", 1.0),
                            spec.get("n_interfaces", 2)),
            density_ratio(spec.get("x_liquid", nx // 2), spec.get("x_gas", 0))]


def flat_slab(W, G, spec):
    """Differentiable (sigma_0, delta, interface width, n_l/n_g) of a flat slab
    (torch, shape [4]): W a tensor of group weights (the order of
    spec['bases']), G a scalar tensor; spec holds lattice, shape, rho, bases,
    steps, n_liquid, n_gas (width reference), x_liquid, x_gas (ratio columns)
    and optionally precision, tau, convention, psi_eps, checkpoint_every,
    n_interfaces."""
    return _torch_function().apply(W, G, spec)


def flat_sigma(W, G, spec):
    """Differentiable sigma_0 alone (the first output of flat_slab)."""
    return flat_slab(W, G, spec)[0]


__all__ = ["Adjoint", "sigma_and_gradient", "density_functional_and_gradient", "density_ratio",
           "interface_width", "tolman_and_gradient", "flat_quantity_and_gradient",
           "forward_with_checkpoints", "backward_through", "slab_observables", "tune_slab",
           "flat_slab", "flat_sigma", "LB_FLAT_SIGMA", "LB_FLAT_DELTA", "LB_FLAT_WIDTH",
           "LB_FLAT_RATIO", "LbError"]
