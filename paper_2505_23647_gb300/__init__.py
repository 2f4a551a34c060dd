"""Python binding of the GB300 Shan-Chen lattice-Boltzmann library.

Thin ctypes marshalling over the C ABI of ``include/sclbm.h`` (same names:
``lb_create``, ``lb_set_stencil``, ``lb_step``, ``lb_observables``,
``lb_pressure_tensor``, ...).  Every step of the model runs in the CUDA
kernels of ``_lib/libsclbm.so``; this module only converts arguments (numpy
arrays or CPU torch tensors in, numpy arrays out) and raises ``LbError`` for
a non-OK status.  There is no CPU fallback: importing the package without the
built library raises ``ImportError``.

``Lattice`` is a small convenience owner of one context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsclbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"CUDA library not built ({LIB_PATH} missing); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` or "
        "`python paper_2505_23647_gb300/build.py`")

_lib = ctypes.CDLL(LIB_PATH)

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_EUNSUPPORTED, LB_ESTATE = range(7)
LB_D2Q9, LB_D3Q19 = 0, 1
LB_FP64, LB_FP32_SHIFTED = 0, 1
LB_G_LITERAL, LB_G_TIMES_CS2 = 0, 1
LB_PSI_EXP, LB_PSI_EPS = 0, 1
LB_MAX_PAIRS = 160


class lb_params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("precision", ctypes.c_int), ("tau", ctypes.c_double),
                ("G", ctypes.c_double), ("g_convention", ctypes.c_int),
                ("psi_kind", ctypes.c_int), ("psi_eps", ctypes.c_double),
                ("rho0_shift", ctypes.c_double), ("forcing_A", ctypes.c_double)]


class lb_stencil_info(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int), ("n_pairs", ctypes.c_int),
                ("n_vectors", ctypes.c_int), ("radius", ctypes.c_int),
                ("e2", ctypes.c_double), ("e4", ctypes.c_double), ("e6", ctypes.c_double),
                ("e8", ctypes.c_double), ("iso_residual", ctypes.c_double * 4)]


class lb_obs(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("mom", ctypes.c_double * 3),
                ("umax", ctypes.c_double), ("rho_min", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("step", ctypes.c_longlong),
                ("error_step", ctypes.c_longlong), ("exp_ambiguous", ctypes.c_longlong)]


class lb_flat_obs(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("z_s", ctypes.c_double), ("z_e", ctypes.c_double),
                ("delta", ctypes.c_double), ("delta_ads", ctypes.c_double),
                ("n_l", ctypes.c_double), ("n_g", ctypes.c_double),
                ("window_lo", ctypes.c_int), ("window_hi", ctypes.c_int),
                ("rising", ctypes.c_int)]


class lb_curved_obs(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_double), ("n_out", ctypes.c_double),
                ("P_in", ctypes.c_double), ("P_out", ctypes.c_double), ("dP", ctypes.c_double),
                ("R_e", ctypes.c_double), ("R_s", ctypes.c_double),
                ("sigma_s", ctypes.c_double), ("bubble", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p

_SIGS = {
    "lb_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "lb_last_cuda_error": ([], ctypes.c_char_p),
    "lb_params_default": ([ctypes.POINTER(lb_params)], ctypes.c_int),
    "lb_expand_stencil": ([ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_int, _ip, _dp, _ip,
                           ctypes.POINTER(lb_stencil_info)], ctypes.c_int),
    "lb_create": ([ctypes.POINTER(lb_params), _dp, _dp, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "lb_destroy": ([_vp], ctypes.c_int),
    "lb_set_stencil": ([_vp, ctypes.c_int, _ip, _dp, ctypes.POINTER(lb_stencil_info)], ctypes.c_int),
    "lb_step": ([_vp, ctypes.c_int], ctypes.c_int),
    "lb_sync": ([_vp], ctypes.c_int),
    "lb_observables": ([_vp, ctypes.POINTER(lb_obs)], ctypes.c_int),
    "lb_pressure_tensor": ([_vp, _dp], ctypes.c_int),
    "lb_flat_interfaces": ([_vp, ctypes.c_int, ctypes.POINTER(lb_flat_obs), _ip], ctypes.c_int),
    "lb_curved_interface": ([_vp, _dp, ctypes.POINTER(lb_curved_obs)], ctypes.c_int),
    "lb_fit_laplace": ([ctypes.POINTER(lb_curved_obs), ctypes.c_int, ctypes.c_int, _dp, _dp],
                       ctypes.c_int),
    "lb_fit_tolman": ([ctypes.POINTER(lb_curved_obs), ctypes.c_int, ctypes.c_int,
                       ctypes.c_double, _dp, _dp], ctypes.c_int),
    "lb_get_fields": ([_vp, _dp, _dp], ctypes.c_int),
    "lb_get_state": ([_vp, _dp], ctypes.c_int),
    "lb_set_state": ([_vp, _dp], ctypes.c_int),
    "lb_exp_cr": ([_dp, _dp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "lb_psi_eval": ([ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_longlong,
                     ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "lb_kernel_launches": ([_vp], ctypes.c_longlong),
    "lb_device_counters": ([_vp, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "lb_timing": ([_vp, ctypes.c_int], ctypes.c_int),
    "lb_set_option": ([_vp, ctypes.c_int, ctypes.c_longlong], ctypes.c_int),
    "lb_step_fp64_static": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                             ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                             _ip, _dp, _vp, _vp, _vp], ctypes.c_int),
    "lb_fused_active": ([_vp], ctypes.c_int),
    "lb_timing_read": ([_vp, _dp, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "lb_adjoint_create": ([_vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "lb_adjoint_destroy": ([_vp], ctypes.c_int),
    "lb_adjoint_set": ([_vp, _dp], ctypes.c_int),
    "lb_adjoint_get": ([_vp, _dp], ctypes.c_int),
    "lb_adjoint_zero_grad": ([_vp], ctypes.c_int),
    "lb_adjoint_seed_sigma": ([_vp, ctypes.c_int, _dp], ctypes.c_int),
    "lb_adjoint_seed_pt": ([_vp, _dp, _dp], ctypes.c_int),
    "lb_adjoint_seed_flat": ([_vp, ctypes.c_int, _dp, ctypes.c_double, _dp], ctypes.c_int),
    "lb_adjoint_run": ([_vp, ctypes.c_int], ctypes.c_int),
    "lb_adjoint_gradient": ([_vp, _dp, _dp], ctypes.c_int),
    "lb_batch_create": ([ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.POINTER(_vp)],
                        ctypes.c_int),
    "lb_batch_destroy": ([_vp], ctypes.c_int),
    "lb_batch_step": ([_vp, ctypes.c_int], ctypes.c_int),
    "lb_batch_sync": ([_vp], ctypes.c_int),
    "lb_batch_launches": ([_vp], ctypes.c_longlong),
    "lb_batch_tile_count": ([], ctypes.c_int),
    "lb_batch_tile_shape": ([ctypes.c_int, _ip, _ip], ctypes.c_int),
    "lb_batch_set_tile": ([_vp, ctypes.c_int], ctypes.c_int),
    "lb_batch_get_tile": ([_vp], ctypes.c_int),
    "lb_batch_tune": ([_vp, ctypes.c_int, _dp], ctypes.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class LbError(RuntimeError):
    def __init__(self, status, where=""):
        msg = _lib.lb_status_str(status).decode()
        cu = _lib.lb_last_cuda_error().decode()
        if status == LB_ECUDA and cu:
            msg += f" ({cu})"
        super().__init__(f"{where}: {msg}" if where else msg)
        self.status = status


def _check(status, where):
    if status != LB_OK:
        raise LbError(status, where)


def _f64(a, shape=None):
    if a is None:
        return None
    if hasattr(a, "detach"):          # torch tensor (CPU)
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def lb_params_default():
    p = lb_params()
    _check(_lib.lb_params_default(ctypes.byref(p)), "lb_params_default")
    return p


def make_params(lattice="D2Q9", shape=(64, 64), precision="fp64", tau=1.0, G=-5.0,
                convention="literal", rho0_shift=0.5, psi_eps=None, forcing_A=0.0):
    """lb_params from Python values; shape is (nx, ny) or (nx, ny, nz);
    psi_eps (a float) selects psi_eps = (n/(eps+n))^(1/eps), None exp(-1/n)."""
    p = lb_params_default()
    p.lattice = {"D2Q9": LB_D2Q9, "D3Q19": LB_D3Q19}[lattice]
    p.nx, p.ny = int(shape[0]), int(shape[1])
    p.nz = int(shape[2]) if len(shape) > 2 else 1
    p.precision = {"fp64": LB_FP64, "fp32": LB_FP32_SHIFTED}[precision]
    p.tau, p.G = float(tau), float(G)
    p.g_convention = {"literal": LB_G_LITERAL, "paper": LB_G_TIMES_CS2}[convention]
    p.rho0_shift = float(rho0_shift)
    if psi_eps is not None:
        p.psi_kind, p.psi_eps = LB_PSI_EPS, float(psi_eps)
    p.forcing_A = float(forcing_A)
    return p


def _groups_arrays(bases, weights, dim):
    b = np.ascontiguousarray(np.asarray(bases, dtype=np.int32).reshape(-1, dim))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).ravel())
    if len(b) != len(w):
        raise ValueError("one weight per group")
    return b, w


def lb_expand_stencil(dim, bases, weights):
    """(pair vectors [P][3], pair weights [P], lb_stencil_info)."""
    b, w = _groups_arrays(bases, weights, dim)
    vec = np.zeros((LB_MAX_PAIRS, 3), dtype=np.int32)
    pw = np.zeros(LB_MAX_PAIRS)
    n = ctypes.c_int(0)
    info = lb_stencil_info()
    _check(_lib.lb_expand_stencil(dim, len(w), b.ctypes.data_as(_ip), _ptr(w), LB_MAX_PAIRS,
                                  vec.ctypes.data_as(_ip), _ptr(pw), ctypes.byref(n),
                                  ctypes.byref(info)), "lb_expand_stencil")
    return vec[:n.value].copy(), pw[:n.value].copy(), info


def lb_create(params, rho_init, u_init=None, stream=None):
    """Returns an opaque context handle (int).  rho_init: N float64 values
    (x fastest); u_init: [D][N] or None; stream: cudaStream_t as int (e.g.
    ``torch.cuda.current_stream().cuda_stream``) or None."""
    N = max(params.nx * params.ny * params.nz, 0)
    rho = _f64(rho_init).ravel()
    u = _f64(u_init).ravel() if u_init is not None else None
    if rho.size < N:
        raise ValueError(f"rho_init has {rho.size} values, the lattice {N}")
    ctx = _vp()
    _check(_lib.lb_create(ctypes.byref(params), _ptr(rho), _ptr(u),
                          _vp(stream) if stream else None, ctypes.byref(ctx)), "lb_create")
    return ctx.value


def lb_destroy(ctx):
    _check(_lib.lb_destroy(_vp(ctx)), "lb_destroy")


def lb_set_stencil(ctx, dim, bases, weights):
    b, w = _groups_arrays(bases, weights, dim)
    info = lb_stencil_info()
    _check(_lib.lb_set_stencil(_vp(ctx), len(w), b.ctypes.data_as(_ip), _ptr(w),
                               ctypes.byref(info)), "lb_set_stencil")
    return info


def lb_step(ctx, nsteps=1):
    _check(_lib.lb_step(_vp(ctx), int(nsteps)), "lb_step")


def lb_sync(ctx):
    """Returns the status (LB_OK or LB_EUNSTABLE); raises for other errors."""
    s = _lib.lb_sync(_vp(ctx))
    if s not in (LB_OK, LB_EUNSTABLE):
        raise LbError(s, "lb_sync")
    return s


def lb_observables(ctx):
    """dict of observables; 'status' is LB_OK or LB_EUNSTABLE."""
    o = lb_obs()
    s = _lib.lb_observables(_vp(ctx), ctypes.byref(o))
    if s not in (LB_OK, LB_EUNSTABLE):
        raise LbError(s, "lb_observables")
    return {"mass": o.mass, "mom": list(o.mom), "umax": o.umax, "rho_min": o.rho_min,
            "rho_max": o.rho_max, "step": o.step, "error_step": o.error_step,
            "exp_ambiguous": o.exp_ambiguous, "status": s}


def lb_pressure_tensor(ctx, N, dim, out=None):
    nc = 3 if dim == 2 else 6
    out = np.empty((nc, N)) if out is None else out
    _check(_lib.lb_pressure_tensor(_vp(ctx), _ptr(out)), "lb_pressure_tensor")
    return out


def _struct_dict(o):
    return {k: getattr(o, k) for k, _ in o._fields_}


def lb_flat_interfaces(ctx, max_interfaces=64):
    """Per-interface dicts (sigma, z_s, z_e, delta, delta_ads, n_l, n_g,
    window_lo, window_hi, rising) of a flat slab, computed on the device."""
    out = (lb_flat_obs * max(1, max_interfaces))()
    n = ctypes.c_int(0)
    _check(_lib.lb_flat_interfaces(_vp(ctx), int(max_interfaces), out, ctypes.byref(n)),
           "lb_flat_interfaces")
    return [_struct_dict(out[i]) for i in range(min(n.value, max_interfaces))]


def lb_curved_interface(ctx, center):
    """Dict (n_in, n_out, P_in, P_out, dP, R_e, R_s, sigma_s, bubble) of a
    droplet or bubble centred at `center` (x, y[, z]), computed on the device."""
    c = np.ascontiguousarray(np.asarray(center, dtype=np.float64))
    o = lb_curved_obs()
    _check(_lib.lb_curved_interface(_vp(ctx), _ptr(c), ctypes.byref(o)), "lb_curved_interface")
    d = _struct_dict(o)
    d["bubble"] = bool(d["bubble"])
    return d


def _curved_array(runs):
    arr = (lb_curved_obs * len(runs))()
    for i, r in enumerate(runs):
        for k, _ in lb_curved_obs._fields_:
            setattr(arr[i], k, int(r[k]) if k == "bubble" else float(r[k]))
    return arr


def lb_fit_laplace(runs, dim):
    """(sigma, intercept) of the Laplace law over curved-interface results."""
    s, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.lb_fit_laplace(_curved_array(runs), len(runs), dim, ctypes.byref(s),
                               ctypes.byref(b)), "lb_fit_laplace")
    return s.value, b.value


def lb_fit_tolman(runs, dim, sigma0):
    """(delta, intercept) of the curved Tolman fit over curved-interface results."""
    d, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.lb_fit_tolman(_curved_array(runs), len(runs), dim, float(sigma0), ctypes.byref(d),
                              ctypes.byref(b)), "lb_fit_tolman")
    return d.value, b.value


def lb_get_fields(ctx, N, dim):
    rho = np.empty(N)
    u = np.empty((dim, N))
    _check(_lib.lb_get_fields(_vp(ctx), _ptr(rho), _ptr(u)), "lb_get_fields")
    return rho, u


def lb_get_state(ctx, Q, N, out=None):
    f = np.empty((Q, N)) if out is None else out
    _check(_lib.lb_get_state(_vp(ctx), _ptr(f)), "lb_get_state")
    return f


def lb_set_state(ctx, f):
    f = _f64(f)
    _check(_lib.lb_set_state(_vp(ctx), _ptr(f)), "lb_set_state")


def lb_exp_cr(x):
    x = _f64(x).ravel()
    y = np.empty_like(x)
    amb = ctypes.c_longlong(0)
    _check(_lib.lb_exp_cr(_ptr(x), _ptr(y), len(x), ctypes.byref(amb)), "lb_exp_cr")
    return y, amb.value


def lb_psi_eval(n, eps=None):
    """Binary64 psi of the step's device code: exp(-1/n), or psi_eps when eps
    is given.  Returns (psi, number of uncertified roundings)."""
    x = _f64(n).ravel()
    y = np.empty_like(x)
    amb = ctypes.c_longlong(0)
    kind, e = (LB_PSI_EXP, 0.0) if eps is None else (LB_PSI_EPS, float(eps))
    _check(_lib.lb_psi_eval(kind, e, _ptr(x), _ptr(y), len(x), ctypes.byref(amb)), "lb_psi_eval")
    return y, amb.value


def lb_kernel_launches(ctx):
    return int(_lib.lb_kernel_launches(_vp(ctx)))


def lb_device_counters(ctx):
    """Raw device counters: dict with error_step, device_step, exp_ambiguous,
    blocks_done, timeouts."""
    out = (ctypes.c_longlong * 5)()
    _check(_lib.lb_device_counters(_vp(ctx), out), "lb_device_counters")
    keys = ("error_step", "device_step", "exp_ambiguous", "blocks_done", "timeouts")
    return dict(zip(keys, (int(v) for v in out)))


LB_OPT_FUSED, LB_OPT_ZCHUNK, LB_OPT_TMA, LB_OPT_WAIT_POLLS = 1, 2, 3, 5


def lb_set_option(ctx, option, value):
    _check(_lib.lb_set_option(_vp(ctx), int(option), int(value)), "lb_set_option")


def lb_fused_active(ctx):
    """0: two-kernel path, 1: fused D3Q19 kernel (cp.async), 2: fused D3Q19
    kernel (TMA), 3: fused D2Q9 kernel."""
    return int(_lib.lb_fused_active(_vp(ctx)))


def lb_batch_tile_shapes():
    """The candidate tile shapes (tx, ty) of batches, by index."""
    out = []
    for i in range(_lib.lb_batch_tile_count()):
        tx, ty = ctypes.c_int(), ctypes.c_int()
        _check(_lib.lb_batch_tile_shape(i, ctypes.byref(tx), ctypes.byref(ty)), "lb_batch_tile_shape")
        out.append((tx.value, ty.value))
    return out


class Batch:
    """Many D2Q9 shifted-FP32 lattices stepped by one launch per step
    (``lb_batch_*``).  ``lattices`` are :class:`Lattice` objects (kept alive
    by the batch); destroy the batch before them."""

    def __init__(self, lattices, stream=None):
        self.members = list(lattices)
        arr = (_vp * len(self.members))(*[m.ctx for m in self.members])
        out = _vp()
        _check(_lib.lb_batch_create(arr, len(self.members), _vp(stream) if stream else None,
                                    ctypes.byref(out)), "lb_batch_create")
        self.b = out.value

    def step(self, n=1):
        _check(_lib.lb_batch_step(_vp(self.b), int(n)), "lb_batch_step")

    def sync(self):
        return _lib.lb_batch_sync(_vp(self.b))

    def launches(self):
        return int(_lib.lb_batch_launches(_vp(self.b)))

    def set_tile(self, index):
        _check(_lib.lb_batch_set_tile(_vp(self.b), int(index)), "lb_batch_set_tile")

    def tile(self):
        return int(_lib.lb_batch_get_tile(_vp(self.b)))

    def tune(self, steps_per_trial=20):
        """Pick the fastest tile shape; returns (index, trial ms per shape)."""
        ms = np.zeros(_lib.lb_batch_tile_count())
        _check(_lib.lb_batch_tune(_vp(self.b), int(steps_per_trial), _ptr(ms)), "lb_batch_tune")
        return self.tile(), ms

    def close(self):
        if self.b:
            _lib.lb_batch_destroy(_vp(self.b))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


LB_STATIC_MAX_NODES = 1 << 20


def lb_step_fp64_static(params, pair_vec, pair_w, f_in_ptr, f_out_ptr, stream=None):
    """One binary64 step that allocates nothing (see sclbm.h).  f_in_ptr and
    f_out_ptr are device addresses (e.g. ``tensor.data_ptr()``) of [Q][N]
    float64 buffers the caller owns; pair_vec/pair_w come from
    lb_expand_stencil.  Enqueued on ``stream`` (a cudaStream_t as int)."""
    vec = np.ascontiguousarray(np.asarray(pair_vec, dtype=np.int32).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(pair_w, dtype=np.float64).ravel())
    _check(_lib.lb_step_fp64_static(params.lattice, params.nx, params.ny, params.nz,
                                    params.tau, params.G, params.g_convention, len(w),
                                    vec.ctypes.data_as(_ip), _ptr(w), _vp(f_in_ptr),
                                    _vp(f_out_ptr), _vp(stream) if stream else None),
           "lb_step_fp64_static")


LB_KERNEL_PSI, LB_KERNEL_COLLIDE, LB_KERNEL_FUSED, LB_KERNEL_OTHER = range(4)
KERNEL_KINDS = ("psi", "collide", "fused", "other")


def lb_timing(ctx, enable):
    _check(_lib.lb_timing(_vp(ctx), int(bool(enable))), "lb_timing")


def lb_timing_read(ctx):
    """{kind: (milliseconds, launches)} of the kernels timed since lb_timing(1)."""
    ms = np.zeros(4)
    n = (ctypes.c_longlong * 4)()
    _check(_lib.lb_timing_read(_vp(ctx), _ptr(ms), n), "lb_timing_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


class Lattice:
    """Owner of one context: ``Lattice('D3Q19', (nx, ny, nz), rho, ...)``.
    Arrays in and out are numpy with shape (nz, ny, nx) / (C, nz, ny, nx)."""

    def __init__(self, lattice, shape_xyz, rho, stencil_bases=None, stencil_weights=None,
                 precision="fp64", tau=1.0, G=-5.0, convention="literal", rho0_shift=0.5,
                 u=None, stream=None, psi_eps=None, forcing_A=0.0):
        self.params = make_params(lattice, shape_xyz, precision, tau, G, convention, rho0_shift,
                                  psi_eps, forcing_A)
        self.D = 2 if lattice == "D2Q9" else 3
        self.Q = 9 if lattice == "D2Q9" else 19
        p = self.params
        self.shape = (p.nz, p.ny, p.nx)
        self.N = p.nx * p.ny * p.nz
        self.ctx = lb_create(p, rho, u, stream)
        self.info = None
        if stencil_bases is not None:
            self.set_stencil(stencil_bases, stencil_weights)

    def set_stencil(self, bases, weights):
        self.info = lb_set_stencil(self.ctx, self.D, bases, weights)
        self.stencil_bases = np.asarray(bases)
        self.stencil_weights = np.asarray(weights, dtype=np.float64)
        return self.info

    def step(self, n=1):
        lb_step(self.ctx, n)

    def sync(self):
        return lb_sync(self.ctx)

    def observables(self):
        return lb_observables(self.ctx)

    def pressure_tensor(self):
        return lb_pressure_tensor(self.ctx, self.N, self.D).reshape((-1,) + self.shape)

    def flat_interfaces(self, max_interfaces=64):
        return lb_flat_interfaces(self.ctx, max_interfaces)

    def curved_interface(self, center):
        return lb_curved_interface(self.ctx, center)

    def fields(self):
        rho, u = lb_get_fields(self.ctx, self.N, self.D)
        return rho.reshape(self.shape), u.reshape((self.D,) + self.shape)

    def state(self):
        return lb_get_state(self.ctx, self.Q, self.N).reshape((self.Q,) + self.shape)

    def set_state(self, f):
        lb_set_state(self.ctx, np.asarray(f).reshape(self.Q, self.N))

    def launches(self):
        return lb_kernel_launches(self.ctx)

    def close(self):
        if self.ctx:
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
