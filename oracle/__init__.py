"""FP64 CPU oracle of the Shan-Chen extended-stencil lattice-Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  It shares no code with the CUDA library (``paper_2505_23647_gb300``)
and the product never calls it.

The C core (``sclbm_oracle.c``) is compiled with gcc ``-O2
-ffp-contract=off`` (IEEE binary64, no FMA contraction) into
``oracle/_build/``.  ``stencil.py`` holds the exact-rational stencil algebra
and ``analysis.py`` the post-processing (surface tension, Tolman length,
coexistence) written from the paper.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values the paper prints, closed forms, invariants or brute force;
see the test files for the pin of each function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import fsum

import numpy as np

from . import stencil as _st

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sclbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")

_lib = None

LATTICES = {"D2Q9": (2, 9), "D3Q19": (3, 19)}

# Velocity tables in the oracle's (and the state layout's) order.
C9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
               [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
C19 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                [0, 0, 1], [0, 0, -1], [1, 1, 0], [-1, -1, 0], [1, -1, 0],
                [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
                [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.int64)


def build(force=False):
    """Compile the C oracle (gcc, no contraction) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
    lib.or_psi.argtypes = [d, i, d]
    lib.or_psi.restype = d
    lib.or_exp_cr.argtypes = [d]
    lib.or_exp_cr.restype = d
    lib.or_step.argtypes = [i, i, i, i, i, dp, i, ip, dp, d, d, i, d, i, d]
    lib.or_step.restype = i
    lib.or_fields.argtypes = [i, i, i, i, i, dp, i, ip, dp, d, i, d, dp, dp, dp, dp, dp]
    lib.or_fields.restype = i
    lib.or_node_post.argtypes = [i, i, i, i, i, dp, l, l, l, i, ip, dp, d, d, i, d, dp, d]
    lib.or_node_post.restype = i
    lib.or_init_feq.argtypes = [i, i, i, i, i, dp, dp, dp]
    lib.or_init_feq.restype = i
    lib.or_pressure_tensor.argtypes = [i, i, i, i, dp, dp, i, ip, dp, d, dp]
    lib.or_pressure_tensor.restype = i
    lib.or_force_field.argtypes = [i, i, i, i, dp, i, ip, dp, d, dp]
    lib.or_force_field.restype = i
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def pair_arrays(groups, dim):
    """Canonical (e, -e) pair list as C arrays: int32 [P][3], float64 [P]."""
    pairs = _st.canonical_pairs(groups)
    vec = np.zeros((len(pairs), 3), dtype=np.int32)
    w = np.zeros(len(pairs), dtype=np.float64)
    for k, (v, wt) in enumerate(pairs):
        vec[k, :dim] = v
        w[k] = float(wt)
    return np.ascontiguousarray(vec), w


def g_prime(G, convention="literal"):
    """Force prefactor G' of eq. ``sc_f``: G (literal, no c_s^2) or G c_s^2 =
    G/3 (the paper's convention)."""
    if convention == "literal":
        return float(G)
    if convention == "paper":
        return float(G) / 3.0
    raise ValueError(convention)


class Oracle:
    """A periodic lattice with a forcing stencil, advanced by the C oracle.

    ``f`` holds post-streaming populations, shape (Q, nz, ny, nx), float64.
    """

    def __init__(self, lattice, shape, groups, tau=1.0, G=-5.0,
                 convention="literal", psi_kind=0, psi_eps=0.0, forcing_A=0.0):
        self.D, self.Q = LATTICES[lattice]
        nz, ny, nx = shape if len(shape) == 3 else (1,) + tuple(shape)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.groups = [(tuple(b), w) for b, w in groups]
        self.vec, self.w = pair_arrays(self.groups, self.D)
        self.tau = float(tau)
        self.Gp = g_prime(G, convention)
        self.psi_kind = int(psi_kind)
        self.psi_eps = float(psi_eps)
        self.forcing_A = float(forcing_A)
        self.f = None
        self.steps_done = 0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def init_equilibrium(self, rho, u=None):
        lib = _load()
        rho = np.ascontiguousarray(np.broadcast_to(rho, self.shape), dtype=np.float64)
        f = np.empty((self.Q,) + self.shape, dtype=np.float64)
        up = None
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.D, *self.shape)
            up = _dp(u)
        rc = lib.or_init_feq(self.D, self.Q, self.nx, self.ny, self.nz, _dp(rho), up, _dp(f))
        if rc:
            raise ValueError(f"or_init_feq failed ({rc})")
        self.f = f
        return self

    def set_state(self, f):
        self.f = np.ascontiguousarray(f, dtype=np.float64).reshape((self.Q,) + self.shape).copy()
        return self

    def step(self, nsteps=1):
        lib = _load()
        rc = lib.or_step(self.D, self.Q, self.nx, self.ny, self.nz, _dp(self.f),
                         len(self.w), _ip(self.vec), _dp(self.w), self.tau, self.Gp,
                         self.psi_kind, self.psi_eps, int(nsteps), self.forcing_A)
        if rc < 0:
            raise RuntimeError(f"or_step failed ({rc})")
        self.steps_done += nsteps
        return rc  # 0, or 1 + first step with n <= 0 / NaN

    def fields(self):
        """dict with n, psi, F (D,...), mom = j + F/2 (D,...), u (D,...)."""
        lib = _load()
        n = np.empty(self.shape)
        psi = np.empty(self.shape)
        F = np.empty((self.D,) + self.shape)
        mom = np.empty((self.D,) + self.shape)
        u = np.empty((self.D,) + self.shape)
        rc = lib.or_fields(self.D, self.Q, self.nx, self.ny, self.nz, _dp(self.f),
                           len(self.w), _ip(self.vec), _dp(self.w), self.Gp,
                           self.psi_kind, self.psi_eps, _dp(n), _dp(psi), _dp(F),
                           _dp(mom), _dp(u))
        if rc:
            raise RuntimeError(f"or_fields failed ({rc})")
        return {"n": n, "psi": psi, "F": F, "mom": mom, "u": u}

    def node_post(self, x, y, z=0):
        """Post-collision populations at node (x, y, z) from the current f."""
        lib = _load()
        out = np.empty(self.Q)
        rc = lib.or_node_post(self.D, self.Q, self.nx, self.ny, self.nz, _dp(self.f),
                              int(x), int(y), int(z), len(self.w), _ip(self.vec),
                              _dp(self.w), self.tau, self.Gp, self.psi_kind,
                              self.psi_eps, _dp(out), self.forcing_A)
        if rc:
            raise RuntimeError(f"or_node_post failed ({rc})")
        return out

    def pressure_tensor(self):
        """Lattice pressure tensor incl. (n/3) delta; components (xx,xy,yy) in
        2D or (xx,xy,xz,yy,yz,zz) in 3D, shape (ncomp, nz, ny, nx)."""
        lib = _load()
        fl = self.fields()
        nc = 3 if self.D == 2 else 6
        P = np.empty((nc,) + self.shape)
        rc = lib.or_pressure_tensor(self.D, self.nx, self.ny, self.nz, _dp(fl["n"]),
                                    _dp(fl["psi"]), len(self.w), _ip(self.vec),
                                    _dp(self.w), self.Gp, _dp(P))
        if rc == -3:
            raise NotImplementedError("stencil group outside Appendices E/F")
        if rc:
            raise RuntimeError(f"or_pressure_tensor failed ({rc})")
        return P

    def observables(self):
        """mass, momentum (exact sums rounded once), max |u|, min/max n."""
        fl = self.fields()
        n = fl["n"]
        mom = [fsum(fl["mom"][k].ravel().tolist()) for k in range(self.D)]
        uu = fl["u"][0] * fl["u"][0]
        for k in range(1, self.D):
            uu = uu + fl["u"][k] * fl["u"][k]
        return {"mass": fsum(n.ravel().tolist()),
                "mom": mom + [0.0] * (3 - self.D),
                "umax": float(np.sqrt(uu).max()),
                "rho_min": float(n.min()), "rho_max": float(n.max())}


def force_from_psi(lattice, psi_field, groups, Gp):
    """F [D][nz][ny][nx] of eq. ``sc_f`` for a given psi field (G' given)."""
    lib = _load()
    D, _ = LATTICES[lattice]
    psi_field = np.ascontiguousarray(psi_field, dtype=np.float64)
    nz, ny, nx = psi_field.shape if psi_field.ndim == 3 else (1,) + psi_field.shape
    vec, w = pair_arrays(groups, D)
    F = np.empty((D, nz, ny, nx))
    rc = lib.or_force_field(D, nx, ny, nz, _dp(psi_field), len(w), _ip(vec), _dp(w),
                            float(Gp), _dp(F))
    if rc:
        raise RuntimeError(f"or_force_field failed ({rc})")
    return F


def pressure_tensor_from_fields(lattice, n, psi_field, groups, Gp):
    """Lattice pressure tensor (Appendices E/F) for given n and psi fields."""
    lib = _load()
    D, _ = LATTICES[lattice]
    n = np.ascontiguousarray(n, dtype=np.float64)
    psi_field = np.ascontiguousarray(psi_field, dtype=np.float64)
    nz, ny, nx = n.shape if n.ndim == 3 else (1,) + n.shape
    vec, w = pair_arrays(groups, D)
    nc = 3 if D == 2 else 6
    P = np.empty((nc, nz, ny, nx))
    rc = lib.or_pressure_tensor(D, nx, ny, nz, _dp(n), _dp(psi_field), len(w), _ip(vec),
                                _dp(w), float(Gp), _dp(P))
    if rc == -3:
        raise NotImplementedError("stencil group outside Appendices E/F")
    if rc:
        raise RuntimeError(f"or_pressure_tensor failed ({rc})")
    return P


def psi(n, kind=0, eps=0.0):
    lib = _load()
    return lib.or_psi(float(n), int(kind), float(eps))


def exp_cr(x):
    """Correctly rounded exp (binary128 evaluation rounded once)."""
    lib = _load()
    return lib.or_exp_cr(float(x))


def exp_cr_array(xs):
    lib = _load()
    return np.array([lib.or_exp_cr(float(v)) for v in np.ravel(xs)]).reshape(np.shape(xs))
