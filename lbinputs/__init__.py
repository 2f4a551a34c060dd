"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds *inputs only*: initial density fields, population fields
for brute-force checks, and the forcing-stencil weights that a user hands to
``lb_set_stencil``.  It contains none of the lattice-Boltzmann arithmetic
(no densities from populations, no forces, no collision); both the oracle
and the CUDA library consume what it produces.

Stencil weights
---------------
A forcing stencil is a list of symmetry groups, each given by one base
vector (its orbit under coordinate permutations and sign flips is the group,
Sec. III A) and one weight W(|e|^2).  The named stencils below are the ones
the paper prints:

* ``E4_2D``: W(1)=1/3, W(2)=1/12 (Appendix A).
* ``E6_2D`` / ``E8_2D``: maximally isotropic stencils of Table
  ``tab:e2n_values``; the E8 weights 4/21, 4/45, 1/60, 2/315, 1/5040 are the
  ones printed in Appendix B (multibelt paragraph).
* ``E4_3D``: groups (1,0,0), (1,1,0) with W = 1/6, 1/12 (the 3D fourth-order
  stencil with e2 = 1; N_e = 18 as in Table ``tab:e2n_values``).
* ``E8_3D``: groups (1,0,0), (1,1,0), (1,1,1), (2,0,0), (2,1,0), (2,1,1),
  (2,2,0) with W = 4/45, 1/21, 2/105, 5/504, 1/315, 1/630, 1/5040.  These are
  not printed in the paper; they solve its isotropy conditions (Sec. IV, e2=1,
  all anisotropy coefficients through eighth order zero).  The oracle tests
  pin them to Table ``tab:e2n_values`` (e4=4/7, e6=32/105, e8=16/105,
  N_e=92) and to the 3D->2D projection of eq. ``wproj``.
* Tuned families (Tables ``tab:e4_tuning_6``, ``tab:e4e6_tuning_8``,
  ``tab:e4e6e8_tuning_6_2d``, ``tab:e4e6e8_tuning_6_3d``) as functions of
  the knobs sigma0_hat, sigma1_hat, delta0_hat.

All weights are returned as exact ``fractions.Fraction`` values together with
their float conversion.
"""
from __future__ import annotations

from fractions import Fraction as Fr
import math

import numpy as np

__all__ = [
    "Stencil", "E4_2D", "E6_2D", "E8_2D", "E4_3D", "E8_3D",
    "stencil_e4_tuning_6", "stencil_e4e6_tuning_8",
    "stencil_e4e6e8_tuning_6", "named_stencil",
    "tanh_slab", "tanh_sphere", "random_density", "random_populations",
    "batched_instances", "splitmix64",
]


class Stencil:
    """A forcing stencil as (base vector, weight) groups in dimension ``dim``."""

    def __init__(self, name, dim, groups):
        self.name = name
        self.dim = dim
        self.groups = [(tuple(int(c) for c in b), Fr(w)) for b, w in groups]
        for b, _ in self.groups:
            if len(b) != dim:
                raise ValueError(f"base vector {b} is not {dim}-dimensional")

    @property
    def bases(self):
        return np.array([b for b, _ in self.groups], dtype=np.int32)

    @property
    def weights(self):
        return np.array([float(w) for _, w in self.groups], dtype=np.float64)

    @property
    def weights_exact(self):
        return [w for _, w in self.groups]

    def __repr__(self):
        return f"Stencil({self.name!r}, dim={self.dim}, groups={len(self.groups)})"


# --- maximally isotropic stencils (Appendix A, Appendix B, Table e2n_values) --
E4_2D = Stencil("E4_2D", 2, [((1, 0), Fr(1, 3)), ((1, 1), Fr(1, 12))])
# E6 (2D): groups 1, 2, 4 with e2 = 1 and I_{4,0} = I_{6,0} = 0.
E6_2D = Stencil("E6_2D", 2, [((1, 0), Fr(4, 15)), ((1, 1), Fr(1, 10)),
                             ((2, 0), Fr(1, 120))])
E8_2D = Stencil("E8_2D", 2, [((1, 0), Fr(4, 21)), ((1, 1), Fr(4, 45)),
                             ((2, 0), Fr(1, 60)), ((2, 1), Fr(2, 315)),
                             ((2, 2), Fr(1, 5040))])
E4_3D = Stencil("E4_3D", 3, [((1, 0, 0), Fr(1, 6)), ((1, 1, 0), Fr(1, 12))])
E8_3D = Stencil("E8_3D", 3, [((1, 0, 0), Fr(4, 45)), ((1, 1, 0), Fr(1, 21)),
                             ((1, 1, 1), Fr(2, 105)), ((2, 0, 0), Fr(5, 504)),
                             ((2, 1, 0), Fr(1, 315)), ((2, 1, 1), Fr(1, 630)),
                             ((2, 2, 0), Fr(1, 5040))])


def _groups2(d):
    return {1: (1, 0), 2: (1, 1), 4: (2, 0), 5: (2, 1), 8: (2, 2), 9: (3, 0),
            16: (4, 0), 18: (3, 3)}[d]


def _groups3(d):
    return {1: (1, 0, 0), 2: (1, 1, 0), 3: (1, 1, 1), 4: (2, 0, 0),
            5: (2, 1, 0), 6: (2, 1, 1), 8: (2, 2, 0), "9a": (2, 2, 1),
            9: (3, 0, 0), 16: (4, 0, 0), 18: (3, 3, 0)}[d]


def stencil_e4_tuning_6(dim, s0):
    """Table ``tab:e4_tuning_6``: 6th-order isotropic weights vs sigma0_hat."""
    s0 = Fr(s0)
    if dim == 2:
        w = {1: Fr(8, 15) + 4 * s0 / 3, 2: -s0 / 6 + Fr(1, 15),
             4: -5 * s0 / 24 - Fr(1, 30), 8: -s0 / 48 - Fr(1, 240)}
        return Stencil(f"T_e4_6_2D({s0})", 2, [(_groups2(k), v) for k, v in w.items()])
    w = {1: Fr(4, 15) + 2 * s0 / 3, 2: Fr(2, 15) + s0 / 3, 3: -s0 / 4 - Fr(1, 30),
         4: -s0 / 6 - Fr(1, 40), 8: -s0 / 48 - Fr(1, 240)}
    return Stencil(f"T_e4_6_3D({s0})", 3, [(_groups3(k), v) for k, v in w.items()])


def stencil_e4e6_tuning_8(dim, s0, s1):
    """Table ``tab:e4e6_tuning_8``: 8th-order isotropic weights vs (sigma0_hat, sigma1_hat)."""
    s0, s1 = Fr(s0), Fr(s1)
    if dim == 2:
        w = {1: 59 * s0 / 20 + 4 * s1 + Fr(51, 70),
             2: -187 * s0 / 240 - 41 * s1 / 24 - Fr(1, 280),
             4: -5 * s0 / 8 - s1 - Fr(3, 35),
             5: 7 * s0 / 60 + s1 / 3 + Fr(1, 70),
             8: -13 * s0 / 240 - s1 / 12 - Fr(1, 112),
             9: 59 * s0 / 1620 + 2 * s1 / 27 + Fr(1, 210),
             18: 17 * s0 / 6480 + s1 / 216 + Fr(1, 2520)}
        return Stencil(f"T_e4e6_8_2D({s0},{s1})", 2, [(_groups2(k), v) for k, v in w.items()])
    w = {1: 1789 * s0 / 420 + 121 * s1 / 18 + Fr(4, 5),
         2: -11 * s0 / 28 - 65 * s1 / 72,
         3: -s0 / 5 - 7 * s1 / 15,
         4: -1181 * s0 / 1680 - 109 * s1 / 90 - Fr(1, 10),
         5: -s0 / 56 - s1 / 72,
         6: 2 * s0 / 105 + 31 * s1 / 360,
         8: 9 * s0 / 1120 + 11 * s1 / 360,
         "9a": -s0 / 1680 - s1 / 720,
         9: 103 * s0 / 1134 + 281 * s1 / 1620 + Fr(4, 315),
         18: -s0 / 11340 - s1 / 3240,
         16: -41 * s0 / 6720 - s1 / 90 - Fr(1, 1120)}
    return Stencil(f"T_e4e6_8_3D({s0},{s1})", 3, [(_groups3(k), v) for k, v in w.items()])


def stencil_e4e6e8_tuning_6(dim, s0, s1, d0):
    """Tables ``tab:e4e6e8_tuning_6_2d`` / ``_3d``: weights vs (sigma0_hat, sigma1_hat, delta0_hat)."""
    s0, s1, d0 = Fr(s0), Fr(s1), Fr(d0)
    if dim == 2:
        w = {1: 9 * d0 / 5 + 47 * s0 / 12 + 19 * s1 / 5 + Fr(3, 5),
             2: 3 * d0 / 10 - 89 * s0 / 144 - 209 * s1 / 120 - Fr(1, 40),
             4: 9 * d0 / 10 - 17 * s0 / 120 - 11 * s1 / 10 - Fr(3, 20),
             5: -6 * d0 / 5 - 19 * s0 / 36 + 7 * s1 / 15 + Fr(1, 10),
             8: 3 * d0 / 4 + 251 * s0 / 720 - s1 / 6 - Fr(1, 16),
             9: d0 / 15 + 13 * s0 / 180 + s1 / 15,
             18: -d0 / 30 - 11 * s0 / 720 + s1 / 120 + Fr(1, 360)}
        return Stencil(f"T_e4e6e8_6_2D({s0},{s1},{d0})", 2,
                       [(_groups2(k), v) for k, v in w.items()])
    w = {1: 339 * d0 / 10 + 14359 * s0 / 720 - 149 * s1 / 120 - Fr(81, 40),
         2: -27 * d0 / 2 - 107 * s0 / 16 + 151 * s1 / 72 + Fr(9, 8),
         3: 36 * d0 / 5 + 19 * s0 / 6 - 61 * s1 / 30 - Fr(3, 5),
         4: -21 * d0 / 10 - 613 * s0 / 360 - 49 * s1 / 60 + Fr(3, 40),
         5: -9 * d0 / 20 - 19 * s0 / 96 + 137 * s1 / 720 + Fr(3, 80),
         6: -3 * d0 / 10 - 19 * s0 / 144 + 41 * s1 / 360 + Fr(1, 40),
         8: 9 * d0 / 10 + 199 * s0 / 480 - 31 * s1 / 144 - Fr(3, 40),
         "9a": -3 * d0 / 40 - 19 * s0 / 576 + 7 * s1 / 288 + Fr(1, 160),
         9: 11 * d0 / 15 + 17 * s0 / 40 - s1 / 60 - Fr(61, 1260),
         18: -d0 / 30 - 11 * s0 / 720 + s1 / 120 + Fr(1, 360),
         16: -3 * d0 / 40 - 29 * s0 / 720 + s1 / 120 + Fr(3, 560)}
    return Stencil(f"T_e4e6e8_6_3D({s0},{s1},{d0})", 3,
                   [(_groups3(k), v) for k, v in w.items()])


def named_stencil(name):
    return {"E4_2D": E4_2D, "E6_2D": E6_2D, "E8_2D": E8_2D,
            "E4_3D": E4_3D, "E8_3D": E8_3D}[name]


# --- density fields -----------------------------------------------------------
# psi_eps workload of the benchmark (D3Q19 E8 bubble): eps = 10/31 is the eps
# that eq. eps_moments gives for the E8 stencils' e4 = 4/7 (e2 = 1);
# Gp = 1.1 G'_c of psi_eps at that eps (literal reading); n_gas, n_liquid its
# coexistence pair from eq. SCMaxwell.  tests/test_oracle_physics.py checks
# the three numbers against the oracle's critical point and Maxwell
# construction.
PSI_EPS_BUBBLE = {"eps": 10.0 / 31.0, "Gp": -2.6857441579840247,
                  "n_gas": 0.43663686360362103, "n_liquid": 1.5757138898336904}


def _coords(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def tanh_slab(nx, ny, nz, x0, x1, rho_out, rho_in, width):
    """Flat liquid slab x in [x0, x1): rho = rho_out + (rho_in - rho_out) *
    (tanh((x-x0)/w) - tanh((x-x1)/w))/2, shape (nz, ny, nx), x fastest."""
    x, _, _ = _coords(nx, ny, nz)
    return rho_out + (rho_in - rho_out) * 0.5 * (np.tanh((x - x0) / width)
                                                 - np.tanh((x - x1) / width))


def tanh_sphere(nx, ny, nz, radius, rho_in, rho_out, width, center=None):
    """Droplet (rho_in > rho_out) or bubble (rho_in < rho_out) of radius R:
    rho = rho_out + (rho_in - rho_out) * (1 - tanh((r - R)/w))/2.  For nz == 1
    the shape is a disc.  The default centre is the box centre."""
    x, y, z = _coords(nx, ny, nz)
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    cx, cy, cz = center
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    if nz > 1:
        r2 = r2 + (z - cz) ** 2
    r = np.sqrt(r2)
    return rho_out + (rho_in - rho_out) * 0.5 * (1.0 - np.tanh((r - radius) / width))


def random_density(shape, seed, mean=1.0, amp=0.05):
    rng = np.random.default_rng(seed)
    return mean + amp * (2.0 * rng.random(shape) - 1.0)


def random_populations(q, shape, seed, lo=0.01, hi=0.2):
    """Positive random populations f[q][nz][ny][nx] (for brute-force checks)."""
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random((q,) + tuple(shape))


# --- batched droplet / bubble instances --------------------------------------
def splitmix64(x):
    """SplitMix64 (Steele, Lea, Flood 2014): one 64-bit output from state x."""
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def batched_instances(count=64, seed_base=0xC3,
                      sides=(64, 96, 128, 192, 256, 384, 512)):
    """Independent 2D droplet/bubble instances: square side drawn uniformly
    from ``sides``, radius uniform in [0.1, 0.35]*side, stencil uniform in
    {E4, E6, E8}, droplet or bubble with probability 1/2; instance i is
    seeded with splitmix64(seed_base + i)."""
    out = []
    for i in range(count):
        s = splitmix64(seed_base + i)
        u = [(splitmix64(s + k) >> 11) / float(1 << 53) for k in range(4)]
        side = sides[min(int(u[0] * len(sides)), len(sides) - 1)]
        radius = (0.1 + 0.25 * u[1]) * side
        stencil = (E4_2D, E6_2D, E8_2D)[min(int(u[2] * 3), 2)]
        bubble = u[3] < 0.5
        out.append({"side": side, "radius": radius, "stencil": stencil,
                    "bubble": bubble, "seed": s})
    return out
