"""Oracle: forcing-stencil algebra in exact rational arithmetic.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / reference leg use the oracle.

Every function restates a definition of Lulli & Ching, "Higher-order Tuning
of Interface Physics in Multiphase Lattice Boltzmann":

* groups of stencil vectors are orbits under coordinate permutations and sign
  flips, one weight per group (Sec. III A, text after eq. ``sc_f``);
* moments <e^{mu_1}...e^{mu_2n}>_W = sum_a W_a e_a^{mu_1}...e_a^{mu_2n}
  (Sec. III A);
* isotropy coefficients e_{2n}: the coefficient of the fully isotropic
  tensor Delta^{(2n)} in the 2n-th moment (Sec. IV, eq. after ``sec:met``),
  read off the mixed moments e2=<x^2>, e4=<x^2y^2>, e6=<x^4y^2>/3,
  e8=<x^4y^4>/9 (Table ``tab:defe2nI2n`` reproduces these readings);
* anisotropy/isotropy conditions (Sec. IV, Appendix D);
* the canonical pair order used by the step (a reading of how the symmetric
  sum of eq. ``sc_f`` is accumulated, stated in ``canonical_pairs``).
"""
from __future__ import annotations

from fractions import Fraction as Fr
from itertools import permutations, product
from math import factorial

__all__ = ["orbit", "canonical_pairs", "full_vectors", "moment", "isotropy_coeffs",
           "isotropic_tensor_value", "isotropy_residual", "n_vectors",
           "anisotropy_2d", "radius"]


def orbit(base):
    """All vectors obtained from ``base`` by permuting coordinates and
    flipping signs (the dihedral/octahedral group of Sec. III A)."""
    out = set()
    for p in permutations(base):
        for s in product((1, -1), repeat=len(base)):
            out.add(tuple(a * b for a, b in zip(p, s)))
    out.discard(tuple(0 for _ in base))
    return sorted(out)


def _canon_base(base):
    return tuple(sorted((abs(c) for c in base), reverse=True))


def _sq(v):
    return sum(c * c for c in v)


def _is_rep(v):
    for c in v:
        if c != 0:
            return c > 0
    return False


def canonical_pairs(groups):
    """Ordered (+e/-e) representatives with their weights.

    Reading adopted for the accumulation order of the symmetric sum in
    eq. ``sc_f``: the stencil is split into pairs (e, -e), which share one
    weight; a pair is represented by the vector whose first non-zero
    component is positive.  Groups are ordered by |e|^2, ties broken by the
    base vector's sorted absolute components in descending lexicographic
    order ((3,0,0) before (2,2,1)); inside a group the representatives are
    in descending lexicographic order of (e_x, e_y, e_z).

    ``groups`` is a list of (base_vector, weight).  Returns a list of
    (vector_tuple, weight).
    """
    seen = set()
    keyed = []
    for base, w in groups:
        cb = _canon_base(base)
        if cb in seen:
            raise ValueError(f"group {cb} given twice")
        if _sq(cb) == 0:
            raise ValueError("zero base vector")
        seen.add(cb)
        keyed.append(((_sq(cb), tuple(-c for c in cb)), cb, w))
    keyed.sort(key=lambda t: t[0])
    out = []
    for _, cb, w in keyed:
        reps = [v for v in orbit(cb) if _is_rep(v)]
        reps.sort(reverse=True)
        out.extend((v, w) for v in reps)
    return out


def full_vectors(groups):
    """Every stencil vector with its weight (both members of each pair)."""
    out = []
    for v, w in canonical_pairs(groups):
        out.append((v, w))
        out.append((tuple(-c for c in v), w))
    return out


def n_vectors(groups):
    return 2 * len(canonical_pairs(groups))


def radius(groups):
    return max(max(abs(c) for c in b) for b, _ in groups)


def moment(groups, powers):
    """<prod_mu (e^mu)^{powers[mu]}>_W = sum_a W_a prod_mu (e_a^mu)^{p_mu}."""
    s = Fr(0)
    for v, w in full_vectors(groups):
        t = Fr(w)
        for c, p in zip(v, powers):
            t *= Fr(c) ** p
        s += t
    return s


def isotropy_coeffs(groups, dim):
    """(e2, e4, e6, e8) read off the mixed moments of the isotropic tensors:
    <x^2> = e2, <x^2 y^2> = e4, <x^4 y^2> = 3 e6, <x^4 y^4> = 9 e8."""
    z = [0] * dim

    def m(px, py):
        p = list(z)
        p[0] = px
        p[1] = py
        return moment(groups, p)
    return m(2, 0), m(2, 2), m(4, 2) / 3, m(4, 4) / 9


def isotropic_tensor_value(indices):
    """Delta^{mu_1...mu_2n} for one index tuple: the number of ways to split
    the indices into pairs of equal indices (recursive definition, Sec. IV).
    For counts c_k of each axis k this is prod_k (c_k - 1)!! if all c_k are
    even, else 0."""
    counts = {}
    for i in indices:
        counts[i] = counts.get(i, 0) + 1
    v = 1
    for c in counts.values():
        if c % 2:
            return 0
        v *= factorial(c) // (2 ** (c // 2) * factorial(c // 2))
    return v


def isotropy_residual(groups, dim, order):
    """max over index tuples of |<e...e>_W - e_order * Delta| at the given
    even order (Sec. IV): zero iff the moment of that order is isotropic."""
    vecs = full_vectors(groups)
    worst = Fr(0)
    e_val = None
    for idx in product(range(dim), repeat=order):
        if list(idx) != sorted(idx):
            continue
        m = Fr(0)
        for v, w in vecs:
            t = Fr(w)
            for i in idx:
                t *= v[i]
            m += t
        d = isotropic_tensor_value(idx)
        if d == 0:
            worst = max(worst, abs(m))
            continue
        if e_val is None:
            e_val = m / d
        worst = max(worst, abs(m - e_val * d))
    return worst


def anisotropy_2d(groups):
    """Two-dimensional anisotropy coefficients of Table ``tab:defe2nI2n`` as
    combinations of raw moments (reading: the combinations that vanish for an
    isotropic moment tensor and reproduce the table's coefficients):
    I40 = <x^4> - 3<x^2y^2>,  I60 = <x^6> - 5<x^4y^2>,
    I80 = <x^6y^2> - (5/3)<x^4y^4>,  I81 = <x^8> - 7<x^6y^2>."""
    m = lambda a, b: moment(groups, [a, b])
    return {"I40": m(4, 0) - 3 * m(2, 2),
            "I60": m(6, 0) - 5 * m(4, 2),
            "I80": m(6, 2) - Fr(5, 3) * m(4, 4),
            "I81": m(8, 0) - 7 * m(6, 2)}
