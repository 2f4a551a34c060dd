"""Pin of the oracle's pseudopotential arithmetic: psi = RN(exp(RN(-1/n))) with
a correctly rounded exp (Sec. IV B, psi = exp(-1/n)).  The reference is an
independent 400-bit mpmath evaluation rounded once to binary64 by exact
rational arithmetic (Python's int division is correctly rounded, subnormals
included)."""
from fractions import Fraction

import mpmath
import numpy as np

import oracle


def cr_exp_reference(x):
    with mpmath.workprec(400):
        v = mpmath.exp(mpmath.mpf(x))
        man, exp = v.man, v.exp
    q = Fraction(int(man)) * (Fraction(2) ** int(exp))
    return q.numerator / q.denominator if q.numerator else 0.0


def _inputs():
    rng = np.random.default_rng(2024)
    xs = list(-rng.random(3000) * 30.0)                 # psi range (n >= 1/30)
    xs += list(-rng.random(600) * 745.2)                # full normal range
    xs += list(-708.0 - rng.random(600) * 37.2)         # subnormal results
    xs += list(-np.exp(rng.uniform(np.log(1e-300), np.log(1.0), 400)))
    xs += [0.0, -0.0, -1e-320, -745.1332191019411, -745.1332191019412, -745.14,
           -708.3964185322641, -708.39641853226, -1.0, -0.5, -2.0, -1e6]
    return xs


def test_exp_is_correctly_rounded():
    bad = []
    for x in _inputs():
        got = oracle.exp_cr(x)
        want = cr_exp_reference(x)
        if got != want:
            bad.append((x, got, want))
    assert not bad, bad[:5]


def test_psi_uses_rounded_argument():
    rng = np.random.default_rng(7)
    for n in list(0.05 + 6.0 * rng.random(300)) + [1.0, 0.15, 1.9, 5.294]:
        a = -1.0 / n
        assert oracle.psi(n) == cr_exp_reference(a)


def cr_pow_reference(r, e):
    with mpmath.workprec(400):
        v = mpmath.power(mpmath.mpf(r), mpmath.mpf(e))
        man, exp = v.man, v.exp
    q = Fraction(int(man)) * (Fraction(2) ** int(exp))
    return q.numerator / q.denominator if q.numerator else 0.0


def _psi_eps_inputs():
    rng = np.random.default_rng(29)
    ns = list(0.02 + 6.0 * rng.random(400)) + list(np.exp(rng.uniform(np.log(1e-3), np.log(50.0), 100)))
    return ns + [0.15, 1.9, 1.0, 0.456, 2.25, 1e-3, 50.0]


def test_psi_eps_is_a_correctly_rounded_power():
    # eq. psieps, psi_eps = (n/(eps+n))^(1/eps), read as
    # RN(RN(n/RN(eps+n)) ^ RN(1/eps)) with the power rounded once
    for eps in (14.0 / 29.0, 10.0 / 31.0, 0.25, 1.0, 3.0):
        e = 1.0 / eps
        for n in _psi_eps_inputs():
            r = n / (eps + n)
            assert oracle.psi(n, 1, eps) == cr_pow_reference(r, e), (eps, n)


def test_psi_eps_tends_to_exp():
    # (1 + eps/n)^(-1/eps) = exp(-1/n + eps/(2 n^2) - eps^2/(3 n^3) + ...):
    # the ratio to exp(-1/n) is 1 + eps/(2 n^2) to first order in eps; the
    # rounded base n/(eps+n) carries a relative error of at most 2^-53, which
    # the power 1/eps amplifies to 2^-53/eps
    for n in (0.15, 0.5, 1.0, 1.9, 3.0):
        for eps in (1e-4, 1e-6):
            rel = oracle.psi(n, 1, eps) / oracle.psi(n) - 1.0
            first = eps / (2.0 * n * n)
            bound = eps * eps / n ** 3 + 2.0 ** -52 / eps + 1e-13
            assert abs(rel - first) < bound, (n, eps, rel, first)
