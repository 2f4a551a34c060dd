"""Pins of the oracle's stencil algebra and of the stencil inputs against what
the paper prints (Tables tab:e2n_values, tab:e4_tuning_6, tab:e4e6_tuning_8,
tab:e4e6e8_tuning_6_2d/3d, tab:defe2nI2n, tab:pnptcoeffs,
tab:pn_minus_ptcoeffs; eqs. eps_moments, hatsigma01eI, hatdelta0eI, wproj;
Appendices A and B) and the velocity-set isotropy of Sec. II."""
from fractions import Fraction as Fr
from itertools import product
import random

import numpy as np
import pytest
import sympy as sp

import lbinputs as L
import oracle
from oracle import stencil as st
from tests import _golden as G

pytestmark = pytest.mark.filterwarnings("ignore")


def _iprod(it):
    r = 1
    for v in it:
        r *= int(v)
    return r


def _dfact(k):
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def e2n_table_convention(groups, dim, n):
    """e_{2n} = <x^{2a} y^{2b}> / ((2a-1)!!(2b-1)!!), a = ceil(n/2), b = floor(n/2)."""
    a, b = (n + 1) // 2, n // 2
    p = [0] * dim
    p[0], p[1] = 2 * a, 2 * b
    return st.moment(groups, p) / (_dfact(2 * a - 1) * _dfact(2 * b - 1))


def solve_max_isotropic(bases, dim, order):
    """Weights of the maximally isotropic stencil on the given groups:
    e2 = 1 and every moment up to ``order`` isotropic (Sec. IV)."""
    Ws = sp.symbols(f"w0:{len(bases)}")
    groups = list(zip(bases, Ws))
    vecs = []
    for b, w in groups:
        for v in st.orbit(b):
            vecs.append((v, w))

    def M(idx):
        return sum(w * sp.Integer(_iprod(v[i] for i in idx)) for v, w in vecs)
    eqs = [M((0, 0)) - 1]
    for o in range(4, order + 1, 2):
        ref = tuple([0] * ((o // 2 + 1) // 2 * 2) + [1] * (o // 2 // 2 * 2))
        dref = st.isotropic_tensor_value(ref)
        Mref = M(ref)
        for idx in product(range(dim), repeat=o):
            if list(idx) != sorted(idx):
                continue
            eqs.append(M(idx) * dref - Mref * st.isotropic_tensor_value(idx))
    sol = sp.linsolve(eqs, Ws)
    (vals,) = list(sol)
    assert all(v.free_symbols == set() for v in vals), "not unique"
    return [(b, Fr(int(sp.fraction(v)[0]), int(sp.fraction(v)[1]))) for b, v in zip(bases, vals)]


E_GROUPS_2D = {
    4: [(1, 0), (1, 1)],
    6: [(1, 0), (1, 1), (2, 0)],
    8: [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2)],
    10: [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)],
    12: [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1), (3, 2), (4, 0), (4, 1)],
}
E_GROUPS_3D = {
    4: [(1, 0, 0), (1, 1, 0)],
    6: [(1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 0, 0)],
    8: [(1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 1, 0), (2, 1, 1), (2, 2, 0)],
}


# --- velocity sets (Sec. II) --------------------------------------------------
def _extract_velocity_table(lattice):
    """Recover the oracle C core's velocity vectors and weights by behaviour:
    weights from f_eq at u = 0, vectors by streaming one step with F = 0 and
    a vanishing relaxation rate."""
    D, Q = oracle.LATTICES[lattice]
    shape = (5, 5, 5) if D == 3 else (1, 5, 5)
    o = oracle.Oracle(lattice, shape, L.named_stencil("E4_3D" if D == 3 else "E4_2D").groups,
                      tau=1e300, G=0.0)
    o.init_equilibrium(np.ones(shape))
    w = o.f[:, 0, 0, 0].copy()
    f = np.zeros((Q,) + shape)
    c = (2, 2, 2) if D == 3 else (0, 2, 2)
    for i in range(Q):
        f[(i,) + c] = 1.0 + i
    o.set_state(f)
    o.step(1)
    vecs = []
    for i in range(Q):
        loc = np.argwhere(np.abs(o.f[i] - (1.0 + i)) < 1e-12)
        assert len(loc) == 1
        d = loc[0] - np.array(c)
        vecs.append(tuple(int(v) for v in d[::-1][:D]))  # (x, y[, z])
    return w, vecs


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_velocity_set_isotropy(lattice):
    D, Q = oracle.LATTICES[lattice]
    w, vecs = _extract_velocity_table(lattice)
    table = oracle.C9 if D == 2 else oracle.C19
    assert [tuple(v) for v in table.tolist()] == vecs
    exact = {0: Fr(4, 9), 1: Fr(1, 9), 2: Fr(1, 36)} if Q == 9 else \
        {0: Fr(1, 3), 1: Fr(1, 18), 2: Fr(1, 36)}
    W = [exact[sum(abs(c) for c in v)] for v in vecs]
    assert np.array_equal(w, np.array([float(x) for x in W]))
    # <1> = 1, <xi xi> = c_s^2 delta, <xi^4> = c_s^4 Delta, odd moments 0
    for order in range(0, 6):
        for idx in product(range(D), repeat=order):
            m = sum(Wi * _iprod(v[k] for k in idx) for Wi, v in zip(W, vecs))
            if order % 2:
                assert m == 0
            else:
                assert m == Fr(1, 3) ** (order // 2) * st.isotropic_tensor_value(idx) \
                    or order > 4
    assert sum(W) == 1


# --- group expansion and maximal isotropy (Table tab:e2n_values) --------------
def test_orbit_sizes():
    sizes = {(1, 0): 4, (1, 1): 4, (2, 1): 8, (3, 3): 4, (1, 0, 0): 6, (1, 1, 0): 12,
             (1, 1, 1): 8, (2, 1, 0): 24, (2, 1, 1): 24, (2, 2, 1): 24, (3, 0, 0): 6,
             (2, 2, 0): 12, (4, 0, 0): 6, (3, 3, 0): 12}
    for b, n in sizes.items():
        assert len(st.orbit(b)) == n
    pairs = st.canonical_pairs(L.E8_3D.groups)
    assert len(pairs) == 46
    assert len({v for v, _ in pairs}) == 46
    assert all(tuple(-c for c in v) not in {u for u, _ in pairs} for v, _ in pairs)


@pytest.mark.parametrize("order", [4, 6, 8, 10, 12])
def test_max_isotropic_2d_matches_table(order):
    tab = G.e2n_values()
    col = [4, 6, 8, 10, 12].index(order)
    W = solve_max_isotropic(E_GROUPS_2D[order], 2, order)
    assert st.n_vectors(W) == tab["Ne2"][col]
    for n in (2, 3, 4, 5, 6):
        assert e2n_table_convention(W, 2, n) == tab[f"e{2 * n}"][col]
    assert st.moment(W, [2, 0]) == 1


@pytest.mark.parametrize("order", [4, 6, 8])
def test_max_isotropic_3d_matches_table(order):
    tab = G.e2n_values()
    col = [4, 6, 8].index(order)
    W = solve_max_isotropic(E_GROUPS_3D[order], 3, order)
    assert st.n_vectors(W) == tab["Ne3"][col]
    for n in (2, 3, 4, 5, 6):
        assert e2n_table_convention(W, 3, n) == tab[f"e{2 * n}"][col]


def test_named_stencils_are_the_max_isotropic_ones():
    sc = G.scalars()
    W4 = solve_max_isotropic(E_GROUPS_2D[4], 2, 4)
    assert [w for _, w in W4] == sc["W_E4_2D"] == L.E4_2D.weights_exact
    W8 = solve_max_isotropic(E_GROUPS_2D[8], 2, 8)
    assert [w for _, w in W8] == sc["W_E8_2D"] == L.E8_2D.weights_exact
    assert solve_max_isotropic(E_GROUPS_2D[6], 2, 6) == L.E6_2D.groups
    assert solve_max_isotropic(E_GROUPS_3D[4], 3, 4) == L.E4_3D.groups
    assert solve_max_isotropic(E_GROUPS_3D[8], 3, 8) == L.E8_3D.groups


# --- Table tab:defe2nI2n ------------------------------------------------------
def _unit(dim, key):
    b = (G.GROUPS2 if dim == 2 else G.GROUPS3)[key]
    return [(b, Fr(1))]


def test_defe2nI2n_2d_rows():
    rows = G.defe2nI2n()
    for key in G.GROUPS2:
        g = _unit(2, key)
        e2, e4, e6, e8 = st.isotropy_coeffs(g, 2)
        an = st.anisotropy_2d(g)
        got = {"e2": e2, "e4": e4, "e6": e6, "e8": e8, **an}
        for name in ("e2", "e4", "e6", "e8", "I40", "I60", "I80", "I81"):
            row = rows[(2, name)]
            if key == "16" and name not in ("e2", "e4", "e6", "e8"):
                continue  # the 2D anisotropy rows of the table omit the (4,0) group
            assert got[name] == row.get(key, Fr(0)), (name, key)


def _monomials(order):
    """Sorted exponent tuples (a >= b >= c, all even) of total degree ``order``."""
    out = []
    for a in range(order, -1, -2):
        for b in range(min(a, order - a), -1, -2):
            c = order - a - b
            if c <= b and c % 2 == 0:
                out.append((a, b, c))
    return out


@pytest.mark.parametrize("name,order", [("I40", 4), ("I60", 6), ("I61", 6), ("I80", 8),
                                        ("I81", 8), ("I82", 8), ("I100", 10),
                                        ("I101", 10), ("I102", 10)])
def test_defe2nI2n_3d_rows_are_isotropy_conditions(name, order):
    """Every 3D row of the table must be one fixed linear combination of the
    raw moments of its order (the same across all eleven groups) that
    vanishes on the isotropic tensor: the oracle's moments reproduce the
    printed coefficients of all groups."""
    row = G.defe2nI2n()[(3, name)]
    mons = _monomials(order)
    keys = list(G.GROUPS3)
    A = sp.Matrix([[st.moment(_unit(3, k), list(m)) for m in mons] for k in keys])
    y = sp.Matrix([row.get(k, Fr(0)) for k in keys])
    sol, params = A.gauss_jordan_solve(y)
    sol = sol.subs({p: 0 for p in params})
    assert A * sol == y
    iso = sum(c * st.isotropic_tensor_value([0] * m[0] + [1] * m[1] + [2] * m[2])
              for c, m in zip(sol, mons))
    assert iso == 0


# --- tuned stencil tables ------------------------------------------------------
def _rand_fr(rng):
    return Fr(rng.randint(-60, 60), rng.randint(1, 97))


def test_table_e4_tuning_6():
    rng = random.Random(1)
    for dim in (2, 3):
        for _ in range(3):
            s0 = _rand_fr(rng)
            S = L.stencil_e4_tuning_6(dim, s0)
            assert st.moment(S.groups, [2] + [0] * (dim - 1)) == 1
            assert st.isotropy_residual(S.groups, dim, 4) == 0
            assert st.isotropy_residual(S.groups, dim, 6) == 0
            assert st.isotropy_coeffs(S.groups, dim)[1] == -2 * s0
    # e4 = 2/5 gives the E6 weights (caption of the table)
    S = L.stencil_e4_tuning_6(2, Fr(-1, 5))
    assert {b: w for b, w in S.groups if w} == dict(L.E6_2D.groups)
    assert st.n_vectors(L.stencil_e4_tuning_6(2, 1).groups) == 16
    assert st.n_vectors(L.stencil_e4_tuning_6(3, 1).groups) == 44


def test_table_e4e6_tuning_8():
    rng = random.Random(2)
    for dim, ne in ((2, 32), (3, 140)):
        for _ in range(2):
            s0, s1 = _rand_fr(rng), _rand_fr(rng)
            S = L.stencil_e4e6_tuning_8(dim, s0, s1)
            assert st.n_vectors(S.groups) == ne
            assert st.moment(S.groups, [2] + [0] * (dim - 1)) == 1
            for o in (4, 6, 8):
                assert st.isotropy_residual(S.groups, dim, o) == 0
            e2, e4, e6, _ = st.isotropy_coeffs(S.groups, dim)
            assert e4 == -2 * s0 and e6 == 4 * s1    # eq. hatsigma01eI


def project_3d_to_2d(groups3):
    """eq. wproj: 2D weights of the x-y projection of a 3D stencil."""
    w = {}
    for v, wt in st.full_vectors(groups3):
        if True:
            key = (v[0], v[1])
            w[key] = w.get(key, Fr(0)) + wt
    out = {}
    for (x, y), wt in w.items():
        if (x, y) == (0, 0):
            continue
        b = tuple(sorted((abs(x), abs(y)), reverse=True))
        if b in out:
            assert out[b] == wt
        out[b] = wt
    return [(b, wt) for b, wt in out.items() if wt != 0]


def cmn_from_table(groups2):
    rows = G.cmn_coeffs()
    by_sq = {}
    for b, w in groups2:
        by_sq[str(sum(c * c for c in b))] = w
    return {name: sum(coef * by_sq.get(k, Fr(0)) for k, coef in row.items())
            for name, row in rows.items()}


def test_wproj_e8_and_tuning_6():
    assert sorted(project_3d_to_2d(L.E8_3D.groups)) == sorted(L.E8_2D.groups)
    s0 = Fr(-3, 7)
    p = dict(project_3d_to_2d(L.stencil_e4_tuning_6(3, s0).groups))
    q = {b: w for b, w in L.stencil_e4_tuning_6(2, s0).groups if w}
    assert p == q


def test_wproj_matches_printed_rows():
    """The printed projection rules of eq. wproj hold for random 3D weights."""
    rng = random.Random(5)
    W3 = {k: _rand_fr(rng) for k in G.GROUPS3}
    groups3 = [(G.GROUPS3[k], W3[k]) for k in G.GROUPS3]
    p = dict(project_3d_to_2d(groups3))
    w2 = lambda b: p.get(b, Fr(0))
    assert w2((1, 0)) == W3["1"] + 2 * W3["2"] + 2 * W3["5"]
    assert w2((1, 1)) == W3["2"] + 2 * W3["3"] + 2 * W3["6"]
    assert w2((2, 0)) == W3["4"] + 2 * W3["5"] + 2 * W3["8"]
    assert w2((2, 1)) == W3["5"] + 2 * W3["6"] + 2 * W3["9a"]
    assert w2((2, 2)) == W3["8"] + 2 * W3["9a"]
    assert w2((3, 0)) == W3["9"] + 2 * W3["18"]
    assert w2((4, 0)) == W3["16"]
    assert w2((3, 3)) == W3["18"]


def test_table_e4e6e8_tuning_6_knobs():
    """Tables tab:e4e6e8_tuning_6_2d/3d: 6th-order isotropy, e2 = 1, and the
    three knobs recovered from the c_mn of Table tab:pn_minus_ptcoeffs
    (sigma0 = c11 - c02, sigma1 = c22 - c13 + c04, delta0 = c02) and from
    eqs. hatsigma01eI / hatdelta0eI."""
    rng = random.Random(3)
    for dim in (2, 3):
        for _ in range(3):
            s0, s1, d0 = _rand_fr(rng), _rand_fr(rng), _rand_fr(rng)
            S = L.stencil_e4e6e8_tuning_6(dim, s0, s1, d0)
            assert st.moment(S.groups, [2] + [0] * (dim - 1)) == 1
            assert st.isotropy_residual(S.groups, dim, 4) == 0
            assert st.isotropy_residual(S.groups, dim, 6) == 0
            g2 = S.groups if dim == 2 else project_3d_to_2d(S.groups)
            c = cmn_from_table(g2)
            assert c["c11"] - c["c02"] == s0
            assert c["c22"] - c["c13"] + c["c04"] == s1
            assert c["c02"] == d0
            e2, e4, e6, e8 = st.isotropy_coeffs(S.groups, dim)
            assert e4 == -2 * s0 and e6 == 4 * s1
            assert d0 == Fr(1, 12) + Fr(95, 432) * e4 + Fr(7, 72) * e6 - Fr(5, 144) * e8


def test_delta0_tuning_leaves_1d_projection_unchanged():
    """Flat-interface invariance under delta0_hat (Sec. V C): for a profile
    along x only the vectors with e_x != 0 act, and their weights summed over
    vectors with the same e_x do not depend on delta0_hat.  This holds for the
    two-dimensional table (the paper's flat runs); the 3D table's (4,0,0)
    weight moves with delta0_hat, so its projection is not invariant."""
    for dim in (2,):
        def proj(d0):
            S = L.stencil_e4e6e8_tuning_6(dim, Fr(-2, 5), Fr(1, 9), d0)
            a = {}
            for v, w in st.full_vectors(S.groups):
                if v[0]:
                    a[v[0]] = a.get(v[0], Fr(0)) + w
            return a
        assert proj(Fr(1, 3)) == proj(Fr(-7, 5))


def test_delta0_reference_value():
    """Sec. V D reference delta0_hat = 7 sqrt5/225 + 32/135 is eq. hatdelta0eI at
    e4 = 4/5, e6 = e4^(3/2), e8 = e4^2."""
    sc = G.scalars()
    e4 = 0.8
    d0 = 1 / 12 + 95 * e4 / 432 + 7 * e4 ** 1.5 / 72 - 5 * e4 ** 2 / 144
    assert abs(d0 - (7 * 5 ** 0.5 / 225 + 32 / 135)) < 1e-15
    assert abs(d0 - sc["delta0_ref"][0]) < 5e-4


def test_epsilon_of_e4():
    from oracle.analysis import epsilon_of_e4
    sc = G.scalars()
    assert abs(epsilon_of_e4(0.8) - float(sc["eps_e4_4_5"][0])) < 1e-15
    assert epsilon_of_e4(1 / 3) == 0.0
    assert abs(epsilon_of_e4(4 / 7) - 10 / 31) < 1e-15


def test_sigma0_hat_is_minus_e4_over_2():
    """eq. hat_sigma_0_moments: c11 - c02 = -I40/4 - e4/2 for any 2D weights."""
    rng = random.Random(9)
    keys = ["1", "2", "4", "5", "8", "9", "16"]
    for _ in range(4):
        groups = [(G.GROUPS2[k], _rand_fr(rng)) for k in keys]
        c = cmn_from_table(groups)
        e4 = st.isotropy_coeffs(groups, 2)[1]
        I40 = st.anisotropy_2d(groups)["I40"]
        assert c["c11"] - c["c02"] == -I40 / 4 - e4 / 2


def test_multirange_sixth_order_weights():
    """Appendix B: the improved multirange stencil is 4th- and 6th-order
    isotropic with e2 = 1 + 2 g and e4 = (1 + 8 g)/3 for every g."""
    for g in (Fr(0), Fr(1, 3), Fr(-2, 7)):
        S = [((1, 0), Fr(14, 45) - 32 * g / 45), ((1, 1), 16 * g / 45 + Fr(17, 180)),
             ((2, 0), 19 * g / 90 + Fr(1, 720)), ((2, 2), 7 * g / 360 - Fr(1, 1440))]
        assert st.anisotropy_2d(S)["I40"] == 0 and st.anisotropy_2d(S)["I60"] == 0
        e2, e4, _, _ = st.isotropy_coeffs(S, 2)
        assert e2 == 1 + 2 * g and e4 == (1 + 8 * g) / 3


def test_cmn_from_1d_pressure_tensor_taylor():
    """Table tab:pn_minus_ptcoeffs follows from eq. 1dPNT with the
    coefficients of Table tab:pnptcoeffs by Taylor expansion."""
    keys = ["1", "2", "4", "5", "8", "9", "16", "18"]
    Wsym = {k: sp.Symbol(f"W{k}") for k in keys}
    d = sp.symbols("p0:6")   # psi and its derivatives at x

    def shift(s):
        return sum(d[m] * sp.Rational(s) ** m / sp.factorial(m) for m in range(6))

    rows = G.pnpt_coeffs()

    def coef(comp, term):
        return sum(sp.Rational(c.numerator, c.denominator) * Wsym[k]
                   for k, c in rows[(comp, term)].items())

    def P(comp):
        e = 0
        for k, t in ((4, "a4"), (3, "a3"), (2, "a2"), (1, "a1")):
            e += coef(comp, t) * d[0] * (shift(k) + shift(-k))
        e += coef(comp, "a0") * d[0] ** 2
        e += coef(comp, "b22") * shift(2) * shift(-2)
        e += coef(comp, "b11") * shift(1) * shift(-1)
        e += coef(comp, "b13") * (shift(3) * shift(-1) + shift(1) * shift(-3))
        e += coef(comp, "b12") * (shift(2) * shift(-1) + shift(1) * shift(-2))
        return e
    diff = sp.expand(P("N") - P("T"))
    poly = sp.Poly(diff, *d)
    got = {}
    for (m, n) in ((0, 2), (1, 1), (0, 4), (1, 3), (2, 2)):
        mono = [0] * 6
        mono[m] += 1
        mono[n] += 1
        got[f"c{m}{n}"] = sp.expand(poly.coeff_monomial(tuple(mono)))
    assert sp.expand(poly.coeff_monomial((2, 0, 0, 0, 0, 0))) == 0   # bulk: P_N = P_T
    for name, row in G.cmn_coeffs().items():
        want = sum(sp.Rational(c.numerator, c.denominator) * Wsym[k] for k, c in row.items())
        assert sp.expand(got[name] - want) == 0, name
