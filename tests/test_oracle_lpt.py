"""Pins of the oracle's lattice pressure tensor (Appendices E and F):

* the irregular terms printed in the appendices, transcribed literally, and
  the regular-group formulas written out group by group, agree with the
  oracle's per-group rule on random fields;
* the one-dimensional projection equals eq. 1dPNT with the coefficients of
  Table tab:pnptcoeffs (3D weights projected by eq. wproj);
* the bulk limit is (n c_s^2 + G' e2 psi^2 / 2) delta (end of Appendix E).
"""
from fractions import Fraction as Fr
import os
import random

import numpy as np
import pytest

import oracle
from oracle import stencil as st
from tests import _golden as G


def _rows():
    out = []
    with open(os.path.join(G.GOLDEN, "lpt_irregular.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, pairs = line.split(":")
            dim, grp, div, vec = head.split()
            e = tuple(int(c) for c in vec.split(","))
            ps = []
            for p in pairs.split():
                a, b = p.split("|")
                ps.append((tuple(int(c) for c in a.split(",")),
                           tuple(int(c) for c in b.split(","))))
            out.append((int(dim), grp, int(div), e, ps))
    return out


def test_printed_irregular_pairs_match_their_vectors():
    bad = []
    for dim, grp, div, e, ps in _rows():
        for a, b in ps:
            if tuple(bb - aa for aa, bb in zip(a, b)) != e:
                bad.append((dim, grp, e, a, b))
    assert bad == [(3, "9a", (2, 2, -1), (-1, -1, 1), (-1, 1, 0))]


def _corrected_rows():
    rows = []
    for dim, grp, div, e, ps in _rows():
        ps = [(a, b) if tuple(bb - aa for aa, bb in zip(a, b)) == e
              else (a, tuple(aa + ee for aa, ee in zip(a, e))) for a, b in ps]
        rows.append((dim, grp, div, e, ps))
    return rows


def _at(field, off):
    """field evaluated at x + off (periodic), field shaped (nz, ny, nx)."""
    off = tuple(off) + (0,) * (3 - len(off))
    return np.roll(field, shift=(-off[2], -off[1], -off[0]), axis=(0, 1, 2))


def literal_lpt(dim, n, psi, groups, Gp):
    """Appendices E/F written out group by group (regular groups by their
    printed formulas, irregular b-parts from the transcribed rows)."""
    comps = [(0, 0), (0, 1), (1, 1)] if dim == 2 else \
        [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    P = [np.where(True, 0.0, 0.0) + (n / 3.0 if a == b else 0.0 * n) for a, b in comps]
    rows = _corrected_rows()
    for base, W in groups:
        W = float(W)
        sq = sum(c * c for c in base)
        mags = sorted((abs(c) for c in base if c), reverse=True)
        regular = len(set(mags)) == 1
        vecs = st.orbit(base)
        for e in vecs:
            ee = [e[a] * e[b] for a, b in comps]
            if regular:
                m = mags[0]
                h = tuple(c // m for c in e)
                term = {1: (Gp / 2) * psi * _at(psi, e)}.get(m)
                if m == 2:
                    term = (Gp / 4) * psi * _at(psi, e) + (Gp / 4) * _at(psi, h) * _at(psi, tuple(-c for c in h))
                elif m == 3:
                    term = (Gp / 6) * psi * _at(psi, e) + (Gp / 3) * _at(psi, h) * _at(psi, tuple(-2 * c for c in h))
                elif m == 4:
                    term = (Gp / 8) * psi * _at(psi, e) \
                        + (Gp / 4) * _at(psi, h) * _at(psi, tuple(-3 * c for c in h)) \
                        + (Gp / 8) * _at(psi, tuple(2 * c for c in h)) * _at(psi, tuple(-2 * c for c in h))
            else:
                term = (Gp / 4) * psi * _at(psi, e)
            for k in range(len(comps)):
                P[k] = P[k] + W * ee[k] * term
        if not regular:
            key = {5: "5", 6: "6", 9: "9a"}[sq]
            for d, grp, div, e, ps in rows:
                if d != dim or grp != key:
                    continue
                ee = [e[a] * e[b] for a, b in comps]
                s = sum(_at(psi, a) * _at(psi, b) for a, b in ps)
                for k in range(len(comps)):
                    P[k] = P[k] + (Gp / div) * W * ee[k] * s
    return np.array(P)


ALL2 = [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 3), (4, 0)]
ALL3 = list(G.GROUPS3.values())


@pytest.mark.parametrize("dim", [2, 3])
def test_oracle_matches_printed_appendix_formulas(dim):
    rng = np.random.default_rng(11)
    shape = (1, 7, 9) if dim == 2 else (5, 6, 7)
    n = 0.5 + rng.random(shape)
    psi = 0.2 + 0.6 * rng.random(shape)
    groups = [(b, Fr(int(rng.integers(1, 50)), int(rng.integers(51, 400))))
              for b in (ALL2 if dim == 2 else ALL3)]
    Gp = -2.7
    lat = "D2Q9" if dim == 2 else "D3Q19"
    got = oracle.pressure_tensor_from_fields(lat, n, psi, groups, Gp)
    want = literal_lpt(dim, n, psi, groups, Gp)
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
    # per group as well (catches compensating errors)
    for g in groups:
        got = oracle.pressure_tensor_from_fields(lat, n, psi, [g], Gp)
        want = literal_lpt(dim, n, psi, [g], Gp)
        assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want)), g


def _pnpt_1d(psi1, W2, Gp):
    """eq. 1dPNT with Table tab:pnptcoeffs for a profile psi(x)."""
    rows = G.pnpt_coeffs()
    by = {str(sum(c * c for c in b)): w for b, w in W2}

    def c(comp, term):
        return float(sum(coef * by.get(k, Fr(0)) for k, coef in rows[(comp, term)].items()))
    s = lambda k: np.roll(psi1, -k)
    out = {}
    for comp in ("N", "T"):
        P = np.zeros_like(psi1)
        for k, t in ((4, "a4"), (3, "a3"), (2, "a2"), (1, "a1")):
            P += c(comp, t) * psi1 * (s(k) + s(-k))
        P += c(comp, "a0") * psi1 ** 2
        P += c(comp, "b22") * s(2) * s(-2)
        P += c(comp, "b11") * s(1) * s(-1)
        P += c(comp, "b13") * (s(3) * s(-1) + s(1) * s(-3))
        P += c(comp, "b12") * (s(2) * s(-1) + s(1) * s(-2))
        out[comp] = Gp * P
    return out


def _project(groups3):
    w = {}
    for v, wt in st.full_vectors(groups3):
        w[(v[0], v[1])] = w.get((v[0], v[1]), Fr(0)) + wt
    out = {}
    for (x, y), wt in w.items():
        if (x, y) != (0, 0):
            out[tuple(sorted((abs(x), abs(y)), reverse=True))] = wt
    return list(out.items())


@pytest.mark.parametrize("dim", [2, 3])
def test_one_dimensional_projection_matches_1dPNT(dim):
    rng = np.random.default_rng(5)
    nx = 17
    psi1 = 0.1 + 0.8 * rng.random(nx)
    shape = (1, 3, nx) if dim == 2 else (4, 3, nx)
    psi = np.broadcast_to(psi1, shape).copy()
    n = np.full(shape, 1.3)
    groups = [(b, Fr(int(rng.integers(-40, 40)), int(rng.integers(50, 300))))
              for b in (ALL2 if dim == 2 else ALL3)]
    W2 = groups if dim == 2 else _project(groups)
    Gp = -1.9
    P = oracle.pressure_tensor_from_fields("D2Q9" if dim == 2 else "D3Q19", n, psi, groups, Gp)
    ref = _pnpt_1d(psi1, W2, Gp)
    PN = P[0] - n / 3.0
    PT = P[2 if dim == 2 else 3] - n / 3.0
    scale = np.max(np.abs(ref["N"])) + np.max(np.abs(ref["T"]))
    assert np.max(np.abs(PN - ref["N"])) < 1e-13 * scale
    assert np.max(np.abs(PT - ref["T"])) < 1e-13 * scale
    if dim == 3:
        assert np.max(np.abs(P[5] - P[3])) < 1e-13 * scale       # P_zz = P_yy
    assert np.max(np.abs(P[1])) < 1e-13 * scale                  # no shear


@pytest.mark.parametrize("dim", [2, 3])
def test_bulk_limit(dim):
    """Uniform fields: P = (n c_s^2 + G' e2 psi^2 / 2) delta."""
    groups = [(b, Fr(random.Random(k).randint(1, 30), 97)) for k, b in
              enumerate(ALL2 if dim == 2 else ALL3)]
    e2 = float(st.moment(groups, [2] + [0] * (dim - 1)))
    shape = (1, 5, 6) if dim == 2 else (5, 5, 6)
    n = np.full(shape, 1.7)
    psi = np.full(shape, 0.61)
    Gp = -3.1
    P = oracle.pressure_tensor_from_fields("D2Q9" if dim == 2 else "D3Q19", n, psi, groups, Gp)
    pb = 1.7 / 3.0 + 0.5 * Gp * e2 * 0.61 ** 2
    diag = (0, 2) if dim == 2 else (0, 3, 5)
    for k in range(P.shape[0]):
        want = pb if k in diag else 0.0
        assert np.max(np.abs(P[k] - want)) < 1e-14 * abs(pb) * 10
