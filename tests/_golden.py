"""Readers for the text fixtures under tests/golden/ (values the paper prints)."""
import os
from fractions import Fraction as Fr

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line


def e2n_values():
    rows = {}
    for line in _lines("e2n_values.txt"):
        k, *vals = line.split()
        rows[k] = [Fr(v) for v in vals]
    return rows


def _pairs(tokens):
    out = {}
    for t in tokens:
        g, c = t.split(":")
        out[g] = Fr(c)
    return out


def defe2nI2n():
    rows = {}
    for line in _lines("defe2nI2n.txt"):
        d, name, *rest = line.split()
        rows[(int(d), name)] = _pairs(rest)
    return rows


def pnpt_coeffs():
    rows = {}
    for line in _lines("pnpt_coeffs.txt"):
        comp, term, *rest = line.split()
        rows[(comp, term)] = _pairs(rest)
    return rows


def cmn_coeffs():
    rows = {}
    for line in _lines("cmn_coeffs.txt"):
        name, *rest = line.split()
        rows[name] = _pairs(rest)
    return rows


def scalars():
    out = {}
    for line in _lines("paper_scalars.txt"):
        k, v = [s.strip() for s in line.split("=", 1)]
        vals = v.split()
        out[k] = [Fr(x) if "/" in x or x.lstrip("-").isdigit() else float(x) for x in vals]
    return out


GROUPS2 = {"1": (1, 0), "2": (1, 1), "4": (2, 0), "5": (2, 1), "8": (2, 2),
           "9": (3, 0), "16": (4, 0), "18": (3, 3)}
GROUPS3 = {"1": (1, 0, 0), "2": (1, 1, 0), "3": (1, 1, 1), "4": (2, 0, 0),
           "5": (2, 1, 0), "6": (2, 1, 1), "8": (2, 2, 0), "9a": (2, 2, 1),
           "9": (3, 0, 0), "16": (4, 0, 0), "18": (3, 3, 0)}
