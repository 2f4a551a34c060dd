"""The binary64 exp and pow of the library (csrc/expcr.cuh) on the host.

The header's device code is compiled here as plain C++ (g++, contraction
off), with the CUDA rounding intrinsics replaced by the IEEE operations they
name, and checked against 200-bit mpmath evaluations rounded once:

* the quick phases (exp_quick, pow_quick): whenever they certify a result,
  it is the correctly rounded value; they decline at most a few percent of
  the arguments;
* the double-double phases (exp_dd_cr, and log_dd + exp_dd_cr for the
  power) return the correctly rounded value for every argument.

Arguments: exp(-1/n) over the densities the steps see and beyond, and the
psi_eps powers (n/(eps + n))^(1/eps) for the paper's eps values and
others, plus random bases and exponents.  No GPU is needed.
"""
import os
import random
import shutil
import subprocess

import pytest

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2505_23647_gb300", "csrc", "expcr.cuh")

SHIMS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#define __device__
#define __forceinline__ inline
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline long long __double_as_longlong(double x) { long long v; std::memcpy(&v, &x, 8); return v; }
static inline double __longlong_as_double(long long v) { double x; std::memcpy(&x, &v, 8); return x; }
static inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) {
    unsigned long long o = *p; *p += v; return o;
}
"""

MAIN = r"""
using namespace sclbm;
int main(int argc, char **argv) {
    FILE *in = std::fopen(argv[1], "r");
    char kind;
    double a, b;
    while (std::fscanf(in, " %c %la %la", &kind, &a, &b) == 3) {
        double q = 0.0, full;
        bool ok;
        if (kind == 'e') {
            ok = exp_quick(a, &q);
            full = exp_dd_cr(ddv{a, 0.0}, 0x1p-97, nullptr);
        } else {
            ok = pow_quick(a, b, &q);
            const ddv y = dd_mul(log_dd(a), ddv{b, 0.0});
            full = exp_dd_cr(y, 0x1p-97 + std::fabs(y.hi) * 0x1p-98, nullptr);
        }
        std::printf("%d %a %a\n", ok ? 1 : 0, q, full);
    }
    return 0;
}
"""


def _cases():
    rng = random.Random(2505)
    cases = []
    for _ in range(6000):
        n = rng.uniform(0.02, 6.0)
        cases.append(("e", -1.0 / n, 0.0))
    for _ in range(3000):
        cases.append(("e", rng.uniform(-700.0, 700.0), 0.0))
    for eps in (14.0 / 29.0, 10.0 / 31.0, 0.25, 2.0):
        e = 1.0 / eps
        for _ in range(1500):
            n = rng.uniform(0.02, 6.0)
            cases.append(("p", n / (eps + n), e))
    for _ in range(3000):
        cases.append(("p", rng.uniform(1e-6, 1.0), rng.uniform(0.1, 20.0)))
    cases += [("e", 0.0, 0.0), ("e", -1e-300, 0.0), ("p", 0.5, 2.0), ("p", 0.999999999999, 3.1)]
    return cases


def _exact(kind, a, b):
    mpmath.mp.prec = 200
    v = mpmath.exp(mpmath.mpf(a)) if kind == "e" else mpmath.power(mpmath.mpf(a), mpmath.mpf(b))
    return float(v)   # nearest binary64


def test_quick_and_double_double_phases_round_correctly(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("needs g++")
    header = open(HEADER).read().replace("#include <cuda_runtime.h>", "")
    src = tmp_path / "expcr_host.cpp"
    src.write_text(SHIMS + header + MAIN)
    exe = tmp_path / "expcr_host"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off", str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    cases = _cases()
    args = tmp_path / "args.txt"
    args.write_text("\n".join(f"{k} {float.hex(a)} {float.hex(b)}" for k, a, b in cases))
    out = subprocess.run([str(exe), str(args)], capture_output=True, text=True, check=True)
    lines = out.stdout.split("\n")
    declined = {"e": 0, "p": 0}
    total = {"e": 0, "p": 0}
    for (kind, a, b), line in zip(cases, lines):
        ok, q, full = line.split()
        want = _exact(kind, a, b)
        total[kind] += 1
        assert float.fromhex(full) == want, (kind, a, b, full, want)
        if ok == "1":
            assert float.fromhex(q) == want, (kind, a, b, q, want)
        else:
            declined[kind] += 1
    assert len(lines) >= len(cases)
    for k in ("e", "p"):
        assert declined[k] < 0.05 * total[k], (k, declined[k], total[k])
