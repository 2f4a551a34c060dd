"""Host logic of the binary32 collision constants (csrc/internal.h,
fill_mass_exact_f32).

The collision conserves n (eqs. lbm, omega_i, f_eq); in binary32 the
constants that carry n through a step must sum to 1 exactly or the lattice
mass drifts by the same amount every step.  For 4000 relaxation times in
(0.5, 3) on D2Q9 and D3Q19 the chosen binary32 constants must satisfy,
exactly in real arithmetic on the binary32 values:

* sum_i w_i = 1 (the two-kernel path);
* keep + sum_c multiplicity_c (omega w)_c = 1 (the fused kernels),

while staying close to what they stand for: each weight within 2.5e-7 and
each omega w within 1e-6 relative, keep within 3.5e-8 of 1 - omega.

The header is compiled here as plain host C++ (g++), no GPU needed.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2505_23647_gb300", "csrc")

HARNESS = r"""
#include "internal.h"
#include <cmath>
#include <cstdio>
int main() {
    int bad_w = 0, bad_fused = 0, bad_close = 0, total = 0;
    for (int Q : {9, 19}) {
        const double w[3] = {Q == 9 ? 4.0 / 9 : 1.0 / 3, Q == 9 ? 1.0 / 9 : 1.0 / 18, 1.0 / 36};
        const int na = Q == 9 ? 4 : 6, m1 = Q == 9 ? 4 : 6, m2 = Q == 9 ? 4 : 12;
        for (int t = 0; t < 4000; ++t) {
            const double tau = 0.5005 + t * (2.5 / 4000.0);
            sclbm::Consts k{};
            k.w[0] = w[0];
            for (int i = 1; i <= na; ++i) k.w[i] = w[1];
            for (int i = na + 1; i < Q; ++i) k.w[i] = w[2];
            k.omega = 1.0 / tau;
            sclbm::fill_mass_exact_f32(k, Q);
            ++total;
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += (double)k.w32[i];
            if (s != 1.0) ++bad_w;
            const double f = (double)k.keep32 + (double)k.omw32[0] + m1 * (double)k.omw32[1] +
                             m2 * (double)k.omw32[2];
            if (f != 1.0) ++bad_fused;
            bool close = std::fabs(k.keep32 - (1.0 - k.omega)) <= 3.5e-8;
            for (int i = 0; i < Q; ++i)
                close = close && std::fabs(k.w32[i] - k.w[i]) <= 2.5e-7 * k.w[i];
            for (int c = 0; c < 3; ++c)
                close = close && std::fabs(k.omw32[c] - k.omega * w[c]) <= 1e-6 * k.omega * w[c];
            if (!close) ++bad_close;
        }
    }
    std::printf("%d %d %d %d\n", total, bad_w, bad_fused, bad_close);
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_binary32_constants_conserve_mass_exactly(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off", "-I", inc, "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    total, bad_w, bad_fused, bad_close = (int(v) for v in out)
    assert total == 8000
    assert bad_w == 0 and bad_fused == 0 and bad_close == 0, out
