"""The library's band intensities (mcrt_set_kdist with B = NULL) against the
input generator's Planck function, on the CPU.

The host function of csrc/planck.h is compiled here with the host C++ compiler
and evaluated on the benchmark's 40 bands of 200 1/cm and on T nodes from 0 K to
4000 K; both sides evaluate the same closed form in binary64 (Section 2.2's
band-centre intensity), so they agree to a few units in the last place, and both
give exactly 0 at 0 K and where exp(h c nu / k T) overflows.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1810_00188_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_planck_table_matches_the_generator(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    nu_c = 200.0 + 200.0 * np.arange(40)
    dnu = np.full(40, 200.0)
    T = np.concatenate([[0.0, 1.0, 20.0], np.linspace(50.0, 4000.0, 80)])
    src = tmp_path / "planck.cpp"
    src.write_text(
        '#include <cstdio>\n#include "planck.h"\n'
        "int main() {\n  double nu, dnu, t;\n"
        '  while (std::scanf("%lf %lf %lf", &nu, &dnu, &t) == 3)\n'
        '    std::printf("%.17g\\n", mcrt::planck_band(nu, dnu, t));\n  return 0;\n}\n')
    exe = tmp_path / "planck"
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1810_00188_gb300", "csrc"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    rows = [(n, d, t) for n, d in zip(nu_c, dnu) for t in T]
    stdin = "\n".join(f"{float(n)!r} {float(d)!r} {float(t)!r}" for n, d, t in rows) + "\n"
    out = subprocess.run([str(exe)], input=stdin, capture_output=True, text=True, check=True).stdout
    lib = np.array([float(v) for v in out.split()]).reshape(len(nu_c), len(T))
    ref = inputs.planck_band_intensity(nu_c, dnu, T)
    assert np.all(lib[:, 0] == 0.0) and np.all(ref[:, 0] == 0.0)
    assert np.array_equal(lib == 0.0, ref == 0.0)  # the same underflow pattern
    nz = ref > 0.0
    assert np.all(np.abs(lib[nz] - ref[nz]) <= 8 * np.finfo(float).eps * ref[nz])
    # the band sum is close to sigma T^4 / pi at 1000 K (the bands cover most of the spectrum)
    sigma = 5.670374419e-8
    k1000 = int(np.argmin(np.abs(T - 1000.0)))
    assert lib[:, k1000].sum() == pytest.approx(sigma * T[k1000] ** 4 / np.pi, rel=0.02)
