"""The register DFT codelets of the data-consistency kernels (csrc/dft_reg.cuh) compiled as host
code and checked against a direct double-precision DFT for every length the kernels use (both
directions), and their compile-time roots against the C library's cos/sin."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1411_6206_gb300", "csrc")
LENGTHS = [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 16, 18, 20, 24, 28, 32]

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include "dft_reg.cuh"
using namespace lps::dftr;
template <int N, bool INV> void run(const double* re, const double* im) {
  float2 v[N];
  for (int i = 0; i < N; ++i) { v[i].x = (float)re[i]; v[i].y = (float)im[i]; }
  dft<N, INV>(v);
  printf("%d %d", N, (int)INV);
  for (int i = 0; i < N; ++i) printf(" %.9e %.9e", v[i].x, v[i].y);
  printf("\n");
}
template <int N> void roots() {
  constexpr Roots<N> R{};
  double e = 0;
  for (int j = 0; j < N; ++j) {
    e = fmax(e, fabs(R.c[j] - cos(2.0 * M_PI * j / N)));
    e = fmax(e, fabs(R.s[j] - sin(2.0 * M_PI * j / N)));
  }
  printf("roots %d %.3e\n", N, e);
}
int main() {
  double re[32], im[32];
  for (int i = 0; i < 32; ++i) { re[i] = std::sin(1.3 * i + 0.2) + 0.1 * i; im[i] = std::cos(0.7 * i * i + 0.4); }
#define BOTH(N) run<N, false>(re, im); run<N, true>(re, im); roots<N>();
  BOTH(2) BOTH(3) BOTH(4) BOTH(5) BOTH(6) BOTH(7) BOTH(8) BOTH(9) BOTH(10) BOTH(12) BOTH(14) BOTH(16)
  BOTH(18) BOTH(20) BOTH(24) BOTH(28) BOTH(32)
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_codelets_match_direct_dft(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "dft_host.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "dft_host"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", f"-I{CSRC}", str(src), "-o", str(exe)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.splitlines()
    i = np.arange(32)
    x = (np.sin(1.3 * i + 0.2) + 0.1 * i + 1j * np.cos(0.7 * i * i + 0.4)).astype(np.complex64).astype(complex)
    seen = set()
    for line in out:
        f = line.split()
        if f[0] == "roots":
            assert float(f[2]) < 6e-8, line     # float rounding of the exact root
            continue
        n, inv = int(f[0]), int(f[1])
        got = np.array([float(a) + 1j * float(b) for a, b in zip(f[2::2], f[3::2])])
        k = np.arange(n)
        W = np.exp((2j if inv else -2j) * np.pi * np.outer(k, k) / n)
        ref = W @ x[:n]
        assert np.linalg.norm(got - ref) < 2e-6 * np.linalg.norm(ref), (n, inv)
        seen.add((n, inv))
    assert seen == {(n, v) for n in LENGTHS for v in (0, 1)}
