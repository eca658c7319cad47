"""Host check of the W-step pivot table the slab kernels read (no GPU needed).

The W-step of Eq. (subquKKT) solves, for every run of missing entries of a
row, the tridiagonal block of K_{mu rho2} = (1 + mu) I + rho2 K^T K (K the
first-difference matrix of Eq. (Toeplitz) on n2 entries) restricted to the run.
The library's table builder (wstep_tables, compiled here for the host with the
same flags as the library) must hold the inverse LU pivots of that block by
position in the run: runs starting at j = 0, runs after an observed entry, and
the pivot of a run's last entry when the run ends at j = n2 - 1.  The expected
values are the pivots of plain Gaussian elimination on the dense matrix."""
import subprocess

import numpy as np
import pytest

from paper_2005_09838_gb300 import build

PROG = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "tc_kernels.cuh"
int main(int argc, char** argv) {
  const int n2 = std::atoi(argv[1]);
  const double mu = std::atof(argv[2]), rho2 = std::atof(argv[3]);
  std::vector<double> w(6 * (size_t)n2);
  tc::wstep_tables<double>(w.data(), n2, mu, rho2);
  for (double v : w) std::printf("%.17g\n", v);
  return 0;
}
'''


@pytest.fixture(scope="module")
def table_prog(tmp_path_factory):
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("wtab")
    src = d / "wtab.cu"
    src.write_text(PROG)
    exe = d / "wtab"
    subprocess.run([nvcc, *build.ARCH, "-std=c++17", "--expt-relaxed-constexpr", "-I", build.INCLUDE,
                    "-I", build.CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return exe


def _table(exe, n2, mu, rho2):
    out = subprocess.run([str(exe), str(n2), repr(mu), repr(rho2)], check=True, capture_output=True, text=True)
    return np.array([float(v) for v in out.stdout.split()]).reshape(6, n2)


def _pivots(A):
    """Pivots of Gaussian elimination without pivoting (a tridiagonal SPD block)."""
    u = [A[0, 0]]
    for k in range(1, A.shape[0]):
        u.append(A[k, k] - A[k, k - 1] * A[k - 1, k] / u[-1])
    return np.array(u)


def _kmat(n2, mu, rho2):
    K = np.zeros((max(n2 - 1, 0), n2))
    for i in range(n2 - 1):
        K[i, i], K[i, i + 1] = -1.0, 1.0
    return (1.0 + mu) * np.eye(n2) + rho2 * K.T @ K


@pytest.mark.parametrize("n2", [1, 2, 7, 40])
@pytest.mark.parametrize("mu,rho2", [(1e-3, 1e-1), (0.0, 1.0), (0.5, 3.0)])
def test_table_holds_inverse_lu_pivots_of_the_run_blocks(table_prog, n2, mu, rho2):
    w = _table(table_prog, n2, mu, rho2)
    A = _kmat(n2, mu, rho2)
    # b = 0: a run starting at j = 0 of length L (not reaching the end when L < n2)
    for L in range(1, n2 + 1):
        u = _pivots(A[:L, :L])
        if L < n2:
            np.testing.assert_allclose(w[0, :L], 1.0 / u, rtol=1e-13)       # inv
            np.testing.assert_allclose(w[2, :L], rho2 / u, rtol=1e-13)      # c = rho2 inv
        else:
            np.testing.assert_allclose(w[4, L - 1], 1.0 / u[-1], rtol=1e-13)  # e: the whole row missing
    # b = 1: a run starting at s >= 1 (after an observed entry)
    for s in range(1, n2):
        for L in range(1, n2 - s + 1):
            u = _pivots(A[s:s + L, s:s + L])
            if s + L < n2:
                np.testing.assert_allclose(w[1, :L], 1.0 / u, rtol=1e-13)
                np.testing.assert_allclose(w[3, :L], rho2 / u, rtol=1e-13)
            else:  # the run ends at j = n2 - 1: its last pivot has one neighbour
                np.testing.assert_allclose(w[1, :L - 1], 1.0 / u[:-1], rtol=1e-13)
                np.testing.assert_allclose(w[5, L - 1], 1.0 / u[-1], rtol=1e-13)
