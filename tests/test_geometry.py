"""The library's neighbour table (csrc/geometry.h, host code the hop and force
kernels index through) against the oracle's lattice shifts, bit-exact, on the
CPU: g++ builds a small program around the header that writes the tables.

For every half site h of either parity and every direction d, the table
must hold the half-site index of the neighbour that the oracle's
shift(f, mu, +1 / -1) reads, with the half-site layout stated in the header
(n = ((t Z + z) Y + y) X + x, h = n / 2).  Shapes cover extents of 2 (where
n + mu and n - mu coincide), unequal extents and the benchmark lattices.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dwf_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "geometry.h"
int main(int argc, char** argv) {
  const int X = std::atoi(argv[1]), Y = std::atoi(argv[2]), Z = std::atoi(argv[3]), T = std::atoi(argv[4]);
  const long Vh = (long)X * Y * Z * T / 2;
  std::vector<int> nb((size_t)8 * Vh);
  FILE* f = std::fopen(argv[5], "wb");
  for (int par = 0; par < 2; ++par) {
    dwf::build_neighbour_table(X, Y, Z, T, par, nb.data());
    std::fwrite(nb.data(), sizeof(int), nb.size(), f);
  }
  std::fclose(f);
  return 0;
}
"""


@pytest.fixture(scope="module")
def table_program(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("geo")
    src, exe = d / "nb.cpp", d / "nb"
    src.write_text(_PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-I",
                    os.path.join(ROOT, "paper_1111_5059_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)

    def tables(dims):
        out = d / ("nb_%d_%d_%d_%d.bin" % dims)
        subprocess.run([str(exe)] + [str(v) for v in dims] + [str(out)], check=True)
        Vh = int(np.prod(dims)) // 2
        return np.fromfile(out, dtype=np.int32).reshape(2, 8, Vh)

    return tables


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4), (4, 4, 2, 6), (6, 4, 8, 2), (24, 24, 24, 64)])
def test_neighbour_table_matches_oracle_shifts(table_program, dims):
    X, Y, Z, T = dims
    nb = table_program(dims)
    full = np.arange(X * Y * Z * T, dtype=np.int64).reshape(T, Z, Y, X)  # n at (t, z, y, x)
    parity = O.parity(dims)
    for par in (0, 1):
        sites = full[parity == par]                                    # ascending n
        h = sites // 2
        assert np.array_equal(h, np.arange(len(h)))                    # h = n / 2 enumerates the parity
        for d in range(8):
            mu, sign = d % 4, (+1 if d < 4 else -1)
            neigh = O.shift(full, mu, sign, 0)[parity == par]          # n + sign mu_hat, per site
            assert np.array_equal(nb[par, d], neigh // 2), (par, d)
            assert np.all(O.parity(dims)[np.unravel_index(neigh, (T, Z, Y, X))] == 1 - par)
