"""The library's host-side cluster tree (coordinate bisection and balanced
2-means) and admissibility lists against the oracle's, on the CPU: the tree
builder is compiled on its own with the host compiler (no floating-point
contraction, as in the library build) and its permutation, near/far lists
and l_top are compared exactly."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import synth
from oracle import h2ulv_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "h2_tree.h"
int main(int argc, char** argv) {
  long long N = atoll(argv[2]);
  int leaf = atoi(argv[3]), part = atoi(argv[4]);
  double eta = atof(argv[5]);
  std::vector<double> P(3 * N);
  FILE* f = fopen(argv[1], "rb");
  if (fread(P.data(), 8, 3 * N, f) != (size_t)(3 * N)) return 2;
  fclose(f);
  h2::Tree t = h2::build_tree(P.data(), N, leaf, eta, part);
  printf("%d %d\n", t.L, t.ltop);
  for (long long q = 0; q < N; ++q) printf("%lld ", (long long)t.perm[q]);
  printf("\n");
  for (int l = 0; l <= t.L; ++l)
    for (size_t i = 0; i < t.near[l].size(); ++i) {
      printf("N %d %zu:", l, i);
      for (int j : t.near[l][i]) printf(" %d", j);
      printf("\nF %d %zu:", l, i);
      for (int j : t.far[l][i]) printf(" %d", j);
      printf("\n");
    }
  return 0;
}
'''


@pytest.fixture(scope="module")
def driver():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "drv.cpp")
    open(src, "w").write(DRIVER)
    exe = os.path.join(d, "drv")
    csrc = os.path.join(ROOT, "paper_2208_10907_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", csrc, src,
                    os.path.join(csrc, "h2_tree.cpp"), "-o", exe], check=True)
    return d, exe


def run_tree(driver, X, leaf, part, eta=1.0):
    d, exe = driver
    pf = os.path.join(d, "pts.bin")
    np.ascontiguousarray(X, dtype=np.float64).tofile(pf)
    out = subprocess.run([exe, pf, str(len(X)), str(leaf), str(part), repr(eta)], capture_output=True, text=True,
                         check=True).stdout.splitlines()
    L, ltop = map(int, out[0].split())
    perm = np.array(out[1].split(), dtype=np.int64)
    near, far = {}, {}
    for line in out[2:]:
        tag, l, rest = line.split(" ", 2)
        i, lst = rest.split(":")
        (near if tag == "N" else far)[(int(l), int(i))] = [int(v) for v in lst.split()]
    return L, ltop, perm, near, far


@pytest.mark.parametrize("part", ["bisection", "kmeans"])
@pytest.mark.parametrize("case", ["surfaces", "sphereball", "cube_ragged"])
def test_host_tree_equals_oracle(driver, part, case):
    X = {"surfaces": lambda: synth.surface_union(6000, 3), "sphereball": lambda: synth.sphere_ball(4096, 8),
         "cube_ragged": lambda: synth.cube(3001, 2)}[case]()
    leaf = 100 if case == "cube_ragged" else 128
    pb = O.Problem(X, "laplace", leaf, 1.0, 1e-8, 64, partition=part)
    L, ltop, perm, near, far = run_tree(driver, X, leaf, 1 if part == "kmeans" else 0)
    assert L == pb.L and ltop == pb.ltop
    np.testing.assert_array_equal(perm, pb.perm)
    for l in range(L + 1):
        for i in range(2 ** l):
            assert near[(l, i)] == pb.near[l][i]
            assert far[(l, i)] == pb.far[l][i]


def test_kmeans_and_bisection_differ_on_surfaces(driver):
    X = synth.surface_union(6000, 3)
    _, _, p0, _, _ = run_tree(driver, X, 128, 0)
    _, _, p1, _, _ = run_tree(driver, X, 128, 1)
    assert not np.array_equal(p0, p1)
