// Host-side cluster tree, strong-admissibility lists and far-field samples.
#pragma once
#include <stdint.h>
#include <vector>

namespace h2 {

struct Box {
  int64_t s, e;  // tree-order point range (within the problem)
  double lo[3], hi[3];
};

struct Tree {
  int64_t N = 0;
  int L = 0, ltop = 0;
  std::vector<int64_t> perm;                       // tree position -> caller index
  std::vector<std::vector<Box>> boxes;             // [level][box]
  std::vector<std::vector<std::vector<int>>> near; // [level][box] -> sorted boxes
  std::vector<std::vector<std::vector<int>>> far;
  std::vector<double> xt, yt, zt;                  // tree-order coordinates
};

// Cluster tree (full binary, 2^L leaves, L = ceil(log2(N/leaf))) by
// coordinate bisection (partition 0) or balanced 2-means (partition 1), and
// the near / far lists of strong admissibility
// max(diam I, diam J) <= eta * dist(I, J).
Tree build_tree(const double* pts_rowmajor, int64_t N, int leaf, double eta, int partition);

// Far-field sample of box i at level l (tree-order indices within the
// problem): the far boxes of level l' (l' = l, l-1, ..., 1, along i's
// ancestors) give max(smin, s0 >> (l - l')) evenly spaced points each, a box
// with at most that many points gives all of them; s0 = 0 gives every point.
void far_samples(const Tree& t, int l, int i, int s0, int smin, std::vector<int64_t>& out);

}  // namespace h2
