// Cluster tree and admissibility (host).  Compiled with -ffp-contract=off so
// the admissibility arithmetic rounds identically on every host CPU.
#include "h2_tree.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace h2 {

static void bounds(const Tree& t, Box& b) {
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = INFINITY;
    b.hi[a] = -INFINITY;
  }
  for (int64_t q = b.s; q < b.e; ++q) {
    const double c[3] = {t.xt[q], t.yt[q], t.zt[q]};
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = std::min(b.lo[a], c[a]);
      b.hi[a] = std::max(b.hi[a], c[a]);
    }
  }
}

static bool admissible(const Box& a, const Box& b, double eta) {
  double da = 0.0, db = 0.0, g2 = 0.0;
  {
    double e0 = a.hi[0] - a.lo[0], e1 = a.hi[1] - a.lo[1], e2 = a.hi[2] - a.lo[2];
    da = std::sqrt(e0 * e0 + e1 * e1 + e2 * e2);
  }
  {
    double e0 = b.hi[0] - b.lo[0], e1 = b.hi[1] - b.lo[1], e2 = b.hi[2] - b.lo[2];
    db = std::sqrt(e0 * e0 + e1 * e1 + e2 * e2);
  }
  double g[3];
  for (int k = 0; k < 3; ++k) g[k] = std::max(0.0, std::max(a.lo[k] - b.hi[k], b.lo[k] - a.hi[k]));
  g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  double dist = std::sqrt(g2);
  return std::max(da, db) <= eta * dist;
}

// Balanced 2-means split of one box (Sec. V's k-means partition, with the
// number of clusters kept a power of two): order the box's caller indices
// as [left child, right child], left = the floor(n/2) points with the
// smallest |x - c0|^2 - |x - c1|^2, then move c0, c1 to the children's
// means and repeat (at most 20 steps) until the left child stops changing.
// Seeds: the point farthest from the box's mean and the point farthest from
// that one.  Sums run in increasing caller index, squared distances are
// ((dx^2 + dy^2) + dz^2), ties go to the lowest caller index; with the host
// code compiled without floating-point contraction every host rounds the
// same way.
static void balanced_two_means(const double* P, int64_t* first, int64_t* last) {
  const int64_t n = last - first;
  if (n < 2) return;
  std::vector<int64_t> idx(first, last);
  std::sort(idx.begin(), idx.end());
  // idx is in increasing caller index, so a position q in it orders the
  // points exactly as their caller indices do
  auto d2 = [&](int64_t i, const double c[3]) {
    const double dx = P[3 * i] - c[0], dy = P[3 * i + 1] - c[1], dz = P[3 * i + 2] - c[2];
    return (dx * dx + dy * dy) + dz * dz;
  };
  auto farthest = [&](const double c[3]) {
    int64_t best = idx[0];
    double bd = d2(idx[0], c);
    for (int64_t i : idx) {
      const double v = d2(i, c);
      if (v > bd) {
        bd = v;
        best = i;
      }
    }
    return best;
  };
  double m[3] = {0.0, 0.0, 0.0}, c0[3], c1[3];
  {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t i : idx) {
      sx += P[3 * i];
      sy += P[3 * i + 1];
      sz += P[3 * i + 2];
    }
    m[0] = sx / (double)n;
    m[1] = sy / (double)n;
    m[2] = sz / (double)n;
  }
  const int64_t a = farthest(m);
  for (int k = 0; k < 3; ++k) c0[k] = P[3 * a + k];
  const int64_t b = farthest(c0);
  for (int k = 0; k < 3; ++k) c1[k] = P[3 * b + k];
  const int64_t h = n / 2;
  std::vector<std::pair<double, int64_t>> key(n);   // (|x-c0|^2 - |x-c1|^2, position)
  std::vector<char> left(n, 0), prev(n, 0);
  auto keys = [&]() {
    for (int64_t q = 0; q < n; ++q) key[q] = {d2(idx[q], c0) - d2(idx[q], c1), q};
  };
  for (int it = 0; it < 20; ++it) {
    // the left child is the set of the h smallest keys (ties -> lower
    // caller index); only the set matters until the last step
    keys();
    std::nth_element(key.begin(), key.begin() + h, key.end());
    std::fill(left.begin(), left.end(), 0);
    for (int64_t q = 0; q < h; ++q) left[key[q].second] = 1;
    if (it > 0 && left == prev) break;
    prev = left;
    // children's means, summed in increasing caller index
    double sl[3] = {0.0, 0.0, 0.0}, sr[3] = {0.0, 0.0, 0.0};
    for (int64_t q = 0; q < n; ++q) {
      double* acc = left[q] ? sl : sr;
      acc[0] += P[3 * idx[q]];
      acc[1] += P[3 * idx[q] + 1];
      acc[2] += P[3 * idx[q] + 2];
    }
    for (int k = 0; k < 3; ++k) {
      c0[k] = sl[k] / (double)h;
      c1[k] = sr[k] / (double)(n - h);
    }
    if (it == 19) keys();
  }
  // final order: the keys of the last assignment, fully sorted
  std::sort(key.begin(), key.end());
  for (int64_t q = 0; q < n; ++q) first[q] = idx[key[q].second];
}

Tree build_tree(const double* P, int64_t N, int leaf, double eta, int partition) {
  Tree t;
  t.N = N;
  t.L = N > leaf ? (int)std::ceil(std::log2((double)N / (double)leaf)) : 0;
  t.perm.resize(N);
  std::iota(t.perm.begin(), t.perm.end(), 0);
  t.boxes.assign(t.L + 1, {});
  t.boxes[0].push_back(Box{0, N, {0, 0, 0}, {0, 0, 0}});
  std::vector<int64_t> tmp;
  for (int l = 0; l < t.L; ++l) {
    for (const Box& b : t.boxes[l]) {
      if (partition == 1) {
        balanced_two_means(P, t.perm.data() + b.s, t.perm.data() + b.e);
        int64_t mid = b.s + (b.e - b.s) / 2;
        t.boxes[l + 1].push_back(Box{b.s, mid, {0, 0, 0}, {0, 0, 0}});
        t.boxes[l + 1].push_back(Box{mid, b.e, {0, 0, 0}, {0, 0, 0}});
        continue;
      }
      // bounding box of the caller points of this box
      double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int64_t q = b.s; q < b.e; ++q) {
        const double* c = P + 3 * t.perm[q];
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], c[a]);
          hi[a] = std::max(hi[a], c[a]);
        }
      }
      int ax = 0;
      double best = hi[0] - lo[0];
      for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > best) { best = hi[a] - lo[a]; ax = a; }
      std::sort(t.perm.begin() + b.s, t.perm.begin() + b.e, [&](int64_t u, int64_t v) {
        double cu = P[3 * u + ax], cv = P[3 * v + ax];
        return cu < cv || (cu == cv && u < v);
      });
      int64_t mid = b.s + (b.e - b.s) / 2;
      t.boxes[l + 1].push_back(Box{b.s, mid, {0, 0, 0}, {0, 0, 0}});
      t.boxes[l + 1].push_back(Box{mid, b.e, {0, 0, 0}, {0, 0, 0}});
    }
  }
  t.xt.resize(N);
  t.yt.resize(N);
  t.zt.resize(N);
  for (int64_t q = 0; q < N; ++q) {
    t.xt[q] = P[3 * t.perm[q] + 0];
    t.yt[q] = P[3 * t.perm[q] + 1];
    t.zt[q] = P[3 * t.perm[q] + 2];
  }
  for (int l = 0; l <= t.L; ++l)
    for (Box& b : t.boxes[l]) bounds(t, b);
  // dual traversal: children of near pairs are far (admissible) or near
  t.near.assign(t.L + 1, {});
  t.far.assign(t.L + 1, {});
  for (int l = 0; l <= t.L; ++l) {
    t.near[l].assign(t.boxes[l].size(), {});
    t.far[l].assign(t.boxes[l].size(), {});
  }
  t.near[0][0].push_back(0);
  for (int l = 1; l <= t.L; ++l) {
    for (size_t p = 0; p < t.boxes[l - 1].size(); ++p)
      for (int q : t.near[l - 1][p])
        for (int a = 2 * (int)p; a < 2 * (int)p + 2; ++a)
          for (int c = 2 * q; c < 2 * q + 2; ++c) {
            if (admissible(t.boxes[l][a], t.boxes[l][c], eta)) t.far[l][a].push_back(c);
            else t.near[l][a].push_back(c);
          }
    for (size_t i = 0; i < t.boxes[l].size(); ++i) {
      std::sort(t.near[l][i].begin(), t.near[l][i].end());
      std::sort(t.far[l][i].begin(), t.far[l][i].end());
    }
  }
  // l_top: largest l such that no level <= l has a far pair
  t.ltop = 0;
  for (int l = 0; l <= t.L; ++l) {
    bool any = false;
    for (auto& f : t.far[l]) any |= !f.empty();
    if (any) break;
    t.ltop = l;
  }
  return t;
}

void far_samples(const Tree& t, int l, int i, int s0, int smin, std::vector<int64_t>& out) {
  out.clear();
  int a = i;
  for (int ll = l; ll >= 1; --ll) {
    int s = 0;
    if (s0 > 0) s = std::max(smin, s0 >> (l - ll));
    for (int J : t.far[ll][a]) {
      const Box& b = t.boxes[ll][J];
      int64_t nJ = b.e - b.s;
      if (s0 == 0 || nJ <= s) {
        for (int64_t q = b.s; q < b.e; ++q) out.push_back(q);
      } else {
        for (int k = 0; k < s; ++k) out.push_back(b.s + ((int64_t)(2 * k + 1) * nJ) / (2 * (int64_t)s));
      }
    }
    a /= 2;
  }
}

}  // namespace h2
