// Point ordering for the cluster tree (host code, no device work): a kd-tree
// whose nodes are the consecutive ranges of Def. 2.1 with the ceiling split
// of Sect. 4, so that for points in 2 or 3 dimensions every node of the tree
// is a spatial cluster (as the 1D workloads get by sorting).
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <utility>
#include <vector>

#include "handle.cuh"

using namespace hodlr;

extern "C" hodlr_status hodlr_tree_order(int32_t n, int32_t dim, const double* points, int32_t depth, int32_t* perm) {
  if (n < 1 || !points || !perm) return set_error(HODLR_EINVAL, "hodlr_tree_order: n >= 1 and non-null arrays");
  if (dim < 1 || dim > 3) return set_error(HODLR_EINVAL, "hodlr_tree_order: dim must be 1, 2 or 3");
  if (depth < 0 || depth > 30 || (int64_t(1) << depth) > n)
    return set_error(HODLR_EINVAL, "hodlr_tree_order: depth must satisfy 0 <= depth and 2^depth <= n");
  for (int64_t i = 0; i < (int64_t)n * dim; ++i)
    if (!std::isfinite(points[i])) return set_error(HODLR_EINVAL, "hodlr_tree_order: points must be finite");
  std::iota(perm, perm + n, 0);
  std::vector<std::pair<int32_t, int32_t>> cur{{0, n}}, nxt;
  for (int k = 0; k < depth; ++k) {
    nxt.clear();
    for (const auto& node : cur) {
      const int32_t s = node.first, m = node.second, left = (m + 1) / 2;
      nxt.push_back({s, left});
      nxt.push_back({s + left, m - left});
      if (m < 2) continue;
      // the coordinate along which the node's points spread most (the lowest
      // one on a tie)
      int d = 0;
      double best = 0.0;
      for (int c = 0; c < dim; ++c) {
        double lo = std::numeric_limits<double>::infinity(), hi = -lo;
        for (int32_t t = s; t < s + m; ++t) {
          const double v = points[(int64_t)perm[t] * dim + c];
          lo = std::min(lo, v);
          hi = std::max(hi, v);
        }
        const double spread = hi - lo;
        if (c == 0 || spread > best) {
          best = spread;
          d = c;
        }
      }
      // by that coordinate, ties by original index: the left child gets the
      // ceil(m/2) smallest
      std::sort(perm + s, perm + s + m, [&](int32_t a, int32_t b) {
        const double xa = points[(int64_t)a * dim + d], xb = points[(int64_t)b * dim + d];
        return xa < xb || (xa == xb && a < b);
      });
    }
    cur.swap(nxt);
  }
  return HODLR_OK;
}
