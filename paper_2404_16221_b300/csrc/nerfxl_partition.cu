// Spatial partitioning of the scene into 2^n disjoint boxes with balanced
// content (Sec. 4.4 "Spatial Partitioning"; the appendix's partition scheme):
// recursively, split a box at the plane where the CDF of the points inside it
// along an axis is 0.5, choosing among the three axes the split whose two
// boxes are closest to cubic. Host code: it runs once per scene on a point
// cloud (SfM points or samples of training rays) and hands the boxes to the
// renderer.
//
// Readings where the paper is silent: the CDF = 0.5 plane of m points is the
// median 0.5 (s[(m-1)/2] + s[m/2]) of their sorted coordinates (FP32); a point
// goes below the plane if its coordinate < plane; a plane not strictly inside
// the box falls back to the box midplane; the aspect ratio of a box is its
// longest side over its shortest (a pair scores the worse of its two boxes);
// ties go to the lowest axis; boxes are listed depth first, lower half first;
// points outside the root box are ignored.

#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "nerfxl_host.h"

namespace nerfxl {
namespace {

struct Box {
  float lo[3], hi[3];
};

double aspect_ratio(const Box& b) {
  double mn = std::numeric_limits<double>::infinity(), mx = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double e = (double)b.hi[a] - (double)b.lo[a];
    mn = std::min(mn, e);
    mx = std::max(mx, e);
  }
  return mn <= 0.0 ? std::numeric_limits<double>::infinity() : mx / mn;
}

// Median plane of points[idx[b..e)] along `axis`, or the box midplane.
float cdf_half_plane(const float* pts, const std::vector<int64_t>& idx, int64_t b, int64_t e, int axis, float lo,
                     float hi, std::vector<float>& scratch) {
  const float mid = 0.5f * (lo + hi);
  const int64_t m = e - b;
  if (m == 0) return mid;
  scratch.resize((size_t)m);
  for (int64_t i = 0; i < m; ++i) scratch[(size_t)i] = pts[3 * idx[(size_t)(b + i)] + axis];
  const size_t ia = (size_t)((m - 1) / 2), ib = (size_t)(m / 2);
  std::nth_element(scratch.begin(), scratch.begin() + ib, scratch.end());
  const float sb = scratch[ib];
  float sa = sb;
  if (ia != ib) sa = *std::max_element(scratch.begin(), scratch.begin() + ib);  // largest of the lower part
  const float plane = 0.5f * (sa + sb);
  return (lo < plane && plane < hi) ? plane : mid;
}

void split(const float* pts, std::vector<int64_t>& idx, int64_t b, int64_t e, const Box& box, int depth,
           std::vector<Box>& out, std::vector<int64_t>& counts, std::vector<float>& scratch) {
  if (depth == 0) {
    out.push_back(box);
    counts.push_back(e - b);
    return;
  }
  double best_cost = 0.0;
  int best_axis = -1;
  float best_plane = 0.0f;
  for (int axis = 0; axis < 3; ++axis) {
    const float plane = cdf_half_plane(pts, idx, b, e, axis, box.lo[axis], box.hi[axis], scratch);
    Box lower = box, upper = box;
    lower.hi[axis] = plane;
    upper.lo[axis] = plane;
    const double cost = std::max(aspect_ratio(lower), aspect_ratio(upper));
    if (best_axis < 0 || cost < best_cost) {
      best_cost = cost;
      best_axis = axis;
      best_plane = plane;
    }
  }
  const int axis = best_axis;
  const float plane = best_plane;
  // stable partition keeps the recursion's point order deterministic
  std::vector<int64_t> below, above;
  below.reserve((size_t)(e - b));
  for (int64_t i = b; i < e; ++i) {
    const int64_t p = idx[(size_t)i];
    if (pts[3 * p + axis] < plane) below.push_back(p);
    else above.push_back(p);
  }
  std::copy(below.begin(), below.end(), idx.begin() + b);
  std::copy(above.begin(), above.end(), idx.begin() + b + (int64_t)below.size());
  const int64_t mid = b + (int64_t)below.size();
  Box lower = box, upper = box;
  lower.hi[axis] = plane;
  upper.lo[axis] = plane;
  split(pts, idx, b, mid, lower, depth - 1, out, counts, scratch);
  split(pts, idx, mid, e, upper, depth - 1, out, counts, scratch);
}

}  // namespace
}  // namespace nerfxl

using namespace nerfxl;

extern "C" nerfxl_status nerfxl_partition(const float* points, int64_t n_points, const float* root, int32_t levels,
                                          float* boxes, int64_t* counts) {
  if (!root || !boxes || n_points < 0 || (n_points > 0 && !points))
    return set_error(NERFXL_E_INVALID, "bad partition arguments");
  if (levels < 0 || levels > 10) return set_error(NERFXL_E_INVALID, "levels must be in 0..10");
  Box rb;
  for (int a = 0; a < 3; ++a) {
    rb.lo[a] = root[a];
    rb.hi[a] = root[3 + a];
    if (!(rb.lo[a] < rb.hi[a])) return set_error(NERFXL_E_INVALID, "root box must have positive extent");
  }
  std::vector<int64_t> idx;
  idx.reserve((size_t)n_points);
  for (int64_t i = 0; i < n_points; ++i) {
    bool in = true;
    for (int a = 0; a < 3; ++a) {
      const float c = points[3 * i + a];
      in = in && c >= rb.lo[a] && c <= rb.hi[a];
    }
    if (in) idx.push_back(i);
  }
  std::vector<Box> out;
  std::vector<int64_t> cnt;
  std::vector<float> scratch;
  split(points, idx, 0, (int64_t)idx.size(), rb, levels, out, cnt, scratch);
  for (size_t k = 0; k < out.size(); ++k) {
    for (int a = 0; a < 3; ++a) {
      boxes[6 * k + a] = out[k].lo[a];
      boxes[6 * k + 3 + a] = out[k].hi[a];
    }
    if (counts) counts[k] = cnt[k];
  }
  return NERFXL_OK;
}
