"""Oracle of the spatial partitioning (Sec. 4.4 "Spatial Partitioning" and the
appendix section of the same name with its partition-scheme figure).

TEST INFRASTRUCTURE ONLY (callers: the test suite). Plain, recursive numpy
code written from the paper's description:

  * the scene content is a point cloud (SfM points, or samples of randomly
    drawn training rays when there is no point cloud);
  * for each axis, the candidate plane is where the cumulative distribution
    of the points along that axis equals 0.5;
  * of the three candidates, the one whose two partitions are closest to
    cubic is taken (aspect ratio of a box = longest side / shortest side;
    the pair is scored by the worse of its two boxes);
  * the step is applied recursively n times, giving 2^n boxes.

Readings where the paper is silent (the same in the library):
  * CDF = 0.5 plane of m points = the median of their coordinates along the
    axis, 0.5 (s[(m-1)//2] + s[m//2]) of the sorted coordinates s;
  * a point goes to the lower box if its coordinate < plane, else the upper;
  * a plane not strictly inside the box (too few points, all points on one
    face) is replaced by the box's midplane along that axis;
  * ties between axes go to the lowest axis (x, then y, then z);
  * boxes are listed depth first, lower half before upper half;
  * points outside the root box are ignored.
"""
from __future__ import annotations

import numpy as np


def aspect_ratio(lo, hi) -> float:
    ext = np.asarray(hi, np.float64) - np.asarray(lo, np.float64)
    if ext.min() <= 0.0:
        return np.inf
    return float(ext.max() / ext.min())


def cdf_half_plane(coords, lo: float, hi: float) -> float:
    """Plane where the points' CDF along one axis is 0.5 (their median),
    or the box midplane when that is not strictly inside (lo, hi)."""
    mid = np.float32(0.5) * (np.float32(lo) + np.float32(hi))
    if len(coords) == 0:
        return float(mid)
    s = np.sort(np.asarray(coords, np.float32))
    m = len(s)
    plane = np.float32(0.5) * (s[(m - 1) // 2] + s[m // 2])
    if not (np.float32(lo) < plane < np.float32(hi)):
        return float(mid)
    return float(plane)


def _split(pts, lo, hi, depth, boxes, counts):
    if depth == 0:
        boxes.append(np.concatenate([lo, hi]).astype(np.float32))
        counts.append(len(pts))
        return
    best = None
    for axis in range(3):
        plane = cdf_half_plane(pts[:, axis], lo[axis], hi[axis])
        hi_a = hi.copy()
        hi_a[axis] = plane
        lo_b = lo.copy()
        lo_b[axis] = plane
        cost = max(aspect_ratio(lo, hi_a), aspect_ratio(lo_b, hi))
        if best is None or cost < best[0]:
            best = (cost, axis, plane)
    _, axis, plane = best
    below = pts[:, axis] < np.float32(plane)
    hi_a = hi.copy()
    hi_a[axis] = plane
    lo_b = lo.copy()
    lo_b[axis] = plane
    _split(pts[below], lo, hi_a, depth - 1, boxes, counts)
    _split(pts[~below], lo_b, hi, depth - 1, boxes, counts)


def partition_boxes(points, root, levels: int):
    """2^levels boxes [K][6] (min xyz, max xyz; float32) and the number of
    points in each."""
    pts = np.asarray(points, np.float32).reshape(-1, 3)
    root = np.asarray(root, np.float32).reshape(6)
    lo, hi = root[:3].copy(), root[3:].copy()
    inside = np.all((pts >= lo) & (pts <= hi), axis=1)
    boxes, counts = [], []
    _split(pts[inside], lo, hi, levels, boxes, counts)
    return np.stack(boxes), np.asarray(counts, np.int64)
