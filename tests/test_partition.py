"""Spatial partitioning (Sec. 4.4 "Spatial Partitioning"): the oracle against
properties the paper's description fixes, and the library's host
implementation against the oracle (bit for bit)."""
import numpy as np
import pytest

from oracle import partition as OP
from paper_2404_16221_b300 import synthetic as sy


def _leaf_of(points, boxes, root):
    """Index of the box holding each point: lower faces inclusive, upper faces
    exclusive except on the root's upper faces."""
    p = np.asarray(points, np.float32)[:, None, :]
    lo, hi = boxes[None, :, :3], boxes[None, :, 3:]
    at_root_hi = hi == np.asarray(root, np.float32)[3:][None, None, :]
    inside = (p >= lo) & ((p < hi) | (at_root_hi & (p <= hi)))
    member = inside.all(-1)
    return member


def test_hand_example_splits_the_long_axis_at_the_median():
    root = [0, 0, 0, 4, 1, 1]
    pts = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5], [2.5, 0.5, 0.5], [3.5, 0.5, 0.5]], np.float32)
    boxes, counts = OP.partition_boxes(pts, root, 1)
    # median plane along x is (1.5 + 2.5) / 2 = 2; halves 2x1x1 (aspect 2) beat y or z splits (aspect 8)
    assert np.array_equal(boxes, np.array([[0, 0, 0, 2, 1, 1], [2, 0, 0, 4, 1, 1]], np.float32))
    assert list(counts) == [2, 2]


def test_aspect_ratio_picks_the_axis_that_keeps_boxes_cubic():
    # uniform content in a 1 x 4 x 1 box: the first split is along y, near y = 2
    g = np.random.default_rng(3)
    pts = (g.uniform(0, 1, (4000, 3)) * [1, 4, 1]).astype(np.float32)
    boxes, _ = OP.partition_boxes(pts, [0, 0, 0, 1, 4, 1], 1)
    assert boxes[0, 4] == boxes[1, 1] and abs(boxes[0, 4] - 2.0) < 0.1
    assert boxes[0, 3] == 1 and boxes[0, 5] == 1  # x and z untouched


@pytest.mark.parametrize("levels", [1, 2, 3, 5])
def test_balanced_disjoint_and_tiling(levels):
    w = sy.workload("city32")
    root = sy.scene_root(w)
    n = (1 << levels) * 1000
    pts = sy.content_points(w, n, seed=11)
    boxes, counts = OP.partition_boxes(pts, root, levels)
    K = 1 << levels
    assert boxes.shape == (K, 6)
    # distinct coordinates: every median split halves exactly
    assert np.all(counts == n // K)
    # boxes tile the root: volumes add up and no two overlap
    ext = boxes[:, 3:].astype(np.float64) - boxes[:, :3]
    assert np.all(ext > 0)
    vol_root = np.prod(root[3:].astype(np.float64) - root[:3])
    assert abs(ext.prod(1).sum() - vol_root) <= 1e-5 * vol_root
    for a in range(K):
        for b in range(a + 1, K):
            ov = np.minimum(boxes[a, 3:], boxes[b, 3:]) - np.maximum(boxes[a, :3], boxes[b, :3])
            assert not np.all(ov > 0)
    # each point lies in exactly one box, and the counts are those memberships
    member = _leaf_of(pts, boxes, root)
    assert np.all(member.sum(1) == 1)
    assert np.array_equal(member.sum(0), counts)


def test_empty_cloud_falls_back_to_midplanes_and_outside_points_are_ignored():
    boxes, counts = OP.partition_boxes(np.zeros((0, 3), np.float32), [0, 0, 0, 2, 1, 1], 1)
    assert np.array_equal(boxes, np.array([[0, 0, 0, 1, 1, 1], [1, 0, 0, 2, 1, 1]], np.float32))
    assert list(counts) == [0, 0]
    pts = np.array([[5, 5, 5], [0.25, 0.5, 0.5], [1.75, 0.5, 0.5]], np.float32)
    boxes, counts = OP.partition_boxes(pts, [0, 0, 0, 2, 1, 1], 1)
    assert list(counts) == [1, 1] and boxes[0, 3] == 1.0


def test_ray_samples_stand_in_for_a_point_cloud():
    # without a point cloud the content comes from samples of training rays
    w = sy.workload("grid8")
    root = sy.scene_root(w)
    o, d = sy.workload_rays(w, 2048, seed=77)
    pts = sy.ray_sample_points(o, d, root, 16, 5)
    assert len(pts) > 0
    assert np.all(pts >= root[:3]) and np.all(pts <= root[3:])
    boxes, counts = OP.partition_boxes(pts, root, 3)
    assert counts.sum() == len(pts) and counts.max() - counts.min() <= 1


@pytest.mark.parametrize("name,levels,source", [("grid8", 3, "content"), ("city32", 5, "content"),
                                                ("city32", 5, "rays"), ("unit", 0, "content"),
                                                ("grid8", 1, "rays")])
def test_library_matches_oracle_bitwise(name, levels, source):
    from paper_2404_16221_b300 import api

    w = sy.workload(name)
    root = sy.scene_root(w)
    if source == "content":
        pts = sy.content_points(w, 50000, seed=13)
    else:
        o, d = sy.workload_rays(w, 2048, seed=71)
        pts = sy.ray_sample_points(o, d, root, 24, 9)
    b_lib, c_lib = api.partition_boxes(pts, root, levels)
    b_ref, c_ref = OP.partition_boxes(pts, root, levels)
    assert np.array_equal(b_lib, b_ref)
    assert np.array_equal(c_lib, c_ref)


def test_library_rejects_bad_arguments():
    from paper_2404_16221_b300 import api, native as N

    pts = np.zeros((4, 3), np.float32)
    for root, levels in (([0, 0, 0, 1, 1, 1], 11), ([0, 0, 0, 0, 1, 1], 1), ([0, 0, 0, 1, 1, 1], -1)):
        with pytest.raises(N.NerfxlError) as e:
            api.partition_boxes(pts, root, levels)
        assert e.value.status == N.E_INVALID
