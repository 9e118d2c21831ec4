"""Pins of the oracle's test diagnostics: the ReLU-margin measure the FP32
gradient tests use to leave out rays whose hidden units sit on a kink, and the
prescribed pinhole ray generation of render requests.

Margins are pinned by planted kinks with closed-form margins: a hidden unit
made to compute the difference of two equal inputs (z = 0 exactly) and the
same unit with one weight shortened by delta, whose margin |z| / s follows
from the definition of the error scale s by hand. A scale that dropped the
propagated term (h + s of the layer below) or an absolute value gives a
different number. Camera rays are pinned by the FP64 pinhole closed form, unit
length and the image's mirror symmetry.
"""
import math

import numpy as np

import oracle
from paper_2404_16221_b300 import synthetic as sy


def _unit_case(L=4):
    w = sy.workload("unit")
    w.level_res = w.level_res[:L]
    E = oracle.table_entries(w.level_res, w.log2_T)
    g = sy.rng(90, "misc")
    tables = g.uniform(0.1, 1.0, (1, E, 2))
    o, d = sy.workload_rays(w, 64)
    return w, E, g, tables, o, d


def _fused_field(w, tables, W1, W2, W3):
    mlp = np.concatenate([W1.reshape(-1), W2.reshape(-1), W3.reshape(-1)])[None, :]
    return oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, tables, mlp)


def test_margin_of_a_planted_first_layer_kink():
    w, E, g, tables, o, d = _unit_case()
    # level 0's two features equal entry by entry, so feat_0 == feat_1 exactly
    l0 = oracle.level_offset(w.level_res, w.log2_T, 1)
    tables[0, :l0, 1] = tables[0, :l0, 0]
    W1 = g.uniform(0.0, 0.05, (w.mlp_in, w.W))
    W1[:, 0] = 0.0
    W1[0, 0] = 1.0
    W2 = g.uniform(0.0, 0.05, (w.W, w.W))
    W3 = g.normal(0.0, 0.1, (w.W, 4))
    hit = np.isfinite(oracle.relu_margin(_fused_field(w, tables, W1, W2, W3), w.S, o, d))
    assert hit.sum() > 40
    for delta in (0.0, 1e-3, 0.25):
        W1[1, 0] = -(1.0 - delta)
        m = oracle.relu_margin(_fused_field(w, tables, W1, W2, W3), w.S, o, d)
        # unit 0: z = delta f0, s = (2 - delta) f0; every other first-layer
        # unit has margin 1 and every second-layer unit about 1/2
        np.testing.assert_allclose(m[hit], delta / (2.0 - delta), rtol=1e-9, atol=1e-15)
        assert np.all(np.isinf(m[~hit]))


def test_margin_of_a_planted_second_layer_kink():
    w, E, g, tables, o, d = _unit_case()
    W1 = g.uniform(0.0, 0.05, (w.mlp_in, w.W))
    W1[:, 1] = W1[:, 0]  # h1_0 == h1_1 exactly
    W2 = g.uniform(0.0, 0.05, (w.W, w.W))
    W3 = g.normal(0.0, 0.1, (w.W, 4))
    hit = np.isfinite(oracle.relu_margin(_fused_field(w, tables, W1, W2, W3), w.S, o, d))
    for delta in (0.0, 1e-3, 0.25):
        W2[:, 0] = 0.0
        W2[0, 0], W2[1, 0] = 1.0, -(1.0 - delta)
        m = oracle.relu_margin(_fused_field(w, tables, W1, W2, W3), w.S, o, d)
        # positive first layer: s1 = h1, so z2_0 = delta h, s2_0 = (2 - delta) (h + h)
        np.testing.assert_allclose(m[hit], delta / (2.0 * (2.0 - delta)), rtol=1e-9, atol=1e-15)


def test_margin_of_a_planted_split_colour_kink():
    """Split representation: a kink in the colour MLP's second hidden layer.
    With positive tables, density weights and the g rows of Wc1 (SH rows
    zero), s1 = h1, sg = 2 g, s2 = 3 z2, so z3_0 = delta h2, s3_0 =
    (2 - delta) 4 h2."""
    w, E, g, tables, o, d = _unit_case()
    W = w.W
    Wd1 = g.uniform(0.0, 0.05, (w.mlp_in, W))
    Wd2 = g.uniform(0.0, 0.05, (W, 16))
    Wc1 = np.zeros((32, W))
    Wc1[:16] = g.uniform(0.0, 0.05, (16, W))
    Wc1[:, 1] = Wc1[:, 0]
    Wc2 = g.uniform(0.0, 0.05, (W, W))
    Wc3 = g.normal(0.0, 0.1, (W, 4))
    for delta in (0.0, 1e-3, 0.25):
        Wc2[:, 0] = 0.0
        Wc2[0, 0], Wc2[1, 0] = 1.0, -(1.0 - delta)
        mlp = np.concatenate([Wd1.reshape(-1), Wd2.reshape(-1), Wc1.reshape(-1), Wc2.reshape(-1),
                              Wc3.reshape(-1)])
        f = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, W, tables, mlp, arch=1)
        m = oracle.relu_margin(f, w.S, o, d)
        hit = np.isfinite(m)
        assert hit.sum() > 40
        np.testing.assert_allclose(m[hit], delta / (4.0 * (2.0 - delta)), rtol=1e-9, atol=1e-15)


def test_margin_ignores_skipped_samples():
    """With an empty occupancy grid no sample is evaluated: every margin is
    infinite."""
    w, E, g, tables, o, d = _unit_case()
    W1 = g.normal(0.0, 0.1, (w.mlp_in, w.W))
    W2 = g.normal(0.0, 0.1, (w.W, w.W))
    W3 = g.normal(0.0, 0.1, (w.W, 4))
    f = _fused_field(w, tables, W1, W2, W3)
    G = 4
    empty = np.zeros((1, oracle.occupancy_words(G)), np.uint32)
    assert np.all(np.isinf(oracle.relu_margin(f.with_occupancy(empty, G), w.S, o, d)))
    assert np.isfinite(oracle.relu_margin(f, w.S, o, d)).sum() > 40


def _frame(eye, target):
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return r, u, f


def test_camera_rays_match_the_fp64_pinhole():
    eye = np.array([0.3, -1.5, 2.5])
    r, u, f = _frame(eye, (0.5, 0.5, 0.1))
    r32, u32, f32 = (v.astype(np.float32) for v in (r, u, f))
    tan = math.tan(math.radians(60.0) / 2.0)
    H, W = 37, 58
    o, d = oracle.camera_rays(eye, r32, u32, f32, tan, W, H)
    assert o.shape == (H * W, 3) and np.all(o == eye.astype(np.float32))
    i, j = np.divmod(np.arange(H * W), W)
    x = ((j + 0.5) / W * 2.0 - 1.0) * tan * (W / H)
    y = (1.0 - (i + 0.5) / H * 2.0) * tan
    v = x[:, None] * r32.astype(np.float64) + y[:, None] * u32.astype(np.float64) + f32.astype(np.float64)
    ref = v / np.linalg.norm(v, axis=1, keepdims=True)
    assert np.abs(d - ref).max() < 1e-6
    assert np.abs(np.linalg.norm(d.astype(np.float64), axis=1) - 1.0).max() < 1e-6
    # a sub-range of pixels is the same rays
    o2, d2 = oracle.camera_rays(eye, r32, u32, f32, tan, W, H, first=100, count=333)
    assert np.array_equal(d2, d[100:433])


def test_camera_rays_centre_and_mirror_symmetry():
    """Odd image: the centre pixel looks along forward; pixels (i, j) and
    (i, W-1-j) mirror about the plane of up and forward."""
    eye = np.array([0.0, 0.0, 0.0])
    r, u, f = (np.eye(3)[k].astype(np.float32) for k in (0, 2, 1))  # right x, up z, forward y
    H, W = 9, 11
    o, d = oracle.camera_rays(eye, r, u, f, 0.5, W, H)
    c = (H // 2) * W + W // 2
    assert np.array_equal(d[c], np.array([0.0, 1.0, 0.0], np.float32))
    img = d.reshape(H, W, 3)
    np.testing.assert_allclose(img[:, ::-1, 0], -img[:, :, 0], atol=1e-7)
    np.testing.assert_allclose(img[:, ::-1, 1:], img[:, :, 1:], atol=1e-7)
    np.testing.assert_allclose(img[::-1, :, 2], -img[:, :, 2], atol=1e-7)
