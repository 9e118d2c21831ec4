"""Occupancy-grid skipping and refresh (the spatial-skipping structure of
Sec. 5.1, the grid of the cited Instant-NGP paper): the oracle against what
the definition fixes -- a full grid changes nothing, an empty grid renders
nothing, hand-placed cells keep exactly the samples whose points they hold,
skipping commutes with the partitioned rendering, gradients match central
differences, the refresh draws its points inside their cells from Philox
(known-answer vectors) and keeps a decaying maximum of the density."""
import os

import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import synthetic as sy

import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(K, G, value):
    return np.full((K, oracle.occupancy_words(G)), value, np.uint32)


def _set_cell(occ, k, G, cx, cy, cz):
    c = cx + G * (cy + G * cz)
    occ[k, c // 32] |= np.uint32(1 << (c % 32))


def _random_grid(K, G, p, seed):
    g = sy.rng(seed, "misc")
    bits = g.random((K, G ** 3)) < p
    pad = np.zeros((K, oracle.occupancy_words(G) * 32), bool)
    pad[:, :G ** 3] = bits
    return np.packbits(pad.reshape(K, -1, 32), axis=-1, bitorder="little").view(np.uint32).reshape(K, -1), bits


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert [int(x) for x in oracle.philox4x32_10(v[0:4], v[4:6])] == v[6:10]


def _small_field(name="grid8", L=4, log2_T=12, S=None):
    w = H.workload(name, L=L, log2_T=log2_T, S=S)
    t, m = H.params(w)
    return w, H.oracle_field(w, t, m)


def test_full_grid_changes_nothing():
    w, f = _small_field()
    o, d = sy.workload_rays(w, 96, seed=5)
    ref = oracle.render(f, w.S, o, d, 0)
    for G in (1, 5, 16):
        out = oracle.render(f.with_occupancy(_grid(w.K, G, 0xFFFFFFFF), G), w.S, o, d, 0)
        for k in ("rgb", "depth", "opacity", "dist", "tfinal", "n_samples"):
            assert np.array_equal(out[k], ref[k]), (G, k)


def test_empty_grid_renders_nothing_and_has_no_gradient():
    w, f = _small_field()
    o, d = sy.workload_rays(w, 64, seed=6)
    fe = f.with_occupancy(_grid(w.K, 8, 0), 8)
    out = oracle.render(fe, w.S, o, d, 1)
    for k in ("rgb", "depth", "opacity", "dist", "n_samples"):
        assert not np.any(out[k]), k
    assert np.all(out["tfinal"] == 1.0)
    tgt = np.full((len(o), 3), 0.5, np.float32)
    L, gt, gm = oracle.loss_grad(fe, w.S, o, d, tgt, 0.01)
    assert L == pytest.approx(0.25) and not gt.any() and not gm.any()


def _unit_samples(f, S, o, d):
    """Per-interval sigma, rgb, tbar, delta of one ray, from the oracle's
    interval, encoding and MLP entry points (no occupancy involved)."""
    count, a, b, region = oracle.intervals(f, S, o[None], d[None], S + 4)
    n = int(count[0])
    a, b, region = a[0, :n], b[0, :n], region[0, :n]
    tb = np.float32(0.5) * (a + b)
    x = (o[None, :] + tb[:, None] * d[None, :]).astype(np.float32)
    raw = oracle.mlp(f, region, oracle.encode_points(f, region, x))
    return np.exp(raw[:, 0]), 1.0 / (1.0 + np.exp(-raw[:, 1:])), tb.astype(np.float64), (b - a).astype(np.float64)


@pytest.mark.parametrize("axis,cell,kept", [
    # ray along +x at y = -0.4, z = 0.4 (u_y = 0.1, u_z = 0.9): cells (cx, 0, 3); u_x = (j + 0.5) / 64
    (0, (2, 0, 3), range(32, 48)),
    # along +y at x = 0.1, z = 0.4: cells (2, cy, 3)
    (1, (2, 0, 3), range(0, 16)),
    # along +z at x = 0.1, y = -0.4: cells (2, 0, cz)
    (2, (2, 0, 3), range(48, 64)),
    # along +x at y = -0.4 (row cy = 0) when only a cell of row cy = 1 is set
    (0, (2, 1, 3), range(0)),
])
def test_hand_placed_cell_keeps_exactly_its_samples(axis, cell, kept):
    """K = 1 over [-0.5, 0.5]^3, G = 4, one set cell. A ray parallel to an axis
    enters at t = 1.5 and leaves at 2.5; its 64 intervals are [1.5 + j/64,
    1.5 + (j+1)/64], so sample j sits at region coordinate (j + 0.5)/64 along
    the axis (exact in binary) and lies in cell floor((j + 0.5) / 16). The
    render must equal the single pass over all intervals with sigma zeroed
    outside the listed j: this fixes the x-fastest cell order and the bit
    order within words."""
    w, f = _small_field("unit", L=4, log2_T=12, S=64)
    G = 4
    occ = _grid(1, G, 0)
    _set_cell(occ, 0, G, *cell)
    fo = f.with_occupancy(occ, G)
    o = np.array([0.1, -0.4, 0.4], np.float32)
    o[axis] = -2.0
    dvec = np.zeros(3, np.float32)
    dvec[axis] = 1.0
    sigma, rgb, tb, dl = _unit_samples(f, w.S, o, dvec)
    assert len(sigma) == 64
    mask = np.zeros(64, bool)
    mask[list(kept)] = True
    s_single, _ = oracle.render_samples(np.zeros(64, np.int32), np.where(mask, sigma, 0.0), rgb, tb, dl)
    for mode in (0, 1):
        out = oracle.render(fo, w.S, o[None], dvec[None], mode)
        got = np.concatenate([out["rgb"][0], [out["depth"][0], out["opacity"][0], out["dist"][0], out["tfinal"][0]]])
        np.testing.assert_allclose(got, s_single[[0, 1, 2, 3, 4, 5, 6]], rtol=1e-13, atol=1e-15)
        assert out["n_samples"][0] == mask.sum()


@pytest.mark.parametrize("name", ["grid8", "city32"])
def test_skipping_commutes_with_partitioned_rendering(name):
    """With a sparse grid, the partitioned render (Algorithm 1-2 over the
    segments' kept samples) still equals the single pass."""
    w, f = _small_field(name)
    G = 16
    occ, _ = _random_grid(w.K, G, 0.3, 21)
    fo = f.with_occupancy(occ, G)
    o, d = sy.workload_rays(w, 128, seed=22)
    a, b = oracle.render(fo, w.S, o, d, 0), oracle.render(fo, w.S, o, d, 1)
    for k in ("rgb", "depth", "opacity", "dist", "tfinal"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-13)
    full = oracle.render(f, w.S, o, d, 0)
    hit = full["n_samples"] > 0
    assert np.all(a["n_samples"] <= full["n_samples"])
    frac = a["n_samples"][hit].sum() / full["n_samples"][hit].sum()
    assert 0.2 < frac < 0.4  # about the occupied share of the cells
    assert np.abs(a["opacity"] - full["opacity"]).max() > 1e-3


def test_gradient_with_skipping_matches_central_differences():
    w, f = _small_field("grid8", L=4, log2_T=12, S=32)
    G = 8
    occ, _ = _random_grid(w.K, G, 0.4, 31)
    fo = f.with_occupancy(occ, G)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 48, 32)
    o, d = o[sel].copy(), d[sel].copy()
    tgt = sy.rng(33, "misc").uniform(0, 1, (len(o), 3)).astype(np.float32)
    lam = 0.01
    L, gt, gm = oracle.loss_grad(fo, w.S, o, d, tgt, lam)
    _, gt_full, _ = oracle.loss_grad(f, w.S, o, d, tgt, lam)
    g = sy.rng(34, "misc")
    tab = g.choice(np.flatnonzero(gt.reshape(-1)), 40, replace=False)
    # entries read only by skipped samples: zero with the grid, non-zero without
    dead = np.flatnonzero((gt.reshape(-1) == 0) & (gt_full.reshape(-1) != 0))
    assert len(dead) > 0
    dead = g.choice(dead, min(20, len(dead)), replace=False)
    mw = g.choice(np.flatnonzero(gm.reshape(-1)), 40, replace=False)
    idx = np.concatenate([tab, dead, mw]).astype(np.int64)
    which = np.concatenate([np.zeros(len(tab) + len(dead)), np.ones(len(mw))]).astype(np.int32)
    an = np.concatenate([gt.reshape(-1)[tab], gt.reshape(-1)[dead], gm.reshape(-1)[mw]])
    scale = np.where(which == 0, np.abs(gt).max(), np.abs(gm).max())
    fd = oracle.fd_grad(fo, w.S, o, d, tgt, lam, which, idx, eps=1e-5)
    err = np.abs(fd - an) / (np.abs(an) + scale)
    assert err.max() <= 1e-4, np.sort(err)[-5:]
    assert np.abs(fd[len(tab):len(tab) + len(dead)]).max() <= 1e-9 * scale[0]


# ---------------------------------------------------------------------------
# refresh


def test_refresh_points_lie_in_their_cells_and_look_uniform():
    w, f = _small_field()
    G = 8
    dens = np.zeros((w.K, G ** 3))
    _, pts = oracle.occupancy_update(f, G, 0, 7, 0.95, 0.01, dens, want_points=True)
    cells = np.arange(G ** 3)
    c3 = np.stack([cells % G, (cells // G) % G, cells // (G * G)], -1)
    assert np.all(pts >= 0) and np.all(pts < 1)
    assert np.array_equal(np.floor(pts.astype(np.float64) * G).astype(int), np.broadcast_to(c3, pts.shape))
    xi = pts.astype(np.float64) * G - c3
    assert abs(xi.mean() - 0.5) < 0.01 and abs(xi.var() - 1 / 12) < 0.005
    # a new step or seed draws new points
    _, p2 = oracle.occupancy_update(f, G, 1, 7, 0.95, 0.01, dens, want_points=True)
    _, p3 = oracle.occupancy_update(f, G, 0, 8, 0.95, 0.01, dens, want_points=True)
    assert np.mean(pts == p2) < 1e-3 and np.mean(pts == p3) < 1e-3
    # the point of cell c is ((float)c + xi) / G with xi from Philox at (c, k, step, 0), key (seed, 0)
    r = oracle.philox4x32_10([37, 3, 0, 0], [7, 0])
    xi = (r[:3] >> 8).astype(np.float32) * np.float32(2.0 ** -24)
    c = c3[37].astype(np.float32)
    assert np.array_equal(pts[3, 37], ((c + xi) / np.float32(G)).astype(np.float32))


def _constant_field(w, level_values, mlp):
    """Tables constant per region (every entry of region k = level_values[k]):
    the encoded features are then the constants, wherever the point."""
    E = oracle.table_entries(w.level_res, w.log2_T)
    tables = np.broadcast_to(np.asarray(level_values, np.float64)[:, None, None], (w.K, E, w.F)).copy()
    return oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, tables, mlp)


def test_refresh_keeps_a_decaying_maximum_of_the_density():
    w = H.workload("grid8", L=4, log2_T=12)
    _, m = H.params(w)
    vals = np.linspace(-1.0, 1.0, w.K)
    f = _constant_field(w, vals, m.astype(np.float64))
    feat = np.zeros((w.K, w.mlp_in))
    feat[:, :w.L * w.F] = vals[:, None]
    sig = np.exp(oracle.mlp(f, np.arange(w.K, dtype=np.int32), feat)[:, 0])  # one density per region
    G = 3  # 27 cells: the top 5 bits of the one word stay clear
    dens = np.zeros((w.K, G ** 3))
    thr = float(np.median(sig))
    bits = oracle.occupancy_update(f, G, 0, 1, 0.5, thr, dens)
    np.testing.assert_allclose(dens, np.broadcast_to(sig[:, None], dens.shape), rtol=1e-12)
    want = np.where(sig > thr, (1 << 27) - 1, 0).astype(np.uint32)
    assert np.array_equal(bits[:, 0], want)
    # the estimate decays towards a lower density and never drops below it
    f_low = _constant_field(w, vals - 3.0, m.astype(np.float64))
    feat_low = feat.copy()
    feat_low[:, :w.L * w.F] -= 3.0
    sig_low = np.exp(oracle.mlp(f_low, np.arange(w.K, dtype=np.int32), feat_low)[:, 0])
    oracle.occupancy_update(f_low, G, 1, 1, 0.5, thr, dens)
    np.testing.assert_allclose(dens[:, 0], np.maximum(0.5 * sig, sig_low), rtol=1e-12)
    dens[:] = 10.0
    oracle.occupancy_update(f, G, 2, 1, 0.25, thr, dens)
    np.testing.assert_allclose(dens[:, 0], np.maximum(2.5, sig), rtol=1e-12)


def test_refresh_bits_are_the_thresholded_estimate():
    w, f = _small_field()
    G = 10  # 1000 cells: 31.25 words, a ragged last word
    dens = np.zeros((w.K, G ** 3))
    bits = oracle.occupancy_update(f, G, 0, 3, 0.95, 1.0, dens)
    on = np.unpackbits(bits.view(np.uint8).reshape(w.K, -1), axis=-1, bitorder="little").astype(bool)
    assert np.array_equal(on[:, :G ** 3], dens > 1.0)
    assert not on[:, G ** 3:].any()
    assert 0.05 < on.mean() < 0.95  # the threshold splits this field's cells
