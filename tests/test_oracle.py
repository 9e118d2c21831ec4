"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form, a brute force on tiny inputs, a library routine, a published constant,
or an invariant the paper states (Sec. 4.3: partitioned rendering equals the
single-pass render). No GPU is used here.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import synthetic as sy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_field(w, table_std=1.0, mlp_std=0.1):
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(w.mlp_in, w.W)
    t, m = sy.field_params(w, E, P, table_std, mlp_std)
    return oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, t, m)


def small_workload(name="grid8", L=None, log2_T=None, S=None):
    w = sy.workload(name)
    if L is not None:
        w.level_res = w.level_res[:L]
    if log2_T is not None:
        w.log2_T = log2_T
    if S is not None:
        w.S = S
    return w


# ---------------------------------------------------------------------------
# Geometry (Sec. 4.2): samples assigned by box; intervals never cross a face.

def test_slab_axis_aligned_closed_form():
    w = small_workload("unit")
    f = make_field(w)
    o = np.array([[-2.0, 0.1, 0.2], [0.1, 3.0, -0.2], [0.0, 0.0, 0.0]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    nseg, region, t0, t1, nint = oracle.segments(f, 64, o, d)
    assert list(nseg) == [1, 1, 1]
    # box [-0.5, 0.5]^3: enters at distance 1.5 and leaves at 2.5 (ray 0),
    # 2.5 and 3.5 (ray 1); ray 2 starts inside so t0 clamps to t_min = 0.
    assert (t0[0, 0], t1[0, 0]) == (1.5, 2.5)
    assert (t0[1, 0], t1[1, 0]) == (2.5, 3.5)
    assert (t0[2, 0], t1[2, 0]) == (0.0, 0.5)
    assert list(nint[:, 0]) == [64, 64, 64]


def test_miss_has_no_segments():
    w = small_workload("unit")
    f = make_field(w)
    o = np.array([[-2.0, 2.0, 0.0]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    nseg = oracle.segments(f, 64, o, d)[0]
    assert nseg[0] == 0
    out = oracle.render(f, 64, o, d, 0)
    assert out["n_samples"][0] == 0
    assert np.all(out["rgb"] == 0) and out["depth"][0] == 0 and out["opacity"][0] == 0 and out["tfinal"][0] == 1


@pytest.mark.parametrize("name", ["grid8", "city32"])
def test_segments_brute_force(name):
    """Region sequence of each ray equals a dense FP64 walk along the ray."""
    w = small_workload(name, L=2, log2_T=10)
    f = make_field(w)
    o, d = sy.workload_rays(w, 150)
    nseg, region, t0, t1, nint = oracle.segments(f, w.S, o, d)
    boxes = w.boxes.astype(np.float64)
    for r in range(len(o)):
        if nseg[r] == 0:
            continue
        ts = np.linspace(max(0.0, t0[r, 0] - 1.0), t1[r, nseg[r] - 1] + 1.0, 20001)
        x = o[r].astype(np.float64)[None] + ts[:, None] * d[r].astype(np.float64)[None]
        inside = np.all((x[:, None, :] > boxes[None, :, :3]) & (x[:, None, :] < boxes[None, :, 3:]), -1)
        hit_any = inside.any(1)
        first = inside.argmax(1)
        step = ts[1] - ts[0]
        segs = {int(region[r, k]): (float(t0[r, k]), float(t1[r, k])) for k in range(nseg[r])}
        assert len(segs) == nseg[r]  # no box visited twice
        # every walk point inside a box lies in that box's segment (FP32 ends)
        for i in np.nonzero(hit_any)[0]:
            k = int(first[i])
            assert k in segs, (r, k)
            assert segs[k][0] - 1e-5 <= ts[i] <= segs[k][1] + 1e-5, (r, k, ts[i], segs[k])
        # every segment longer than two walk steps is seen by the walk
        seen = set(first[hit_any].tolist())
        for k, (a, b) in segs.items():
            if b - a > 2 * step:
                assert k in seen, (r, k)
        for k in range(nseg[r]):
            assert t1[r, k] > t0[r, k]
            if k:
                assert t0[r, k] >= t1[r, k - 1]


def test_adjacent_segments_share_faces_bitwise():
    w = small_workload("grid8", L=2, log2_T=10)
    f = make_field(w)
    o, d = sy.workload_rays(w, 2000)
    nseg, region, t0, t1, nint = oracle.segments(f, w.S, o, d)
    pairs = 0
    for r in range(len(o)):
        for k in range(1, nseg[r]):
            # boxes of a 2x2x2 grid are face-adjacent: no gap, bitwise equal.
            assert t0[r, k] == t1[r, k - 1]
            pairs += 1
    assert pairs > 500


def test_intervals_partition_each_segment():
    """Intervals tile [t0_k, t1_k]; their midpoints lie in the region's box;
    no interval is longer than the grid step (tf - tn) / S."""
    w = small_workload("grid8", L=2, log2_T=10)
    f = make_field(w)
    o, d = sy.workload_rays(w, 300)
    max_int = w.S + w.max_segments - 1
    count, a, b, reg = oracle.intervals(f, w.S, o, d, max_int)
    nseg, region, t0, t1, nint = oracle.segments(f, w.S, o, d)
    boxes = w.boxes.astype(np.float64)
    for r in range(len(o)):
        n = count[r]
        assert n == nint[r, :nseg[r]].sum()
        assert n <= w.S + nseg[r] - 1
        if n == 0:
            continue
        assert np.all(b[r, :n] > a[r, :n])
        i = 0
        for k in range(nseg[r]):
            seg = slice(i, i + nint[r, k])
            assert a[r, i] == t0[r, k] and b[r, i + nint[r, k] - 1] == t1[r, k]
            assert np.all(a[r, i + 1:i + nint[r, k]] == b[r, i:i + nint[r, k] - 1])
            assert np.all(reg[r, seg] == region[r, k])
            s = np.sum(b[r, seg].astype(np.float64) - a[r, seg].astype(np.float64))
            assert abs(s - (float(t1[r, k]) - float(t0[r, k]))) < 1e-12
            i += nint[r, k]
        tm = 0.5 * (a[r, :n].astype(np.float64) + b[r, :n])
        x = o[r].astype(np.float64) + tm[:, None] * d[r].astype(np.float64)
        bx = boxes[reg[r, :n]]
        assert np.all(x >= bx[:, :3] - 1e-6) and np.all(x <= bx[:, 3:] + 1e-6)
        tn, tf = float(t0[r, 0]), float(t1[r, nseg[r] - 1])
        step = (tf - tn) / w.S
        lens = b[r, :n].astype(np.float64) - a[r, :n]
        assert np.all(lens <= step * (1 + 1e-5) + 4 * np.spacing(np.float32(tf)))


# ---------------------------------------------------------------------------
# Hash-grid encoding (App. A.1 adopts the Instant-NGP encoding per tile).

def _unit_cube_field(level_res, log2_T, table=None, F=2):
    boxes = np.array([[0, 0, 0, 1, 1, 1]], np.float32)
    E = oracle.table_entries(level_res, log2_T)
    P = oracle.mlp_params(32, 64)
    t = np.zeros((1, E, F)) if table is None else table
    return oracle.Field(boxes, level_res, log2_T, F, 32, 64, t, np.zeros((1, P)))


def test_hash_matches_published_primes():
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "instant_ngp_hash.txt"))]
    rows = [list(map(int, r)) for r in rows if r]
    assert len(rows) >= 10
    for log2_T, x, y, z, want in rows:
        N = 4096  # (N+1)^3 > T: a hashed level
        f = _unit_cube_field(np.array([N], np.int32), log2_T)
        assert not oracle.level_dense(f.level_res, log2_T, 0)
        # A point inside cell (x, y, z): corner 0 of that cell is vertex (x, y, z).
        p = (np.array([[x, y, z]], np.float64) + 0.25) / N
        _, idx = oracle.encode_points(f, [0], p.astype(np.float32), want_idx=True)
        assert idx[0, 0, 0] == want, (log2_T, x, y, z, idx[0, 0, 0], want)


def _dense_vertex_index_map(N, log2_T):
    cells = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij"), -1).reshape(-1, 3)
    f = _unit_cube_field(np.array([N], np.int32), log2_T)
    _, idx = oracle.encode_points(f, np.zeros(len(cells), np.int32), ((cells + 0.5) / N).astype(np.float32),
                                  want_idx=True)
    seen = {}
    for c, ids in zip(cells, idx[:, 0, :]):
        for e in range(8):
            v = (c[0] + (e & 1), c[1] + ((e >> 1) & 1), c[2] + ((e >> 2) & 1))
            assert seen.setdefault(v, ids[e]) == ids[e]
    return seen


def test_dense_level_is_a_bijection():
    N = 12
    assert oracle.level_dense(np.array([N], np.int32), 14, 0)
    seen = _dense_vertex_index_map(N, 14)
    assert len(seen) == (N + 1) ** 3
    assert sorted(seen.values()) == list(range((N + 1) ** 3))


def test_trilinear_reproduces_linear_function_on_dense_levels():
    level_res = np.array([7, 11], np.int32)
    log2_T = 14
    E = oracle.table_entries(level_res, log2_T)
    table = np.zeros((1, E, 2))
    coef = np.array([[0.3, -1.1, 2.0, 0.7], [-0.4, 0.25, 1.5, -2.0]])
    for l, N in enumerate(level_res):
        off = oracle.level_offset(level_res, log2_T, l)
        for v, i in _dense_vertex_index_map(int(N), log2_T).items():
            for j in range(2):
                table[0, off + i, j] = coef[j, :3] @ np.array(v, np.float64) + coef[j, 3]
    f = _unit_cube_field(level_res, log2_T, table)
    pts = sy.rng(5, "misc").uniform(0, 1, (500, 3)).astype(np.float32)
    feat = oracle.encode_points(f, np.zeros(500, np.int32), pts)
    for l, N in enumerate(level_res):
        p = pts.astype(np.float64) * N  # continuous lattice coordinate
        for j in range(2):
            np.testing.assert_allclose(feat[:, l * 2 + j], p @ coef[j, :3] + coef[j, 3], rtol=1e-6, atol=1e-6)
    assert np.all(feat[:, 2 * len(level_res):] == 0)


def test_partition_of_unity_and_continuity_on_hashed_levels():
    w = small_workload("grid8", L=16, log2_T=12)
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(32, 64)
    f1 = oracle.Field(w.boxes, w.level_res, w.log2_T, 2, 32, 64, np.ones((w.K, E, 2)), np.zeros((w.K, P)))
    pts = sy.rng(6, "misc").uniform(-0.99, 0.99, (300, 3)).astype(np.float32)
    reg = ((pts[:, 0] > 0).astype(int) + 2 * (pts[:, 1] > 0) + 4 * (pts[:, 2] > 0)).astype(np.int32)
    feat = oracle.encode_points(f1, reg, pts)
    np.testing.assert_allclose(feat, 1.0, atol=1e-12)
    f = make_field(w)
    fa = oracle.encode_points(f, reg, pts)
    fb = oracle.encode_points(f, reg, pts + np.float32(1e-5))
    lip = 2 * 8 * np.abs(f.tables).max() * w.level_res.max() * math.sqrt(3)
    assert np.abs(fa - fb).max() <= lip * 2e-5


def test_vertex_query_returns_table_entry():
    """At a lattice vertex the trilinear weights are one-hot."""
    level_res = np.array([4096], np.int32)
    log2_T = 19
    E = oracle.table_entries(level_res, log2_T)
    f = _unit_cube_field(level_res, log2_T, np.arange(2 * E, dtype=np.float64).reshape(1, -1, 2))
    feat, idx = oracle.encode_points(f, [0], (np.array([[3, 2, 0]], np.float64) / 4096).astype(np.float32), True)
    assert idx[0, 0, 0] == 455521  # golden hash of (3, 2, 0) at T = 2^19
    assert feat[0, 0] == 2 * 455521 and feat[0, 1] == 2 * 455521 + 1


# ---------------------------------------------------------------------------
# MLP: reduces to library GEMMs.

def test_mlp_equals_numpy_gemms():
    w = small_workload("grid8", L=16, log2_T=12)
    f = make_field(w)
    g = sy.rng(7, "misc")
    feat = g.standard_normal((256, 32))
    reg = g.integers(0, w.K, 256).astype(np.int32)
    o = oracle.mlp(f, reg, feat)
    Wd = 64
    for k in range(w.K):
        p = f.mlp[k]
        W1 = p[:32 * Wd].reshape(32, Wd)
        W2 = p[32 * Wd:32 * Wd + Wd * Wd].reshape(Wd, Wd)
        W3 = p[32 * Wd + Wd * Wd:].reshape(Wd, 4)
        sel = reg == k
        np.testing.assert_allclose(o[sel], np.maximum(np.maximum(feat[sel] @ W1, 0) @ W2, 0) @ W3, rtol=1e-12,
                                   atol=1e-12)


# ---------------------------------------------------------------------------
# Rendering (Eq. 1-8).

def test_constant_slab_closed_forms():
    n, sigma, L0, t0 = 37, 2.3, 1.7, 0.4
    dl = L0 / n
    tb = t0 + (np.arange(n) + 0.5) * dl
    c = np.array([0.2, 0.5, 0.9])
    single, part = oracle.render_samples(np.zeros(n, np.int32), np.full(n, sigma), np.tile(c, (n, 1)), tb,
                                         np.full(n, dl))
    T = math.exp(-sigma * L0)
    np.testing.assert_allclose(single[6], T, rtol=1e-13)
    np.testing.assert_allclose(single[4], 1 - T, rtol=1e-13)
    np.testing.assert_allclose(single[:3], c * (1 - T), rtol=1e-13)
    # depth: sum_i q^i (1-q) (t0 + (i+1/2) dl) with q = exp(-sigma dl), summed in closed form
    q = math.exp(-sigma * dl)
    s0 = (1 - q ** n) / (1 - q)
    s1 = q * (1 - n * q ** (n - 1) + (n - 1) * q ** n) / (1 - q) ** 2
    np.testing.assert_allclose(single[3], (1 - q) * ((t0 + dl / 2) * s0 + dl * s1), rtol=1e-12)
    np.testing.assert_allclose(part, single, rtol=1e-12, atol=1e-15)


def test_single_interval_distortion():
    s, _ = oracle.render_samples([0], [3.0], [[0.1, 0.2, 0.3]], [1.0], [0.25])
    wgt = 1 - math.exp(-0.75)
    np.testing.assert_allclose(s[5], wgt * wgt * 0.25 / 3, rtol=1e-14)


def _quadrature_distortion(w, tb, dl, m=400):
    """Brute force of Eq. 2 for step-function weights: each w_i spread
    uniformly over its interval, double integral by the midpoint rule."""
    xs, ws = [], []
    for wi, t, d in zip(w, tb, dl):
        xs.append(t - d / 2 + (np.arange(m) + 0.5) * d / m)
        ws.append(np.full(m, wi / m))
    x = np.concatenate(xs)
    ww = np.concatenate(ws)
    return float(np.sum(ww[:, None] * ww[None, :] * np.abs(x[:, None] - x[None, :])))


def test_distortion_matches_quadrature_brute_force():
    g = sy.rng(8, "misc")
    for trial in range(4):
        n = int(g.integers(2, 7))
        dl = g.uniform(0.05, 0.3, n)
        edges = 0.5 + np.concatenate([[0], np.cumsum(dl)])
        tb = 0.5 * (edges[:-1] + edges[1:])
        sig = g.uniform(0.0, 6.0, n)
        rgb = g.uniform(0, 1, (n, 3))
        segs = np.sort(g.integers(0, 3, n)).astype(np.int32)
        single, part = oracle.render_samples(segs, sig, rgb, tb, dl)
        acc = np.concatenate([[0], np.cumsum(sig * dl)])
        w = np.exp(-acc[:-1]) * (1 - np.exp(-sig * dl))
        brute = _quadrature_distortion(w, tb, dl)
        np.testing.assert_allclose(single[5], brute, rtol=2e-5)
        np.testing.assert_allclose(part[5], brute, rtol=2e-5)


def test_partitioned_equals_single_pass_random_partitions():
    g = sy.rng(9, "misc")
    for trial in range(50):
        n = int(g.integers(1, 40))
        dl = g.uniform(0.001, 0.2, n)
        edges = g.uniform(0, 2) + np.concatenate([[0], np.cumsum(dl)])
        tb = 0.5 * (edges[:-1] + edges[1:])
        sig = g.exponential(5.0, n)
        rgb = g.uniform(0, 1, (n, 3))
        segs = np.sort(g.integers(0, 6, n)).astype(np.int32)
        single, part = oracle.render_samples(segs, sig, rgb, tb, dl)
        np.testing.assert_allclose(part, single, rtol=1e-11, atol=1e-14)
        assert abs(single[4] + single[6] - 1) < 1e-13  # sum of weights = 1 - T_final


def test_cross_term_vanishes_with_one_weighted_segment():
    # Sec. 4.3: the S term is zero if only one segment has non-zero weight.
    tb = np.array([0.1, 0.3, 0.5, 0.7])
    dl = np.full(4, 0.2)
    rgb = np.full((4, 3), 0.5)
    sig = np.array([0.0, 0.0, 3.0, 1.0])
    p1 = oracle.render_local(sig[:2], rgb[:2], tb[:2], dl[:2])
    p2 = oracle.render_local(sig[2:], rgb[2:], tb[2:], dl[2:])
    assert p1[4] == 0 and p1[5] == 0
    out = oracle.composite(np.stack([p1, p2]))
    np.testing.assert_allclose(out[5], p2[6], rtol=1e-15)  # L = T_1^2 L_2 with T_1 = 1


@pytest.mark.parametrize("name", ["unit", "grid8", "city32"])
def test_field_render_partitioned_equals_single_pass(name):
    w = small_workload(name, L=None if name != "city32" else 6, log2_T=None if name != "city32" else 14)
    f = make_field(w)
    o, d = sy.workload_rays(w, 256)
    a = oracle.render(f, w.S, o, d, 0)
    b = oracle.render(f, w.S, o, d, 1)
    for k in ("rgb", "depth", "opacity", "dist", "tfinal"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(a["opacity"] + a["tfinal"], 1.0, atol=1e-13)
    assert (a["n_samples"] > 0).mean() > 0.5


def test_constant_field_renders_as_constant_slab():
    """A constant table gives constant features, hence constant sigma and colour:
    the whole ray is one homogeneous slab (Eq. 1 in closed form)."""
    w = small_workload("grid8", L=4, log2_T=12)
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(32, 64)
    _, mlp = sy.field_params(w, E, P)
    mlp = np.tile(mlp[:1], (w.K, 1))  # same MLP everywhere
    f = oracle.Field(w.boxes, w.level_res, w.log2_T, 2, 32, 64, np.full((w.K, E, 2), 0.7), mlp)
    o, d = sy.workload_rays(w, 64)
    out = oracle.render(f, w.S, o, d, 1)
    feat = np.zeros((1, 32))
    feat[0, :8] = 0.7
    raw = oracle.mlp(f, [0], feat)[0]
    sigma = math.exp(raw[0])
    c = 1 / (1 + np.exp(-raw[1:]))
    nseg, region, t0, t1, nint = oracle.segments(f, w.S, o, d)
    for r in range(len(o)):
        if nseg[r] == 0:
            continue
        length = float(np.sum(t1[r, :nseg[r]].astype(np.float64) - t0[r, :nseg[r]]))
        T = math.exp(-sigma * length)
        np.testing.assert_allclose(out["tfinal"][r], T, rtol=1e-10)
        np.testing.assert_allclose(out["rgb"][r], c * (1 - T), rtol=1e-10)


# ---------------------------------------------------------------------------
# Gradients: analytic reverse mode vs central finite differences.

def _grad_case(n_rays=256, S=128, L=16, log2_T=19):
    w = small_workload("grid8", L=L, log2_T=log2_T, S=S)
    f = make_field(w)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, n_rays, 77)
    o, d = o[sel], d[sel]
    tgt = sy.rng(78, "misc").uniform(0, 1, (n_rays, 3)).astype(np.float32)
    return w, f, o, d, tgt


@pytest.mark.slow
def test_analytic_gradient_matches_central_differences():
    """Per-coordinate central differences (eps = 1e-3, FP64) on 256 rays of
    the K=8 scene: table entries and MLP weights of two regions."""
    w, f, o, d, tgt = _grad_case()
    lam = 0.01
    L, gt, gm = oracle.loss_grad(f, w.S, o, d, tgt, lam)
    np.testing.assert_allclose(L, oracle.loss(f, w.S, o, d, tgt, lam), rtol=1e-13)
    g = sy.rng(79, "misc")
    tab = g.choice(np.flatnonzero(gt.reshape(-1)), 96, replace=False)
    mw = []
    for k in (0, 5):
        mw.extend(g.choice(np.flatnonzero(gm[k]) + k * f.P, 32, replace=False))
    mw = np.array(mw)
    which = np.concatenate([np.zeros(len(tab)), np.ones(len(mw))]).astype(np.int32)
    idx = np.concatenate([tab, mw]).astype(np.int64)
    an = np.concatenate([gt.reshape(-1)[tab], gm.reshape(-1)[mw]])
    # s = max |g| of the tensor the coordinate belongs to.
    scale = np.where(which == 0, np.abs(gt).max(), np.abs(gm).max())
    # At eps = 1e-3 a perturbation can push a sample across a ReLU kink, so a
    # few coordinates may miss the tight bound; all must meet a loose one.
    fd = oracle.fd_grad(f, w.S, o, d, tgt, lam, which, idx, eps=1e-3)
    err = np.abs(fd - an) / (np.abs(an) + scale)
    assert np.mean(err <= 1e-3) >= 0.95 and err.max() <= 1e-2, np.sort(err)[-5:]
    fd = oracle.fd_grad(f, w.S, o, d, tgt, lam, which, idx, eps=1e-5)
    err = np.abs(fd - an) / (np.abs(an) + scale)
    assert err.max() <= 1e-4, np.sort(err)[-5:]


def _directional(objective, f, g, gt, gm, eps):
    vt = g.standard_normal(f.tables.shape)
    vm = g.standard_normal(f.mlp.shape)
    fp = f.with_params(f.tables + eps * vt, f.mlp + eps * vm)
    fm = f.with_params(f.tables - eps * vt, f.mlp - eps * vm)
    return (objective(fp) - objective(fm)) / (2 * eps), np.sum(gt * vt) + np.sum(gm * vm)


def test_directional_derivative_of_loss():
    """Along random directions over every parameter (all tables, all MLP
    weights of all regions) the central difference matches <grad, v>. The
    step is tiny so that almost no ReLU changes side (a kink crossed by the
    perturbation costs ~1e-3 of agreement); a wrong term or sign misses by O(1)."""
    w, f, o, d, tgt = _grad_case(n_rays=64, S=32, L=6, log2_T=12)
    lam = 0.01
    _, gt, gm = oracle.loss_grad(f, w.S, o, d, tgt, lam)
    g = sy.rng(80, "misc")
    for trial in range(3):
        fd, an = _directional(lambda ff: oracle.loss(ff, w.S, o, d, tgt, lam), f, g, gt, gm, 1e-8)
        np.testing.assert_allclose(fd, an, rtol=5e-4)


@pytest.mark.parametrize("which", ["rgb", "depth", "opacity", "dist"])
def test_render_adjoint_per_output(which):
    """Adjoint for each output on its own (colour, depth, opacity,
    distortion), against the directional difference of sum(g * output)."""
    w, f, o, d, tgt = _grad_case(n_rays=32, S=24, L=5, log2_T=12)
    g = sy.rng(81, "misc")
    R = len(o)
    adj = {"rgb": np.zeros((R, 3)), "depth": np.zeros(R), "opacity": np.zeros(R), "dist": np.zeros(R)}
    adj[which] = g.uniform(0.5, 1.5, adj[which].shape)
    gt, gm = oracle.render_grad(f, w.S, o, d, adj["rgb"], adj["depth"], adj["opacity"], adj["dist"])

    def obj(field):
        r = oracle.render(field, w.S, o, d, 0)
        return float(np.sum(adj[which] * r[which]))

    fd, an = _directional(obj, f, g, gt, gm, 1e-7)
    np.testing.assert_allclose(fd, an, rtol=1e-3)


# ---------------------------------------------------------------------------
# Adam (Kingma & Ba) closed forms.

def test_adam_first_step_is_signed_lr():
    g = sy.rng(82, "misc")
    n = 1000
    grad = g.standard_normal(n)
    p0 = g.standard_normal(n)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    oracle.adam(p, m, v, grad.copy(), 1, 1e-2, 0.9, 0.99, 1e-15)
    # bias-corrected moments of one step are g and g^2: update = lr g / (|g| + eps)
    np.testing.assert_allclose(p, p0 - 1e-2 * grad / (np.abs(grad) + 1e-15), rtol=1e-13, atol=1e-16)


def test_adam_constant_gradient_keeps_constant_step():
    n = 10
    grad = np.linspace(-2, 3, n)
    p, m, v = np.zeros(n), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        before = p.copy()
        oracle.adam(p, m, v, grad.copy(), t, 1e-3, 0.9, 0.99, 1e-8)
        np.testing.assert_allclose(before - p, 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=1e-10, atol=1e-18)


# ---------------------------------------------------------------------------
# Blob target field.

def test_single_blob_against_gaussian_integrals():
    from scipy import integrate, special

    boxes = np.array([[-1, -1, -1, 1, 1, 1]], np.float32)
    lr = np.array([4], np.int32)
    E = oracle.table_entries(lr, 10)
    f = oracle.Field(boxes, lr, 10, 2, 32, 64, np.zeros((1, E, 2)), np.zeros((1, oracle.mlp_params(32, 64))))
    a, s = 2.0, 0.1
    blob = np.array([[0.0, 0.0, 0.0, s, a, 0.2, 0.6, 0.9]])
    o = np.array([[-3.0, 0.0, 0.0]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    rgb, depth, op = oracle.blob_render(f, 512, o, d, blob)
    tau = a * s * math.sqrt(2 * math.pi)  # int a exp(-t^2 / 2 s^2) dt over the line
    np.testing.assert_allclose(op[0], 1 - math.exp(-tau), rtol=1e-4)
    np.testing.assert_allclose(rgb[0], np.array([0.2, 0.6, 0.9]) * (1 - math.exp(-tau)), rtol=1e-4)
    # depth (Eq. 6): int t sigma(t) T(t) dt with the erf closed form of T(t)
    sig = lambda t: a * math.exp(-(t - 3) ** 2 / (2 * s * s))
    T = lambda t: math.exp(-a * s * math.sqrt(math.pi / 2) * (1 + special.erf((t - 3) / (s * math.sqrt(2)))))
    D = integrate.quad(lambda t: t * sig(t) * T(t), 2.0, 4.0, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    np.testing.assert_allclose(depth[0], D, rtol=1e-4)


# ---------------------------------------------------------------------------
# Workload configuration: the Instant-NGP level schedule values.

def test_level_schedule_values():
    assert list(sy.level_resolutions(16, 256, 8)) == [16, 23, 35, 52, 78, 115, 172, 256]
    assert list(sy.level_resolutions(16, 2048, 16)) == [16, 22, 30, 42, 58, 80, 111, 153, 212, 294, 406, 561, 776,
                                                         1072, 1482, 2048]
    r = sy.level_resolutions(16, 8192, 16)
    assert r[0] == 16 and r[-1] == 8192 and r[5] == 128 and r[10] == 1024
