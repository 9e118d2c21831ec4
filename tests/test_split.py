"""Split representation (App. A.1: per-region hash encoding and density MLP,
one colour MLP shared by all regions, conditioned on the view direction):
the oracle against what mathematics and the definition fix -- the spherical
harmonics are orthonormal on the sphere and obey the addition theorem, the
two MLPs equal plain numpy GEMMs, the colour block is shared across regions,
the density does not depend on the view direction, partitioned == single
pass, and the gradient (including the shared block) matches central
differences."""
import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import synthetic as sy

import helpers as H


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_sh_orthonormal_on_the_sphere():
    """Gauss-Legendre in cos(theta) x uniform in phi integrates every product
    Y_i Y_j (polynomials of degree <= 6) exactly."""
    xg, wg = np.polynomial.legendre.leggauss(8)
    phi = (np.arange(16) + 0.5) * 2 * np.pi / 16
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(16, 2 * np.pi / 16)[None, :]).reshape(-1)
    Y = oracle.sh4(dirs)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_addition_theorem():
    """sum_m Y_lm(a) Y_lm(b) = (2l + 1) / (4 pi) P_l(a . b) for every degree l."""
    g = np.random.default_rng(5)
    a = _unit(g.standard_normal((64, 3)))
    b = _unit(g.standard_normal((64, 3)))
    Ya, Yb = oracle.sh4(a), oracle.sh4(b)
    cos = np.sum(a * b, -1)
    for l in range(4):
        sl = slice(l * l, (l + 1) * (l + 1))
        lhs = np.sum(Ya[:, sl] * Yb[:, sl], -1)
        coef = np.zeros(l + 1)
        coef[l] = 1.0
        rhs = (2 * l + 1) / (4 * np.pi) * np.polynomial.legendre.legval(cos, coef)
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)
    # degree 0 is the constant 1 / (2 sqrt(pi)); degree 1 is linear in the direction
    assert np.allclose(Ya[:, 0], 0.5 / np.sqrt(np.pi))
    np.testing.assert_allclose(oracle.sh4(-a)[:, 1:4], -Ya[:, 1:4], atol=1e-15)


def split_field(name="grid8", L=4, log2_T=12, S=None, mlp_std=0.1):
    w = H.workload(name, L=L, log2_T=log2_T, S=S)
    t, _ = H.params(w)
    n = w.K * oracle.density_params(w.mlp_in, w.W) + oracle.color_params(w.W)
    m = sy.split_mlp_params(w, n, mlp_std)
    return w, t, m, oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, t.astype(np.float64),
                                 m.astype(np.float64), arch=1)


def _numpy_split(f, region, feat, dirs):
    W, I, K = f.W, f.mlp_in, f.K
    Pd = f.Pd
    out = np.zeros((len(feat), 4))
    c = f.mlp[K * Pd:]
    Wc1 = c[:32 * W].reshape(32, W)
    Wc2 = c[32 * W:32 * W + W * W].reshape(W, W)
    Wc3 = c[32 * W + W * W:].reshape(W, 4)
    sh = oracle.sh4(np.asarray(dirs, np.float64))
    for i, (k, x) in enumerate(zip(region, feat)):
        d = f.mlp[k * Pd:(k + 1) * Pd]
        Wd1 = d[:I * W].reshape(I, W)
        Wd2 = d[I * W:].reshape(W, 16)
        g = np.maximum(x @ Wd1, 0) @ Wd2
        xc = np.concatenate([g, sh[i]])
        h3 = np.maximum(np.maximum(xc @ Wc1, 0) @ Wc2, 0)
        out[i, 0] = g[0]
        out[i, 1:] = (h3 @ Wc3)[:3]
    return out


def test_split_mlp_equals_numpy_gemms_and_shares_the_colour_block():
    w, t, m, f = split_field()
    g = np.random.default_rng(7)
    n = 64
    region = g.integers(0, w.K, n).astype(np.int32)
    feat = g.standard_normal((n, w.mlp_in))
    dirs = _unit(g.standard_normal((n, 3))).astype(np.float32)
    got = oracle.mlp(f, region, feat, dirs)
    np.testing.assert_allclose(got, _numpy_split(f, region, feat, dirs), rtol=1e-12, atol=1e-12)
    # the density does not depend on the view direction; the colour does
    other = _unit(g.standard_normal((n, 3))).astype(np.float32)
    got2 = oracle.mlp(f, region, feat, other)
    assert np.array_equal(got[:, 0], got2[:, 0])
    assert np.abs(got[:, 1:] - got2[:, 1:]).max() > 1e-3
    # one colour block for all regions: perturbing it moves every region's colour
    m2 = f.mlp.copy()
    m2[w.K * f.Pd + 5] += 1.0  # Wc1[0][5]
    f2 = f.with_params(f.tables, m2)
    moved = np.abs(oracle.mlp(f2, region, feat, dirs)[:, 1:] - got[:, 1:]).max(1)
    for k in range(w.K):
        assert np.any(moved[region == k] > 0)


@pytest.mark.parametrize("name", ["grid8", "city32"])
def test_split_partitioned_equals_single_pass(name):
    w, t, m, f = split_field(name)
    o, d = sy.workload_rays(w, 128, seed=9)
    a, b = oracle.render(f, w.S, o, d, 0), oracle.render(f, w.S, o, d, 1)
    for k in ("rgb", "depth", "opacity", "dist", "tfinal"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-13)
    assert (a["opacity"] > 0.1).mean() > 0.3


def test_split_gradient_matches_central_differences():
    w, t, m, f = split_field("grid8", L=4, log2_T=12, S=32)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 48, 8)
    o, d = o[sel].copy(), d[sel].copy()
    tgt = sy.rng(9, "misc").uniform(0, 1, (len(o), 3)).astype(np.float32)
    lam = 0.01
    L, gt, gm = oracle.loss_grad(f, w.S, o, d, tgt, lam)
    np.testing.assert_allclose(L, oracle.loss(f, w.S, o, d, tgt, lam), rtol=1e-13)
    g = sy.rng(10, "misc")
    K, Pd = w.K, f.Pd
    tab = g.choice(np.flatnonzero(gt.reshape(-1)), 30, replace=False)
    dens = g.choice(np.flatnonzero(gm[:K * Pd]), 30, replace=False)
    col = K * Pd + g.choice(np.flatnonzero(gm[K * Pd:]), 30, replace=False)
    assert gm[K * Pd:].reshape(-1, 4)[-64:, 3].max() == 0  # the unused fourth colour output
    idx = np.concatenate([tab, dens, col]).astype(np.int64)
    which = np.concatenate([np.zeros(len(tab)), np.ones(len(dens) + len(col))]).astype(np.int32)
    an = np.concatenate([gt.reshape(-1)[tab], gm[dens], gm[col]])
    scale = np.where(which == 0, np.abs(gt).max(), np.abs(gm).max())
    fd = oracle.fd_grad(f, w.S, o, d, tgt, lam, which, idx, eps=1e-5)
    err = np.abs(fd - an) / (np.abs(an) + scale)
    assert err.max() <= 1e-4, np.sort(err)[-5:]
