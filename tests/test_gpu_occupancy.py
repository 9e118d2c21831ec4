"""Occupancy-grid skipping on the GPU (Sec. 5.1's spatial-skipping structure,
the cited Instant-NGP grid) against the FP64 oracle: renders, sample counts
and gradients with a sparse grid, the full grid as an exact no-op, and the
grid refresh (density estimates and bits) on the same seeded fields."""
import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import synthetic as sy

import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_16221_b300 import build

    build.build()


def _random_grid(K, G, p, seed):
    g = sy.rng(seed, "misc")
    bits = g.random((K, G ** 3)) < p
    pad = np.zeros((K, oracle.occupancy_words(G) * 32), bool)
    pad[:, :G ** 3] = bits
    return np.packbits(pad.reshape(K, -1, 32), axis=-1, bitorder="little").view(np.uint32).reshape(K, -1)


def _rounded(a, dtype):
    return torch.from_numpy(a).to(dtype).float().numpy()


def _render(gf, samp, o, d, for_backward=False):
    from paper_2404_16221_b300 import api

    ws = api.alloc_workspace(gf, samp, len(o), for_backward=for_backward)
    out = api.render_fwd(gf, samp, o, d, workspace=ws)
    api.check(ws)
    return {k: v.cpu().numpy() for k, v in out.items()}, ws


@pytest.mark.parametrize("mlp", [None, torch.bfloat16])
def test_full_grid_renders_bitwise_like_no_grid(mlp):
    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16 if mlp else None, mlp_dtype=mlp)
    o, d = sy.workload_rays(w, 2048, seed=3)
    samp = H.sampling(w)
    ref, _ = _render(gf, samp, o, d)
    for G in (1, 13, 64):
        gf.set_occupancy(np.full((w.K, oracle.occupancy_words(G)), 0xFFFFFFFF, np.uint32), G)
        out, _ = _render(gf, samp, o, d)
        for k in ref:
            assert np.array_equal(out[k], ref[k]), (G, k)


@pytest.mark.parametrize("name,G,p", [("grid8", 16, 0.3), ("grid8", 7, 0.6), ("city32", 32, 0.15)])
def test_sparse_grid_forward_matches_oracle(name, G, p):
    from paper_2404_16221_b300 import api

    w = H.workload(name, L=16, log2_T=14 if name == "grid8" else 15)
    t, m = H.params(w)
    occ = _random_grid(w.K, G, p, 41)
    gf = H.gpu_field(w, t, m)
    gf.set_occupancy(occ, G)
    of = H.oracle_field(w, t, m).with_occupancy(occ, G)
    o, d = sy.workload_rays(w, 2048, seed=42)
    samp = H.sampling(w)
    out, ws = _render(gf, samp, o, d)
    ref = oracle.render(of, w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    errs = H.assert_forward_close(out, ref, t_far)
    n_samples, _ = api.workspace_stats(ws)
    assert n_samples == int(ref["n_samples"].sum())
    assert n_samples < 0.9 * int(nint.sum())
    print(name, G, p, "kept %d of %d samples" % (n_samples, int(nint.sum())), errs)


@pytest.mark.parametrize("tab,mlp", [(torch.float16, torch.bfloat16), (torch.float32, torch.float16)])
def test_sparse_grid_mixed_forward_matches_oracle(tab, mlp):
    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    G = 16
    occ = _random_grid(w.K, G, 0.3, 43)
    gf = H.gpu_field(w, t, m, table_dtype=tab, mlp_dtype=mlp)
    gf.set_occupancy(occ, G)
    tq = _rounded(t, tab) if tab != torch.float32 else t
    of = H.oracle_field(w, tq, _rounded(m, mlp)).with_occupancy(occ, G)
    o, d = sy.workload_rays(w, 2048, seed=44)
    out, _ = _render(gf, H.sampling(w), o, d)
    ref = oracle.render(of, w.S, o, d, 1)
    assert np.abs(out["rgb"] - ref["rgb"]).max() <= 2e-3
    assert np.abs(out["opacity"] - ref["opacity"]).max() <= 2e-3


def _grad_close(g, ref, tol):
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    err = np.abs(g - ref) / max(np.abs(ref).max(), 1e-30)
    return float(np.mean(err > tol)), float(err.max())


def test_sparse_grid_backward_matches_oracle():
    """FP32 backward with skipping: every gradient entry within 1e-4 of
    max|ref| on the rays clear of ReLU kinks, and exactly zero on the entries
    that only skipped samples read."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    G = 16
    occ = _random_grid(w.K, G, 0.3, 45)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 1280, 46)
    o, d = o[sel].copy(), d[sel].copy()
    keep = H.kink_free(H.oracle_field(w, t, m).with_occupancy(occ, G), w.S, o, d)
    o, d = o[keep].copy(), d[keep].copy()
    R = len(o)
    g = sy.rng(47, "misc")
    gC, gD, gA, gL = g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R)
    gf = H.gpu_field(w, t, m)
    gf.set_occupancy(occ, G)
    samp = H.sampling(w)
    _, ws = _render(gf, samp, o, d, for_backward=True)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    of = H.oracle_field(w, t, m).with_occupancy(occ, G)
    gt_ref, gm_ref = oracle.render_grad(of, w.S, o, d, gC, gD, gA, gL)
    for a, b in ((gt.cpu().numpy(), gt_ref), (gm.cpu().numpy(), gm_ref)):
        ok, emax = H.grad_close(a, b, 1e-4)
        assert ok, emax
    gt_full, _ = oracle.render_grad(H.oracle_field(w, t, m), w.S, o, d, gC, gD, gA, gL)
    dead = (gt_ref.reshape(-1) == 0) & (gt_full.reshape(-1) != 0)
    assert dead.sum() > 1000 and not gt.cpu().numpy().reshape(-1)[dead].any()


@pytest.mark.parametrize("saved", [False, True])
def test_sparse_grid_mixed_backward_matches_oracle(saved):
    """Tensor-core backward with skipping, on the kink-free network of the
    mixed-backward structure test (every pre-activation well above zero):
    no entry off by more than 1e-2 of max|ref|."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    E = oracle.table_entries(w.level_res, w.log2_T)
    g = sy.rng(22, "misc")
    t = g.uniform(0.1, 1.0, (w.K, E, 2)).astype(np.float32)
    m = np.concatenate([g.uniform(0.0, 0.05, (w.K, 32 * 64)), g.uniform(0.0, 0.05, (w.K, 64 * 64)),
                        g.normal(0.0, 0.1, (w.K, 64 * 4))], 1).astype(np.float32)
    G = 16
    occ = _random_grid(w.K, G, 0.3, 48)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 2048, 49)
    o, d = o[sel].copy(), d[sel].copy()
    R = len(o)
    gg = sy.rng(50, "misc")
    gC, gD, gA, gL = gg.standard_normal((R, 3)), gg.standard_normal(R), gg.standard_normal(R), gg.standard_normal(R)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    gf.set_occupancy(occ, G)
    samp = H.sampling(w)
    if saved:
        samp = api.Sampling(samp.n_samples, samp.max_segments, flags=api.SAVE_FEATURES)
    _, ws = _render(gf, samp, o, d, for_backward=True)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    of = H.oracle_field(w, _rounded(t, torch.float16), _rounded(m, torch.bfloat16)).with_occupancy(occ, G)
    gt_ref, gm_ref = oracle.render_grad(of, w.S, o, d, gC, gD, gA, gL)
    for a, b in ((gt.cpu().numpy(), gt_ref), (gm.cpu().numpy(), gm_ref)):
        frac, emax = _grad_close(a, b, 1e-2)
        assert frac == 0.0, (frac, emax)


@pytest.mark.parametrize("G", [16, 9])
def test_refresh_matches_oracle(G):
    """Two refreshes of every region's grid: densities within 1e-5 relative of
    the FP64 oracle (same Philox points, FP32 field evaluation), bits equal
    wherever the density is not within that tolerance of the threshold."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    of = H.oracle_field(w, t, m)
    thr, decay = 1.0, 0.9
    grid = api.OccupancyGrid(w.K, G, decay=decay, threshold=thr, seed=12345678901)
    dens = np.zeros((w.K, G ** 3))
    for step in range(2):
        if step == 1:  # the field changes between refreshes
            gf.tables.mul_(0.5)
            of = of.with_params(of.tables * 0.5, of.mlp)
        grid.update(gf)
        bits = oracle.occupancy_update(of, G, step, 12345678901, decay, thr, dens)
        got = grid.density.cpu().numpy().astype(np.float64)
        rel = np.abs(got - dens) / np.abs(dens)
        assert rel.max() <= 1e-5, rel.max()
        on_gpu = np.unpackbits(grid.bits.cpu().numpy().view(np.uint32).view(np.uint8).reshape(w.K, -1), axis=-1,
                               bitorder="little").astype(bool)
        on_ref = np.unpackbits(bits.view(np.uint8).reshape(w.K, -1), axis=-1, bitorder="little").astype(bool)
        clear = np.ones_like(on_ref)
        clear[:, :G ** 3] = np.abs(dens - thr) > 1e-5 * thr
        assert np.array_equal(on_gpu[clear], on_ref[clear])
        assert 0.05 < on_ref.mean() < 0.95
    assert grid.updates == 2


def test_refresh_rejects_bad_arguments():
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gf16 = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    with pytest.raises(N.NerfxlError) as e:
        api.OccupancyGrid(w.K, 8).update(gf16)
    assert e.value.status == N.E_UNSUPPORTED
    gf = H.gpu_field(w, t, m)
    for G, decay in ((0, 0.9), (2048, 0.9), (8, 1.5)):
        grid = api.OccupancyGrid(w.K, max(G, 1) if G <= 1024 else 8, decay=decay)
        grid.G = G
        with pytest.raises(N.NerfxlError) as e:
            grid.update(gf)
        assert e.value.status == N.E_INVALID
    bad = H.gpu_field(w, t, m)
    bad.set_occupancy(np.zeros((w.K, 1), np.uint32), 1)
    bad.occ_res = 0
    with pytest.raises(N.NerfxlError) as e:
        api.render_fwd(bad, H.sampling(w), *sy.workload_rays(w, 16))
    assert e.value.status == N.E_INVALID


def _psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - b) ** 2))
    return 10 * np.log10(1.0 / max(mse, 1e-12))


def test_training_with_a_refreshed_grid():
    """Train a sparse K=8 blob scene (24 small blobs, about 10% of the volume
    above density 0.4) with the grid refreshed from the masters every 16 steps
    (all cells occupied for the first 64). The grid must not cost quality
    against training without it, and on held-out views it must drop most
    samples (the empty space the training has learned)."""
    from paper_2404_16221_b300 import api

    w = H.workload("train8", L=16, log2_T=16)
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(w.mlp_in, w.W)
    t0, m0 = sy.field_params(w, E, P, table_std=1e-4, mlp_std=0.1, table_init="uniform")
    blobs = sy.sparse_blobs(w.seed)
    o_tr, d_tr = sy.orbit_cameras(16, 3.0, 64, 64, 50.0, 0, 20)
    o_te, d_te = sy.orbit_cameras(4, 3.0, 64, 64, 50.0, 16, 20)
    of = H.oracle_field(w, t0, m0)
    tgt_tr = oracle.blob_render(of, w.S, o_tr, d_tr, blobs)[0].astype(np.float32)
    tgt_te = oracle.blob_render(of, w.S, o_te, d_te, blobs)[0]
    G = 32

    def run(with_grid: bool, steps: int = 400, batch: int = 8192):
        gf = H.gpu_field(w, t0.copy(), m0.copy())
        tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01)
        grid = api.OccupancyGrid(w.K, G, decay=0.95, threshold=0.01, seed=5) if with_grid else None
        if grid:
            grid.attach(gf)
        g = sy.rng(16, "batch")
        o_dev, d_dev = torch.from_numpy(o_tr).cuda(), torch.from_numpy(d_tr).cuda()
        tgt_dev = torch.from_numpy(tgt_tr).cuda()
        for s in range(steps):
            if grid and s >= 64 and s % 16 == 0:
                grid.update(gf)
            idx = torch.from_numpy(g.integers(0, len(o_tr), batch)).cuda()
            tr.step(o_dev[idx], d_dev[idx], tgt_dev[idx])
        samp = H.sampling(w)
        ws = api.alloc_workspace(gf, samp, len(o_te))
        out = api.render_fwd(gf, samp, o_te, d_te, workspace=ws)
        n_samples, _ = api.workspace_stats(ws)
        return _psnr(out["rgb"].cpu().numpy(), tgt_te), n_samples, grid.occupied_fraction() if grid else 1.0

    p_plain, n_plain, _ = run(False)
    p_grid, n_grid, occ = run(True)
    print("held-out PSNR without grid %.2f (%d samples), with grid %.2f (%d samples, %.1f%% cells occupied)"
          % (p_plain, n_plain, p_grid, n_grid, 100 * occ))
    assert p_grid > p_plain - 0.5
    assert n_grid < 0.25 * n_plain


@pytest.mark.parametrize("mixed", [False, True])
def test_empty_grid_renders_nothing_and_has_no_gradient(mixed):
    """Every cell clear: no sample survives, the rays render black with
    opacity 0, no chunk is formed, and the backward leaves every gradient 0."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16 if mixed else None,
                     mlp_dtype=torch.bfloat16 if mixed else None)
    G = 8
    gf.set_occupancy(np.zeros((w.K, oracle.occupancy_words(G)), np.uint32), G)
    o, d = sy.workload_rays(w, 1024, seed=71)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, len(o), for_backward=True)
    out = api.render_fwd(gf, samp, o, d, workspace=ws)
    api.check(ws)
    for k in ("rgb", "depth", "opacity", "dist"):
        assert not out[k].any(), k
    assert api.workspace_stats(ws) == (0, 0)
    gt, gm = api.render_bwd(gf, samp, o, d, ws, torch.ones(len(o), 3, device="cuda"))
    api.check(ws)
    assert not gt.any() and not gm.any()


def test_no_rays_with_a_grid():
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    gf.set_occupancy(np.full((w.K, oracle.occupancy_words(4)), 0xFFFFFFFF, np.uint32), 4)
    z = np.zeros((0, 3), np.float32)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, 0, for_backward=True)
    out = api.render_fwd(gf, samp, z, z, workspace=ws)
    assert out["rgb"].shape == (0, 3)
    api.render_bwd(gf, samp, z, z, ws, torch.zeros(0, 3, device="cuda"))
    api.check(ws)


def test_full_size_forward_with_grid_sampled_rays():
    """The bench's occupancy form in its launch configuration: the full grid8
    workload (2^18 rays, L=16, T=2^19) with the blob scene's 64^3 grid, FP32
    and FP16/BF16 fields; 1024 seeded rays checked against the oracle."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8")
    t, m = H.params(w)
    G = 64
    bits = sy.blob_occupancy(w.boxes, sy.sparse_blobs(w.seed), G, 0.4)
    o, d = sy.workload_rays(w)
    sel = sy.subset(len(o), 1024, 103)
    for tab, mlp in ((None, None), (torch.float16, torch.bfloat16)):
        gf = H.gpu_field(w, t, m, table_dtype=tab, mlp_dtype=mlp)
        gf.set_occupancy(bits, G)
        ws = api.alloc_workspace(gf, H.sampling(w), len(o))
        out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
        api.check(ws)
        got = {k: v.cpu().numpy()[sel] for k, v in out.items()}
        tq = t if tab is None else _rounded(t, tab)
        mq = m if mlp is None else _rounded(m, mlp)
        of = H.oracle_field(w, tq, mq).with_occupancy(bits, G)
        ref = oracle.render(of, w.S, o[sel], d[sel], 1)
        if tab is None:
            nseg, region, t0, t1, nint = oracle.segments(of, w.S, o[sel], d[sel])
            t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(sel))])
            H.assert_forward_close(got, ref, t_far)
        else:
            assert np.abs(got["rgb"] - ref["rgb"]).max() <= 2e-3
            assert np.abs(got["opacity"] - ref["opacity"]).max() <= 2e-3
        del gf, ws, out
        torch.cuda.empty_cache()


def test_refresh_from_mixed_trainer_masters():
    """Training with FP16 tables and a BF16 MLP keeps FP32 masters; the grid
    refresh reads them through Trainer.master_field() (no copy) and matches
    the oracle on the same FP32 values."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    tr = api.Trainer(gf, H.sampling(w), master_tables=torch.from_numpy(t), master_mlp=torch.from_numpy(m))
    mf = tr.master_field()
    assert mf.tables.data_ptr() == tr.tables.data_ptr() and mf.mlp.data_ptr() == tr.mlp.data_ptr()
    G = 8
    grid = api.OccupancyGrid(w.K, G, decay=0.9, threshold=1.0, seed=9)
    grid.update(mf)
    dens = np.zeros((w.K, G ** 3))
    oracle.occupancy_update(H.oracle_field(w, t, m), G, 0, 9, 0.9, 1.0, dens)
    assert (np.abs(grid.density.cpu().numpy() - dens) / dens).max() <= 1e-5
