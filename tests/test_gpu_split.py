"""Split representation on the GPU (App. A.1: per-region density MLP, one
colour MLP shared by all regions, conditioned on the view direction's
spherical harmonics) against the FP64 oracle: forward, backward (including
the shared colour block's gradient, reduced over every region's samples),
the training step, skipping and the grid refresh, and argument checks."""
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


def _split(name="grid8", L=16, log2_T=14, S=None):
    from paper_2404_16221_b300 import api, native as N

    w = H.workload(name, L=L, log2_T=log2_T, S=S)
    t, _ = H.params(w)
    n = w.K * oracle.density_params(w.mlp_in, w.W) + oracle.color_params(w.W)
    assert n == api.split_mlp_params(w.K, w.mlp_in, w.W)
    m = sy.split_mlp_params(w, n)
    of = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, t.astype(np.float64), m.astype(np.float64),
                      arch=1)
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t), torch.from_numpy(m), F=w.F,
                              mlp_in=w.mlp_in, width=w.W, arch=N.ARCH_SPLIT)
    assert int(N.lib().nerfxl_field_mlp_params(api.C_ref(gf.desc()))) == n
    return w, t, m, of, gf


_grad_ok = H.grad_close


def _kink_free_rays(of, w, n, seed, pool=16384):
    """Up to n seeded rays clear of ReLU kinks at FP32 precision. The split
    representation stacks three hidden layers (density, two colour layers),
    so only about one ray in ten qualifies; they are drawn from a larger
    pool."""
    o, d = sy.workload_rays(w, pool)
    sel = sy.subset(pool, pool // 2, seed)
    o, d = o[sel].copy(), d[sel].copy()
    keep = np.nonzero(H.kink_free(of, w.S, o, d))[0][:n]
    assert len(keep) >= min(n, 400), len(keep)
    return o[keep].copy(), d[keep].copy()


@pytest.mark.parametrize("name,n", [("grid8", 2048), ("city32", 1024), ("unit", 1024)])
def test_split_forward_matches_oracle(name, n):
    from paper_2404_16221_b300 import api

    w, t, m, of, gf = _split(name, L=16 if name != "unit" else None, log2_T=14 if name != "unit" else None)
    o, d = sy.workload_rays(w, n, seed=61)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, len(o))
    out = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, samp, o, d, workspace=ws).items()}
    api.check(ws)
    ref = oracle.render(of, w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    errs = H.assert_forward_close(out, ref, t_far)
    print(name, "split forward", errs)


def test_split_colour_depends_on_view_direction():
    """Two rays through the same point from opposite sides: the densities
    along the shared segment agree, the colours differ."""
    from paper_2404_16221_b300 import api

    w, t, m, of, gf = _split("unit", L=None, log2_T=None)
    o = np.array([[-2.0, 0.05, 0.1], [2.0, 0.05, 0.1]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]], np.float32)
    out = api.render_fwd(gf, H.sampling(w), o, d)
    op = out["opacity"].cpu().numpy()
    rgb = out["rgb"].cpu().numpy()
    ref = oracle.render(of, w.S, o, d, 1)
    np.testing.assert_allclose(op, ref["opacity"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(rgb, ref["rgb"], rtol=1e-5, atol=1e-6)
    assert abs(op[0] - op[1]) < 1e-3  # same densities, traversed in opposite order
    assert np.abs(rgb[0] - rgb[1]).max() > 1e-3


@pytest.mark.parametrize("save", [False, True])
def test_split_backward_matches_oracle(save):
    """FP32 split backward: with the forward's feature records
    (NERFXL_SAVE_FEATURES) or with the backward encoding and recording the
    features itself, both against the oracle's gradients."""
    import dataclasses

    from paper_2404_16221_b300 import api

    w, t, m, of, gf = _split()
    o, d = _kink_free_rays(of, w, 1024, 62)
    R = len(o)
    g = sy.rng(63, "misc")
    gC, gD, gA, gL = g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R)
    samp = dataclasses.replace(H.sampling(w), flags=api.SAVE_FEATURES if save else 0)
    ws = api.alloc_workspace(gf, samp, R, for_backward=True)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    gt_ref, gm_ref = oracle.render_grad(of, w.S, o, d, gC, gD, gA, gL)
    ok, e = _grad_ok(gt.cpu().numpy(), gt_ref)
    assert ok, ("tables", e)
    gm = gm.cpu().numpy()
    Pd = of.Pd
    for part, a, b in (("density", gm[:w.K * Pd], gm_ref[:w.K * Pd]), ("colour", gm[w.K * Pd:], gm_ref[w.K * Pd:])):
        ok, e = _grad_ok(a, b)
        assert ok, (part, e)
    assert np.abs(gm_ref[w.K * Pd:]).max() > 0


def test_split_training_step_matches_oracle():
    from paper_2404_16221_b300 import api

    w, t, m, of, gf = _split()
    o, d = _kink_free_rays(of, w, 1024, 64)
    tgt = sy.rng(65, "misc").uniform(0, 1, (len(o), 3)).astype(np.float32)
    trainer = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01)
    L = trainer.step(o, d, tgt).cpu().numpy()
    L_ref, gt_ref, gm_ref = oracle.loss_grad(of, w.S, o, d, tgt, 0.01)
    assert abs(L[0] - L_ref) <= 1e-5 * L_ref
    for g, ref in ((trainer.grad_tables, gt_ref), (trainer.grad_mlp, gm_ref)):
        ok, e = _grad_ok(g.cpu().numpy(), ref)
        assert ok, e
    H.assert_first_adam_step(gf.tables.cpu().numpy(), t, gt_ref, 1e-2, 1e-4)
    H.assert_first_adam_step(gf.mlp.cpu().numpy(), m, gm_ref, 1e-2, 1e-4)


def test_split_with_occupancy_and_refresh():
    from paper_2404_16221_b300 import api

    w, t, m, of, gf = _split()
    G = 16
    grid = api.OccupancyGrid(w.K, G, decay=0.9, threshold=1.0, seed=77)
    grid.update(gf)
    dens = np.zeros((w.K, G ** 3))
    bits = oracle.occupancy_update(of, G, 0, 77, 0.9, 1.0, dens)
    got = grid.density.cpu().numpy().astype(np.float64)
    assert (np.abs(got - dens) / dens).max() <= 1e-5
    on = np.unpackbits(bits.view(np.uint8), bitorder="little")
    assert 0.05 < on.mean() < 0.95
    grid.bits.copy_(torch.from_numpy(bits.view(np.int32)))  # the oracle's bits: identical decisions
    grid.attach(gf)
    ofo = of.with_occupancy(bits, G)
    o, d = sy.workload_rays(w, 2048, seed=66)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, len(o))
    out = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, samp, o, d, workspace=ws).items()}
    ref = oracle.render(ofo, w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    H.assert_forward_close(out, ref, t_far)
    assert api.workspace_stats(ws)[0] == int(ref["n_samples"].sum())


@pytest.mark.parametrize("save", [False, True])
def test_split_fp32_backward_with_occupancy_matches_oracle(save):
    """FP32 split backward over the kept samples of an occupancy grid (short,
    ragged chunks in the 256-row tiles of the tiled kernel), with and without
    the forward's feature records, against the oracle's gradient of the same
    skipped render; every entry within 1e-4 of max|ref| on kink-free rays."""
    import dataclasses

    from paper_2404_16221_b300 import api

    w, t, m, of, gf = _split()
    G = 16
    grid = api.OccupancyGrid(w.K, G, decay=0.9, threshold=1.0, seed=77)
    dens = np.zeros((w.K, G ** 3))
    bits = oracle.occupancy_update(of, G, 0, 77, 0.9, 1.0, dens)
    grid.bits.copy_(torch.from_numpy(bits.view(np.int32)))
    grid.attach(gf)
    ofo = of.with_occupancy(bits, G)
    o, d = _kink_free_rays(of, w, 1024, 93)
    R = len(o)
    g = sy.rng(94, "misc")
    gC, gD, gA, gL = g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R)
    samp = dataclasses.replace(H.sampling(w), flags=api.SAVE_FEATURES if save else 0)
    ws = api.alloc_workspace(gf, samp, R, for_backward=True)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    kept = api.workspace_stats(ws)[0]
    gt_ref, gm_ref = oracle.render_grad(ofo, w.S, o, d, gC, gD, gA, gL)
    assert 0 < kept < R * w.S
    for name, a, b in (("tables", gt.cpu().numpy(), gt_ref), ("mlp", gm.cpu().numpy(), gm_ref)):
        ok, e = _grad_ok(a, b)
        assert ok, (name, e)
        assert np.abs(b).max() > 0


def _rounded(a, dtype):
    return torch.from_numpy(a).to(dtype).float().numpy()


@pytest.mark.parametrize("tab,mlp", [(torch.float16, torch.bfloat16), (torch.float32, torch.float16),
                                     (torch.float32, torch.bfloat16)])
@pytest.mark.parametrize("name,n", [("grid8", 2048), ("city32", 1024)])
def test_split_tensor_core_forward_matches_oracle(tab, mlp, name, n):
    """The split representation on the tensor cores (five MMA layers per
    128-row tile): against the oracle on the rounded parameters the GPU reads,
    2e-3 absolute on RGB and opacity (activations rounded to the 16-bit type
    between layers)."""
    from paper_2404_16221_b300 import api, native as N

    w, t, m, of, _ = _split(name, L=16, log2_T=14 if name == "grid8" else 15)
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(tab),
                              torch.from_numpy(m).to(mlp), F=w.F, mlp_in=w.mlp_in, width=w.W, arch=N.ARCH_SPLIT)
    tq = _rounded(t, tab) if tab != torch.float32 else t
    ofq = of.with_params(tq.astype(np.float64), _rounded(m, mlp).astype(np.float64))
    o, d = sy.workload_rays(w, n, seed=67)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, len(o))
    out = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, samp, o, d, workspace=ws).items()}
    api.check(ws)
    ref = oracle.render(ofq, w.S, o, d, 1)
    e_rgb = np.abs(out["rgb"] - ref["rgb"]).max()
    e_op = np.abs(out["opacity"] - ref["opacity"]).max()
    full = oracle.render(of, w.S, o, d, 1)
    print(name, tab, mlp, "split tensor-core forward: rgb %.2e opacity %.2e (vs unrounded FP64 %.2e)"
          % (e_rgb, e_op, np.abs(out["rgb"] - full["rgb"]).max()))
    assert e_rgb <= 2e-3 and e_op <= 2e-3


@pytest.mark.parametrize("name,S", [("grid8", None), ("city32", None), ("grid8", 16)])
def test_split_mixed_backward_matches_oracle(name, S):
    """FP16 tables + BF16 MLPs: forward and backward on the tensor cores.
    Against the oracle on the rounded parameters, on the kink-free network
    (positive features and hidden weights): no entry off by more than 1e-2
    of max|ref| (activations and gradients enter the products as 16-bit
    values; measured 1.1e-3 for the tables, 2.2e-4 for the MLPs)."""
    from paper_2404_16221_b300 import api, native as N

    w = H.workload(name, L=16, log2_T=14, S=S)  # S = 16: every chunk shares its slot
    E = oracle.table_entries(w.level_res, w.log2_T)
    Pd, Pc = oracle.density_params(w.mlp_in, w.W), oracle.color_params(w.W)
    g = sy.rng(24, "misc")
    t = g.uniform(0.1, 1.0, (w.K, E, 2)).astype(np.float32)
    dens = np.concatenate([g.uniform(0.0, 0.05, (w.K, 32 * 64)), g.normal(0.0, 0.1, (w.K, 64 * 16))], 1)
    col = np.concatenate([g.uniform(0.0, 0.05, 32 * 64), g.uniform(0.0, 0.05, 64 * 64), g.normal(0.0, 0.1, 64 * 4)])
    m = np.concatenate([dens.reshape(-1), col]).astype(np.float32)
    assert m.size == w.K * Pd + Pc
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 2048, 68)
    o, d = o[sel].copy(), d[sel].copy()
    R = len(o)
    gg = sy.rng(69, "misc")
    gC, gD, gA, gL = gg.standard_normal((R, 3)), gg.standard_normal(R), gg.standard_normal(R), gg.standard_normal(R)
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(torch.float16),
                              torch.from_numpy(m).to(torch.bfloat16), arch=N.ARCH_SPLIT)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, R, for_backward=True)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    ofq = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, _rounded(t, torch.float16),
                       _rounded(m, torch.bfloat16), arch=1)
    gt_ref, gm_ref = oracle.render_grad(ofq, w.S, o, d, gC, gD, gA, gL)
    for which, a, b in (("tables", gt.cpu().numpy(), gt_ref), ("mlp", gm.cpu().numpy(), gm_ref)):
        err = np.abs(a.astype(np.float64).reshape(-1) - b.reshape(-1)) / np.abs(b).max()
        print("split mixed backward", name, which, "max err / max |grad| %.2e" % err.max())
        assert err.max() <= 1e-2, (which, err.max())


@pytest.mark.parametrize("tab", [torch.float16, torch.float32])
def test_split_saved_records_backward_equals_rebuilt(tab):
    """The split tensor-core backward reads the forward's per-tile records
    (features as the first MMA read them, region coordinates, interval, ray
    direction, chunk adjoints in tile order). Written by the training forward
    (NERFXL_SAVE_FEATURES) or rebuilt by the backward itself, the gradients
    agree up to the order of the FP32 atomic sums, and an occupancy grid
    changes nothing about that."""
    import dataclasses

    from paper_2404_16221_b300 import api, native as N

    w, t, m, of, _ = _split()
    o, d = sy.workload_rays(w, 2048, seed=72)
    R = len(o)
    g = sy.rng(73, "misc")
    adj = [torch.from_numpy(a.astype(np.float32)).cuda() for a in
           (g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R))]
    occ = None
    for with_grid in (False, True):
        runs = []
        for flags in (0, api.SAVE_FEATURES, 0, api.SAVE_FEATURES):
            gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(tab),
                                      torch.from_numpy(m).to(torch.bfloat16), arch=N.ARCH_SPLIT)
            if with_grid:
                if occ is None:  # every other cell of a 16^3 grid per region
                    occ = torch.from_numpy(np.full((w.K, 16 ** 3 // 32), 0x55555555, np.uint32).view(np.int32))
                gf.set_occupancy(occ.cuda(), 16)
            samp = dataclasses.replace(H.sampling(w), flags=flags)
            ws = api.alloc_workspace(gf, samp, R, for_backward=True)
            out = api.render_fwd(gf, samp, o, d, workspace=ws)
            gt, gm = api.render_bwd(gf, samp, o, d, ws, *adj)
            api.check(ws)
            runs.append((out["rgb"].cpu().numpy(), gt.cpu().numpy(), gm.cpu().numpy()))
        assert np.abs(runs[0][1]).max() > 0 and np.abs(runs[0][2]).max() > 0
        for other in runs[1:]:
            assert np.array_equal(runs[0][0], other[0])  # the forward is deterministic
            for a, b in zip(runs[0][1:], other[1:]):
                assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max(), (with_grid, np.abs(a - b).max())


def test_split_mixed_training_step_runs_and_refreshes_copies():
    """nerfxl_step on the split representation with FP16 tables and BF16 MLPs:
    the FP32 masters move by about lr where the gradient is clear, and the
    16-bit copies the forward reads are their rounding."""
    from paper_2404_16221_b300 import api, native as N

    w, t, m, of, _ = _split()
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(torch.float16),
                              torch.from_numpy(m).to(torch.bfloat16), arch=N.ARCH_SPLIT)
    tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=torch.from_numpy(t),
                     master_mlp=torch.from_numpy(m))
    o, d = sy.workload_rays(w, 2048, seed=70)
    tgt = sy.rng(71, "misc").uniform(0, 1, (len(o), 3)).astype(np.float32)
    L = tr.step(o, d, tgt).cpu().numpy()
    assert np.isfinite(L).all() and L[0] > 0
    assert torch.equal(gf.mlp, tr.mlp.to(torch.bfloat16)) and torch.equal(gf.tables, tr.tables.to(torch.float16))
    g = tr.grad_mlp.cpu().numpy()
    moved = tr.mlp.cpu().numpy() - m
    big = np.abs(g) > 1e-2 * np.abs(g).max()
    assert big.sum() > 100 and np.mean(np.abs(np.abs(moved[big]) - 1e-2) < 1e-4) > 0.99


def test_split_rejects_unbuilt_forms():
    from paper_2404_16221_b300 import api, native as N

    w, t, m, of, gf = _split()
    g16 = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(torch.float16),
                               torch.from_numpy(m).to(torch.bfloat16), F=w.F, mlp_in=w.mlp_in, width=w.W,
                               arch=N.ARCH_SPLIT)
    o, d = sy.workload_rays(w, 64)
    samp = H.sampling(w)
    q8 = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t),
                              torch.zeros(m.shape, dtype=torch.uint8), F=w.F, mlp_in=w.mlp_in, width=w.W,
                              arch=N.ARCH_SPLIT, mlp_scales=np.ones((w.K, 3), np.float32))
    ws8 = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    od = [torch.from_numpy(a).cuda() for a in (o, d)]
    out = torch.empty(len(o), 3, device="cuda")
    st = N.lib().nerfxl_render_fwd(api.C_ref(q8.desc()), api.C_ref(samp.desc()), len(o), N._ptr(od[0]),
                                   N._ptr(od[1]), N._ptr(out), N._ptr(out), N._ptr(out), None, N._ptr(ws8),
                                   ws8.numel(), N._stream())
    assert st == N.E_UNSUPPORTED
    gf.arch = 7
    with pytest.raises(N.NerfxlError) as e:
        api.render_fwd(gf, samp, o, d)
    assert e.value.status == N.E_INVALID


def _psnr(a, b):
    return 10 * np.log10(1.0 / max(float(np.mean((np.asarray(a, np.float64) - b) ** 2)), 1e-12))


def test_split_training_gains():
    """Train the split representation on the K=8 blob scene with the
    project's kernels: the training views are fitted closely and held-out
    PSNR rises well above the initial field's. (With 16 training views the
    view-dependent colour MLP fits them at ~38 dB but generalises to the 4
    held-out views less well than the view-independent fused MLP: ~19.8 vs
    ~23.3 dB after 400 steps.)"""
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("train8", L=16, log2_T=16)
    E = oracle.table_entries(w.level_res, w.log2_T)
    t0, _ = sy.field_params(w, E, oracle.mlp_params(w.mlp_in, w.W), table_std=1e-4, mlp_std=0.1,
                            table_init="uniform")
    n = w.K * oracle.density_params(w.mlp_in, w.W) + oracle.color_params(w.W)
    m0 = sy.split_mlp_params(w, n, 0.1)
    blobs = sy.blobs(200, w.seed)
    o_tr, d_tr = sy.orbit_cameras(16, 3.0, 64, 64, 50.0, 0, 20)
    o_te, d_te = sy.orbit_cameras(4, 3.0, 64, 64, 50.0, 16, 20)
    of = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, t0.astype(np.float64),
                      m0.astype(np.float64), arch=1)
    tgt_tr = oracle.blob_render(of, w.S, o_tr, d_tr, blobs)[0].astype(np.float32)
    tgt_te = oracle.blob_render(of, w.S, o_te, d_te, blobs)[0]
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t0), torch.from_numpy(m0),
                              arch=N.ARCH_SPLIT)
    tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01)
    g = sy.rng(16, "batch")
    o_dev, d_dev = torch.from_numpy(o_tr).cuda(), torch.from_numpy(d_tr).cuda()
    tgt_dev = torch.from_numpy(tgt_tr).cuda()
    for s in range(400):
        idx = torch.from_numpy(g.integers(0, len(o_tr), 8192)).cuda()
        tr.step(o_dev[idx], d_dev[idx], tgt_dev[idx])
    out = api.render_fwd(gf, H.sampling(w), o_te, d_te)
    init = _psnr(oracle.render(of, w.S, o_te, d_te, 1)["rgb"], tgt_te)
    trained = _psnr(out["rgb"].cpu().numpy(), tgt_te)
    fit = _psnr(api.render_fwd(gf, H.sampling(w), o_tr[:16384], d_tr[:16384])["rgb"].cpu().numpy(), tgt_tr[:16384])
    print("split representation PSNR: held-out initial %.2f, trained %.2f; training views %.2f" % (init, trained, fit))
    assert trained > init + 4.0
    assert fit > 33.0


def test_full_size_split_forward_sampled_rays():
    """The bench's split form in its launch configuration: the full grid8
    workload (2^18 rays, L=16, T=2^19), FP32 and FP16 tables + BF16 MLPs;
    1024 seeded rays checked against the oracle."""
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("grid8")
    t, _ = H.params(w)
    n = api.split_mlp_params(w.K, w.mlp_in, w.W)
    m = sy.split_mlp_params(w, n)
    o, d = sy.workload_rays(w)
    sel = sy.subset(len(o), 1024, 104)
    for tab, mlp in ((torch.float32, torch.float32), (torch.float16, torch.bfloat16)):
        gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(tab),
                                  torch.from_numpy(m).to(mlp), arch=N.ARCH_SPLIT)
        ws = api.alloc_workspace(gf, H.sampling(w), len(o))
        out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
        api.check(ws)
        got = {k: v.cpu().numpy()[sel] for k, v in out.items()}
        tq = t if tab == torch.float32 else _rounded(t, tab)
        mq = m if mlp == torch.float32 else _rounded(m, mlp)
        of = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, tq.astype(np.float64),
                          mq.astype(np.float64), arch=1)
        ref = oracle.render(of, w.S, o[sel], d[sel], 1)
        if tab == torch.float32:
            nseg, region, t0, t1, nint = oracle.segments(of, w.S, o[sel], d[sel])
            t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(sel))])
            H.assert_forward_close(got, ref, t_far)
        else:
            assert np.abs(got["rgb"] - ref["rgb"]).max() <= 2e-3
            assert np.abs(got["opacity"] - ref["opacity"]).max() <= 2e-3
        del gf, ws, out
        torch.cuda.empty_cache()


def test_split_mixed_backward_random_network_close_to_oracle():
    """On the seeded random network the 16-bit forward takes its own ReLU
    decisions near zero, so the gradient is compared as a whole: cosine
    > 0.999 and relative L2 error below 5% against the oracle on the rounded
    parameters, for the tables, the density blocks and the shared colour
    block."""
    from paper_2404_16221_b300 import api, native as N

    w, t, m, of, _ = _split()
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(torch.float16),
                              torch.from_numpy(m).to(torch.bfloat16), arch=N.ARCH_SPLIT)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 2048, 72)
    o, d = o[sel].copy(), d[sel].copy()
    R = len(o)
    gg = sy.rng(73, "misc")
    gC, gD, gA, gL = gg.standard_normal((R, 3)), gg.standard_normal(R), gg.standard_normal(R), gg.standard_normal(R)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, R, for_backward=True)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    ofq = of.with_params(_rounded(t, torch.float16).astype(np.float64), _rounded(m, torch.bfloat16).astype(np.float64))
    gt_ref, gm_ref = oracle.render_grad(ofq, w.S, o, d, gC, gD, gA, gL)
    Pd = of.Pd
    gm = gm.cpu().numpy()
    for name, a, b in (("tables", gt.cpu().numpy(), gt_ref), ("density", gm[:w.K * Pd], gm_ref[:w.K * Pd]),
                       ("colour", gm[w.K * Pd:], gm_ref[w.K * Pd:])):
        a = a.reshape(-1).astype(np.float64)
        b = b.reshape(-1)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        print("split mixed backward %s: cosine %.6f, relative L2 %.2e" % (name, cos, rel))
        assert cos > 0.999 and rel < 5e-2, (name, cos, rel)


def test_split_mixed_training_gains():
    """The split representation trained with FP16 tables, BF16 MLPs and FP32
    Adam (tensor-core forward and backward) fits the training views and rises
    well above the initial field on held-out views."""
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("train8", L=16, log2_T=16)
    E = oracle.table_entries(w.level_res, w.log2_T)
    t0, _ = sy.field_params(w, E, oracle.mlp_params(w.mlp_in, w.W), table_std=1e-4, mlp_std=0.1,
                            table_init="uniform")
    n = w.K * oracle.density_params(w.mlp_in, w.W) + oracle.color_params(w.W)
    m0 = sy.split_mlp_params(w, n, 0.1)
    blobs = sy.blobs(200, w.seed)
    o_tr, d_tr = sy.orbit_cameras(16, 3.0, 64, 64, 50.0, 0, 20)
    o_te, d_te = sy.orbit_cameras(4, 3.0, 64, 64, 50.0, 16, 20)
    of = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, t0.astype(np.float64),
                      m0.astype(np.float64), arch=1)
    tgt_tr = oracle.blob_render(of, w.S, o_tr, d_tr, blobs)[0].astype(np.float32)
    tgt_te = oracle.blob_render(of, w.S, o_te, d_te, blobs)[0]
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t0).to(torch.float16),
                              torch.from_numpy(m0).to(torch.bfloat16), arch=N.ARCH_SPLIT)
    tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=torch.from_numpy(t0),
                     master_mlp=torch.from_numpy(m0))
    g = sy.rng(16, "batch")
    o_dev, d_dev = torch.from_numpy(o_tr).cuda(), torch.from_numpy(d_tr).cuda()
    tgt_dev = torch.from_numpy(tgt_tr).cuda()
    for s in range(400):
        idx = torch.from_numpy(g.integers(0, len(o_tr), 8192)).cuda()
        tr.step(o_dev[idx], d_dev[idx], tgt_dev[idx])
    init = _psnr(oracle.render(of, w.S, o_te, d_te, 1)["rgb"], tgt_te)
    trained = _psnr(api.render_fwd(gf, H.sampling(w), o_te, d_te)["rgb"].cpu().numpy(), tgt_te)
    fit = _psnr(api.render_fwd(gf, H.sampling(w), o_tr[:16384], d_tr[:16384])["rgb"].cpu().numpy(), tgt_tr[:16384])
    print("split mixed training PSNR: held-out initial %.2f, trained %.2f; training views %.2f" % (init, trained, fit))
    assert trained > init + 4.0
    assert fit > 30.0


def test_split_mixed_backward_with_occupancy_matches_oracle():
    """The split representation's tensor-core backward over the kept samples
    of a sparse occupancy grid, on the kink-free network: no entry off by
    more than 1e-2 of max|ref| against the oracle with the same grid."""
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("grid8", L=16, log2_T=14)
    E = oracle.table_entries(w.level_res, w.log2_T)
    Pd, Pc = oracle.density_params(w.mlp_in, w.W), oracle.color_params(w.W)
    g = sy.rng(26, "misc")
    t = g.uniform(0.1, 1.0, (w.K, E, 2)).astype(np.float32)
    dens = np.concatenate([g.uniform(0.0, 0.05, (w.K, 32 * 64)), g.normal(0.0, 0.1, (w.K, 64 * 16))], 1)
    col = np.concatenate([g.uniform(0.0, 0.05, 32 * 64), g.uniform(0.0, 0.05, 64 * 64), g.normal(0.0, 0.1, 64 * 4)])
    m = np.concatenate([dens.reshape(-1), col]).astype(np.float32)
    G = 16
    bits = (g.integers(0, 2 ** 32, (w.K, oracle.occupancy_words(G)), dtype=np.uint64)
            & g.integers(0, 2 ** 32, (w.K, oracle.occupancy_words(G)), dtype=np.uint64)).astype(np.uint32)  # ~25%
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 2048, 74)
    o, d = o[sel].copy(), d[sel].copy()
    R = len(o)
    gg = sy.rng(75, "misc")
    gC, gD, gA, gL = gg.standard_normal((R, 3)), gg.standard_normal(R), gg.standard_normal(R), gg.standard_normal(R)
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).to(torch.float16),
                              torch.from_numpy(m).to(torch.bfloat16), arch=N.ARCH_SPLIT)
    gf.set_occupancy(bits, G)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, R, for_backward=True)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    dev = lambda a: torch.from_numpy(np.asarray(a, np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    ofq = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, _rounded(t, torch.float16),
                       _rounded(m, torch.bfloat16), arch=1).with_occupancy(bits, G)
    gt_ref, gm_ref = oracle.render_grad(ofq, w.S, o, d, gC, gD, gA, gL)
    for name, a, b in (("tables", gt.cpu().numpy(), gt_ref), ("mlp", gm.cpu().numpy(), gm_ref)):
        err = np.abs(a.astype(np.float64).reshape(-1) - b.reshape(-1)) / np.abs(b).max()
        print("split mixed backward with a grid", name, "max err / max |grad| %.2e" % err.max())
        assert err.max() <= 1e-2, (name, err.max())
