"""Mixed-precision forms of the forward render (tensor-core MLP).

The oracle renders the same field with the parameters the GPU actually reads
(tables rounded to FP16, MLP rounded to BF16/FP16, promoted to FP64); the
remaining difference is the rounding of activations to the MLP's 16-bit type
inside the tensor-core layers. Bound: 2e-3 absolute on RGB and opacity, 2e-3
t_far on depth. The error against the unrounded FP64 field is reported.
"""
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


def _rounded(a, dtype):
    return torch.from_numpy(a).to(dtype).float().numpy()


def test_tensor_core_mlp_smoke():
    """One small call first: the kernel completes (no timeout flag) and the
    image is finite."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=8, log2_T=14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, mlp_dtype=torch.bfloat16)
    o, d = sy.workload_rays(w, 256)
    ws = api.alloc_workspace(gf, H.sampling(w), len(o))
    out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
    api.check(ws)
    assert torch.isfinite(out["rgb"]).all()


@pytest.mark.parametrize("tab,mlp", [(torch.float32, torch.bfloat16), (torch.float32, torch.float16),
                                     (torch.float16, torch.bfloat16), (torch.float16, torch.float16)])
@pytest.mark.parametrize("name,n", [("grid8", 2048), ("city32", 1024)])
def test_mixed_forward_matches_oracle(tab, mlp, name, n):
    from paper_2404_16221_b300 import api

    w = H.workload(name, L=16, log2_T=None if name == "grid8" else 16)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=tab, mlp_dtype=mlp)
    o, d = sy.workload_rays(w, n)
    ws = api.alloc_workspace(gf, H.sampling(w), len(o))
    out = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, H.sampling(w), o, d, workspace=ws).items()}
    api.check(ws)
    tq = _rounded(t, tab) if tab != torch.float32 else t
    mq = _rounded(m, mlp)
    ref = oracle.render(H.oracle_field(w, tq, mq), w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(H.oracle_field(w, tq, mq), w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 1.0 for r in range(len(o))])
    e_rgb = np.abs(out["rgb"] - ref["rgb"]).max()
    e_op = np.abs(out["opacity"] - ref["opacity"]).max()
    e_dep = (np.abs(out["depth"] - ref["depth"]) / t_far).max()
    full = oracle.render(H.oracle_field(w, t, m), w.S, o, d, 1)
    print("%s tables=%s mlp=%s: vs rounded-parameter oracle rgb %.2e opacity %.2e depth/t_far %.2e; "
          "vs FP64 field rgb %.2e" % (name, tab, mlp, e_rgb, e_op, e_dep, np.abs(out["rgb"] - full["rgb"]).max()))
    assert e_rgb <= 2e-3 and e_op <= 2e-3 and e_dep <= 2e-3


def test_mixed_forward_deterministic():
    from paper_2404_16221_b300 import api

    w = H.workload("grid8")
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    o, d = sy.workload_rays(w, 16384)
    a = api.render_fwd(gf, H.sampling(w), o, d)
    b = api.render_fwd(gf, H.sampling(w), o, d)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def _grad_close(g, ref, tol):
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    err = np.abs(g - ref) / max(np.abs(ref).max(), 1e-30)
    return float(np.mean(err > tol)), float(err.max())


def _mixed_backward(w, t, m, tab, mlp, n=1024, seed=21):
    from paper_2404_16221_b300 import api

    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, n, 5)
    o, d = o[sel].copy(), d[sel].copy()
    R = len(o)
    g = sy.rng(seed, "misc")
    gC, gD, gA, gL = g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R)
    gf = H.gpu_field(w, t, m, table_dtype=tab, mlp_dtype=mlp)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, R, for_backward=True)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    dev = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()
    gt, gm = api.render_bwd(gf, samp, o, d, ws, dev(gC), dev(gD), dev(gA), dev(gL))
    api.check(ws)
    tq = _rounded(t, tab) if tab != torch.float32 else t
    gt_ref, gm_ref = oracle.render_grad(H.oracle_field(w, tq, _rounded(m, mlp)), w.S, o, d, gC, gD, gA, gL)
    return gt.cpu().numpy(), gm.cpu().numpy(), gt_ref, gm_ref


@pytest.mark.parametrize("S", [None, 16])
@pytest.mark.parametrize("tab,mlp", [(torch.float16, torch.bfloat16), (torch.float32, torch.float16)])
def test_mixed_backward_structure_matches_oracle(tab, mlp, S):
    """Tensor-core backward against the oracle on a network without ReLU
    kinks (positive features and hidden weights, so every pre-activation is
    well above zero): the 16-bit activations then only perturb values, by
    ~1e-3, and any wrong index, transpose or dropped term shows as O(1).
    With 16 samples per ray every chunk has at most 16 samples, so the
    records, chunk adjoints and render adjoint all run in slots shared by
    two or four chunks."""
    w = H.workload("grid8", L=16, log2_T=14, S=S)
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(w.mlp_in, w.W)
    g = sy.rng(22, "misc")
    t = g.uniform(0.1, 1.0, (w.K, E, 2)).astype(np.float32)
    m = np.concatenate([g.uniform(0.0, 0.05, (w.K, 32 * 64)), g.uniform(0.0, 0.05, (w.K, 64 * 64)),
                        g.normal(0.0, 0.1, (w.K, 64 * 4))], 1).astype(np.float32)
    gt, gm, gt_ref, gm_ref = _mixed_backward(w, t, m, tab, mlp)
    ft, et = _grad_close(gt, gt_ref, 1e-2)
    fm, em = _grad_close(gm, gm_ref, 1e-2)
    print("mixed backward (no kinks) tables=%s mlp=%s: tables frac>1e-2 %.1e max %.2e; mlp frac %.1e max %.2e"
          % (tab, mlp, ft, et, fm, em))
    assert ft == 0.0 and fm == 0.0


@pytest.mark.parametrize("tab,mlp", [(torch.float16, torch.bfloat16), (torch.float32, torch.float16)])
def test_mixed_backward_random_network_close_to_oracle(tab, mlp):
    """On a random network the 16-bit forward takes its own ReLU decisions
    (pre-activations within the 16-bit rounding of zero can flip), so its
    gradient differs from the FP64 one by those units' contributions. The
    gradient as a whole must still agree: cosine > 0.999, relative L2 error
    below 5% (BF16, measured 3.7%) / 2% (FP16)."""
    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    gt, gm, gt_ref, gm_ref = _mixed_backward(w, t, m, tab, mlp)
    for name, a, b in (("tables", gt, gt_ref), ("mlp", gm, gm_ref)):
        a = a.reshape(-1).astype(np.float64)
        b = b.reshape(-1)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        print("mixed backward tables=%s mlp=%s %s: cosine %.6f, relative L2 %.2e" % (tab, mlp, name, cos, rel))
        assert cos > 0.999 and rel < (5e-2 if mlp == torch.bfloat16 else 2e-2)


@pytest.mark.slow
def test_mixed_training_gains():
    """Training with FP16 tables, BF16 MLP and FP32 Adam masters (the c3 form)
    on the Gaussian-blob target: held-out PSNR rises well above the initial
    field's."""
    from paper_2404_16221_b300 import api

    w = H.workload("train8", L=16, log2_T=16)
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(w.mlp_in, w.W)
    t0, m0 = sy.field_params(w, E, P, table_std=1e-4, mlp_std=0.1, table_init="uniform")
    blobs = sy.blobs(200, w.seed)
    o_tr, d_tr = sy.orbit_cameras(16, 3.0, 64, 64, 50.0, 0, 20)
    o_te, d_te = sy.orbit_cameras(4, 3.0, 64, 64, 50.0, 16, 20)
    of = H.oracle_field(w, t0, m0)
    tgt_tr = oracle.blob_render(of, w.S, o_tr, d_tr, blobs)[0].astype(np.float32)
    tgt_te = oracle.blob_render(of, w.S, o_te, d_te, blobs)[0]
    gf = H.gpu_field(w, t0, m0, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=t0, master_mlp=m0)
    g = sy.rng(16, "batch")
    o_dev, d_dev, tgt_dev = (torch.from_numpy(a).cuda() for a in (o_tr, d_tr, tgt_tr))
    for s in range(400):
        idx = torch.from_numpy(g.integers(0, len(o_tr), 8192)).cuda()
        tr.step(o_dev[idx], d_dev[idx], tgt_dev[idx])
    out = api.render_fwd(gf, H.sampling(w), o_te, d_te)
    mse = float(np.mean((out["rgb"].cpu().numpy() - tgt_te) ** 2))
    psnr = 10 * np.log10(1 / mse)
    init = 10 * np.log10(1 / float(np.mean((oracle.render(of, w.S, o_te, d_te, 1)["rgb"] - tgt_te) ** 2)))
    print("mixed training held-out PSNR: initial %.2f, trained %.2f" % (init, psnr))
    assert psnr > init + 6.0
    # the compute copies track the FP32 masters
    assert torch.equal(gf.tables, tr.tables.to(torch.float16))
    assert torch.equal(gf.mlp, tr.mlp.to(torch.bfloat16))


def test_precision_sweep_city32():
    """Street/city precision sweep: the MLP in FP32 (CUDA cores), BF16, FP16
    and E4M3 with per-layer scales (tensor cores), tables FP32. Each variant's
    RGB and depth error against the FP64 oracle of the unrounded FP32 field is
    reported; FP32 must meet 1e-5, BF16/FP16 the 2e-3 RGB bound; E4M3 (3-bit
    mantissa activations) is an experiment and only sanity-bounded."""
    from paper_2404_16221_b300 import api

    w = H.workload("city32", L=16, log2_T=16)
    t, m = H.params(w)
    o, d = sy.workload_rays(w, 2048)
    of = H.oracle_field(w, t, m)
    ref = oracle.render(of, w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 1.0 for r in range(len(o))])
    rows = {}
    for name in ("fp32", "bf16", "fp16", "e4m3"):
        if name == "e4m3":
            q, sc = api.quantize_mlp_e4m3(torch.from_numpy(m))
            gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t), q, mlp_scales=sc)
        else:
            md = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16}[name]
            gf = H.gpu_field(w, t, m, mlp_dtype=md)
        ws = api.alloc_workspace(gf, H.sampling(w), len(o))
        out = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, H.sampling(w), o, d, workspace=ws).items()}
        api.check(ws)
        rows[name] = (np.abs(out["rgb"] - ref["rgb"]).max(), np.abs(out["rgb"] - ref["rgb"]).mean(),
                      (np.abs(out["depth"] - ref["depth"]) / t_far).max())
        print("precision sweep city32 mlp=%s: RGB max %.2e mean %.2e, depth/t_far max %.2e" % ((name,) + rows[name]))
    assert rows["fp32"][0] <= 1e-5 * 2 and rows["bf16"][0] <= 2e-3 and rows["fp16"][0] <= 2e-3
    assert rows["e4m3"][0] <= 0.1 and rows["e4m3"][1] <= 0.02


def test_e4m3_quantisation_matches_its_definition():
    """nerfxl_quantize_e4m3 against the definition written out in torch on the
    CPU: the same scales and the same E4M3 bytes, bit for bit; every weight
    within half an E4M3 step of its quantised value."""
    from paper_2404_16221_b300 import api

    w = H.workload("city32", L=16, log2_T=14)
    _, m = H.params(w)
    m[3, :10] = 0.0  # a few zeros, and one layer of one region all zero (scale floor)
    m[5, 32 * 64 + 64 * 64:] = 0.0
    q, sc = api.quantize_mlp_e4m3(torch.from_numpy(m))
    q_ref, sc_ref = H.e4m3_definition(m)
    assert torch.equal(sc.cpu(), sc_ref)
    assert torch.equal(q.cpu(), q_ref)
    deq = H.e4m3_dequantize(q, sc).numpy()
    v = np.abs(m) / np.repeat(sc_ref.numpy(), H.MLP_LAYER_SIZES, axis=1)
    normal = v >= 2.0 ** -6  # E4M3 normals: 3 mantissa bits, half a step is 2^-4 relative
    assert np.all(np.abs(deq - m)[normal] <= 2.0 ** -4 * np.abs(m)[normal] * (1 + 1e-6))


def test_e4m3_matches_oracle_on_dequantized_weights():
    """E4M3 forward against the oracle run on the dequantized weights: what
    is left is the E4M3 rounding of activations (3 mantissa bits)."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    q, sc = api.quantize_mlp_e4m3(torch.from_numpy(m))
    mq = H.e4m3_dequantize(q, sc).numpy()
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t), q, mlp_scales=sc)
    o, d = sy.workload_rays(w, 2048)
    ws = api.alloc_workspace(gf, H.sampling(w), len(o))
    out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
    api.check(ws)
    ref = oracle.render(H.oracle_field(w, t, mq), w.S, o, d, 1)
    e = np.abs(out["rgb"].cpu().numpy() - ref["rgb"])
    print("e4m3 vs dequantized-weight oracle: RGB max %.2e mean %.2e" % (e.max(), e.mean()))
    assert e.max() <= 0.05 and e.mean() <= 0.01


def test_saved_features_backward_equals_recompute():
    """With NERFXL_SAVE_FEATURES the backward reads the features the forward
    fed its first MMA instead of gathering again; the gradient is the same
    (up to the order of the FP32 atomic sums)."""
    import dataclasses

    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    o, d = sy.workload_rays(w, 2048)
    R = len(o)
    g = sy.rng(23, "misc")
    adj = [torch.from_numpy(a.astype(np.float32)).cuda() for a in
           (g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R))]
    grads = []
    for flags in (0, api.SAVE_FEATURES):
        gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
        samp = dataclasses.replace(H.sampling(w), flags=flags)
        ws = api.alloc_workspace(gf, samp, R, for_backward=True)
        api.render_fwd(gf, samp, o, d, workspace=ws)
        gt, gm = api.render_bwd(gf, samp, o, d, ws, *adj)
        api.check(ws)
        grads.append((gt.cpu().numpy(), gm.cpu().numpy()))
    for a, b in zip(grads[0], grads[1]):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_mixed_backward_repeatable():
    """Four mixed backward passes (fresh workspaces, with and without the
    forward's records) agree up to the order of the FP32 atomic sums. A tile
    whose MMA read a half-written weight tile or stage shows up here as a
    percent-level difference."""
    import dataclasses

    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    o, d = sy.workload_rays(w, 2048)
    R = len(o)
    g = sy.rng(29, "misc")
    adj = [torch.from_numpy(a.astype(np.float32)).cuda() for a in
           (g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R))]
    runs = []
    for flags in (0, api.SAVE_FEATURES, 0, api.SAVE_FEATURES):
        gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
        samp = dataclasses.replace(H.sampling(w), flags=flags)
        ws = api.alloc_workspace(gf, samp, R, for_backward=True)
        api.render_fwd(gf, samp, o, d, workspace=ws)
        gt, gm = api.render_bwd(gf, samp, o, d, ws, *adj)
        api.check(ws)
        runs.append((gt.cpu().numpy(), gm.cpu().numpy()))
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


@pytest.mark.parametrize("n", [1, 3, 37])
def test_mixed_backward_small_batches(n):
    """Batches with far fewer tiles than CTAs (most CTAs get no tile; a
    region may hold a single padded tile) against the oracle, on the
    kink-free network of the structure test."""
    w = H.workload("grid8", L=16, log2_T=14)
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(w.mlp_in, w.W)
    g = sy.rng(22, "misc")
    t = g.uniform(0.1, 1.0, (w.K, E, 2)).astype(np.float32)
    m = np.concatenate([g.uniform(0.0, 0.05, (w.K, 32 * 64)), g.uniform(0.0, 0.05, (w.K, 64 * 64)),
                        g.normal(0.0, 0.1, (w.K, 64 * 4))], 1).astype(np.float32)
    gt, gm, gt_ref, gm_ref = _mixed_backward(w, t, m, torch.float16, torch.bfloat16, n=n, seed=30 + n)
    ft, et = _grad_close(gt, gt_ref, 1e-2)
    fm, em = _grad_close(gm, gm_ref, 1e-2)
    print("mixed backward, %d rays: tables frac>1e-2 %.1e max %.2e; mlp frac %.1e max %.2e" % (n, ft, et, fm, em))
    assert ft == 0.0 and fm == 0.0
