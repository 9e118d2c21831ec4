"""Forward parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer decisions (segments, interval edges, hash indices) must match bit for
bit; floating outputs within the FP32 tolerance |gpu - ref| <= 1e-5 (|ref| + s).
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


def _edge_rays(w, n):
    """Workload rays plus ragged cases: misses, rays starting inside a box,
    axis-parallel rays, and rays along shared faces."""
    o, d = sy.workload_rays(w, n)
    lo, hi = w.boxes[:, :3].min(0), w.boxes[:, 3:].max(0)
    c = 0.5 * (lo + hi)
    extra_o = [c + 3 * (hi - lo), c, c - np.array([0, 0, 2 * (hi[2] - lo[2])], np.float32),
               np.array([lo[0] - 1, c[1], c[2]], np.float32), np.array([lo[0] - 1, lo[1] + 1e-3, c[2]], np.float32)]
    extra_d = [np.array([1, 0, 0], np.float32), np.array([0.3, 0.5, 0.8], np.float32),
               np.array([0, 0, 1], np.float32), np.array([1, 0, 0], np.float32), np.array([1, 0, 0], np.float32)]
    extra_d = [v / np.linalg.norm(v) for v in extra_d]
    return (np.concatenate([o, np.array(extra_o, np.float32)]),
            np.concatenate([d, np.array(extra_d, np.float32)]))


@pytest.mark.parametrize("name", ["unit", "grid8", "city32"])
def test_segments_bit_exact(name):
    w = H.workload(name, L=4, log2_T=12)
    t, m = H.params(w)
    of = H.oracle_field(w, t, m)
    gf = H.gpu_field(w, t, m)
    o, d = _edge_rays(w, 3000)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    from paper_2404_16221_b300 import api

    gn, gr, g0, g1, gi = [x.cpu().numpy() for x in api.debug_segments(gf, H.sampling(w), o, d, w.K)]
    np.testing.assert_array_equal(gn, nseg)
    for r in range(len(o)):
        k = nseg[r]
        np.testing.assert_array_equal(gr[r, :k], region[r, :k])
        np.testing.assert_array_equal(g0[r, :k].view(np.uint32), t0[r, :k].view(np.uint32))
        np.testing.assert_array_equal(g1[r, :k].view(np.uint32), t1[r, :k].view(np.uint32))
        np.testing.assert_array_equal(gi[r, :k], nint[r, :k])


@pytest.mark.parametrize("name", ["unit", "grid8", "city32"])
def test_intervals_and_hash_indices_bit_exact(name):
    w = H.workload(name)
    t, m = H.params(w)
    of = H.oracle_field(w, t, m)
    gf = H.gpu_field(w, t, m)
    o, d = _edge_rays(w, 96)
    max_int = w.S + w.max_segments - 1
    from paper_2404_16221_b300 import api

    cnt, a, b, reg = oracle.intervals(of, w.S, o, d, max_int)
    idx = oracle.hash_indices(of, w.S, o, d, max_int)
    gc, ga, gb, gr, gidx, gfeat, graw = api.debug_samples(gf, H.sampling(w), o, d, max_int, True, True, True)
    gc, ga, gb, gr = gc.cpu().numpy(), ga.cpu().numpy(), gb.cpu().numpy(), gr.cpu().numpy()
    gidx = gidx.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(gc, cnt)
    mask = np.arange(max_int)[None, :] < cnt[:, None]
    np.testing.assert_array_equal(ga[mask].view(np.uint32), a[mask].view(np.uint32))
    np.testing.assert_array_equal(gb[mask].view(np.uint32), b[mask].view(np.uint32))
    np.testing.assert_array_equal(gr[mask], reg[mask])
    np.testing.assert_array_equal(gidx[mask], idx[mask])
    # features and raw MLP outputs (FP32 vs FP64)
    tb = 0.5 * (a + b)
    x = (o[:, None, :] + tb[..., None].astype(np.float32) * d[:, None, :]).astype(np.float32)
    feat = oracle.encode_points(of, reg[mask], x[mask])
    gfe = gfeat.cpu().numpy()[mask]
    assert H.rel_err(gfe, feat, 1.0) < 1e-5
    raw = oracle.mlp(of, reg[mask], feat)
    assert H.rel_err(graw.cpu().numpy()[mask], raw, 1.0) < 1e-5


@pytest.mark.parametrize("name,n", [("unit", 4096), ("grid8", 2048), ("city32", 1024)])
def test_forward_matches_oracle(name, n):
    w = H.workload(name, L=None if name != "city32" else 16, log2_T=None if name != "city32" else 16)
    t, m = H.params(w)
    of = H.oracle_field(w, t, m)
    gf = H.gpu_field(w, t, m)
    o, d = _edge_rays(w, n)
    from paper_2404_16221_b300 import api

    ws = api.alloc_workspace(gf, H.sampling(w), len(o))
    out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
    api.check(ws)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.render(of, w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    errs = H.assert_forward_close(out, ref, t_far)
    # misses are exactly black
    miss = nseg == 0
    assert miss.any()
    assert np.all(out["rgb"][miss] == 0) and np.all(out["opacity"][miss] == 0) and np.all(out["depth"][miss] == 0)
    print(name, errs)


def test_forward_is_deterministic():
    w = H.workload("grid8", L=8)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    o, d = sy.workload_rays(w, 8192)
    from paper_2404_16221_b300 import api

    a = api.render_fwd(gf, H.sampling(w), o, d)
    b = api.render_fwd(gf, H.sampling(w), o, d)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_empty_batch():
    w = H.workload("unit")
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    from paper_2404_16221_b300 import api

    out = api.render_fwd(gf, H.sampling(w), np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    assert out["rgb"].shape == (0, 3)


def test_overflow_is_reported():
    """A ray crossing more regions than max_segments sets the device flag."""
    w = H.workload("grid8", L=4, log2_T=12)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    from paper_2404_16221_b300 import api, native as N

    samp = api.Sampling(w.S, 1)
    o = np.array([[-2.0, -0.5, -0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)  # crosses two boxes
    ws = api.alloc_workspace(gf, samp, 1)
    api.render_fwd(gf, samp, o, d, workspace=ws)
    with pytest.raises(N.NerfxlError) as e:
        api.check(ws)
    assert e.value.status == N.E_OVERFLOW


@pytest.mark.parametrize("name", ["grid8"])
def test_full_size_forward_sampled_rays(name):
    """The full workload (2^18 rays) in one launch; a seeded sample of rays
    is checked against the oracle ray by ray."""
    w = H.workload(name)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    o, d = sy.workload_rays(w)
    from paper_2404_16221_b300 import api

    ws = api.alloc_workspace(gf, H.sampling(w), len(o))
    out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
    api.check(ws)
    sel = sy.subset(len(o), 2048, 99)
    of = H.oracle_field(w, t, m)
    ref = oracle.render(of, w.S, o[sel], d[sel], 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o[sel], d[sel])
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(sel))])
    got = {k: v.cpu().numpy()[sel] for k, v in out.items()}
    H.assert_forward_close(got, ref, t_far)


@pytest.mark.slow
def test_full_size_city32_sampled_rays():
    """The full street/city workload (K=32, T=2^21, 2^20 rays, S=256) in the
    launch configuration the bench times; 512 seeded rays checked against the
    oracle, for the FP32 path (1e-5) and for FP16 tables + BF16 MLP (2e-3
    absolute, against the oracle on the rounded parameters)."""
    from paper_2404_16221_b300 import api

    w = H.workload("city32")
    t, m = H.params(w)
    o, d = sy.workload_rays(w)
    sel = sy.subset(len(o), 512, 101)
    for tab, mlp in ((torch.float32, torch.float32), (torch.float16, torch.bfloat16)):
        gf = H.gpu_field(w, t, m, table_dtype=tab, mlp_dtype=mlp)
        ws = api.alloc_workspace(gf, H.sampling(w), len(o))
        out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
        api.check(ws)
        got = {k: v.cpu().numpy()[sel] for k, v in out.items()}
        del gf, ws, out
        torch.cuda.empty_cache()
        tq = t if tab == torch.float32 else torch.from_numpy(t).to(tab).float().numpy()
        mq = m if mlp == torch.float32 else torch.from_numpy(m).to(mlp).float().numpy()
        of = H.oracle_field(w, tq, mq)
        ref = oracle.render(of, w.S, o[sel], d[sel], 1)
        nseg, region, t0, t1, nint = oracle.segments(of, w.S, o[sel], d[sel])
        t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(sel))])
        del of
        if tab == torch.float32:
            H.assert_forward_close(got, ref, t_far)
        else:
            assert np.abs(got["rgb"] - ref["rgb"]).max() <= 2e-3
            assert np.abs(got["opacity"] - ref["opacity"]).max() <= 2e-3


@pytest.mark.parametrize("form", ["fp32", "mixed"])
def test_paired_slots_render_as_alone(form):
    """With 24 samples per ray over the eight regions almost every chunk has
    at most 16 samples and shares its warp with another ray's chunk. A ray's
    colour must not depend on that partner: rendered in the full batch, in
    a batch of every third ray, and in reversed order, each ray comes out
    bit for bit the same (the half- and quarter-warp scans equal whole-warp ones with
    empty lanes), and the FP32 form matches the oracle."""
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=8, log2_T=14, S=24)
    t, m = H.params(w)
    dt = (None, None) if form == "fp32" else (torch.float16, torch.bfloat16)
    gf = H.gpu_field(w, t, m, table_dtype=dt[0], mlp_dtype=dt[1])
    o, d = sy.workload_rays(w, 6144)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, len(o))
    full = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, samp, o, d, workspace=ws).items()}
    api.check(ws)
    n_samples, n_chunks = api.workspace_stats(ws)
    assert n_samples < 16 * n_chunks  # most chunks fit half a slot or a quarter
    for sel in (np.arange(0, len(o), 3), np.arange(len(o))[::-1].copy()):
        part = api.render_fwd(gf, samp, o[sel].copy(), d[sel].copy())
        for k in full:
            assert np.array_equal(part[k].cpu().numpy(), full[k][sel]), k
    if form == "fp32":
        sub = np.arange(0, len(o), 12)
        of = H.oracle_field(w, t, m)
        ref = oracle.render(of, w.S, o[sub], d[sub], 1)
        nseg, region, t0, t1, nint = oracle.segments(of, w.S, o[sub], d[sub])
        t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(sub))])
        H.assert_forward_close({k: v[sub] for k, v in full.items()}, ref, t_far)


@pytest.mark.parametrize("name", ["unit", "grid8", "city32"])
def test_fp32_forward_kernels_agree_bitwise(name):
    """The fused FP32 field has two kernels: tiled products over 128-row
    sub-tiles (region tables that L2 keeps) and one sample per thread (larger
    tables; the switch is the level-grouped gather's table-size threshold).
    Both take every product in the order of a per-sample dot product, so
    their outputs are identical bit for bit, and the FP32 feature records
    each writes for the backward give the same gradients (up to the order of
    the FP32 atomic sums); the tiled form also matches the oracle."""
    import dataclasses

    from paper_2404_16221_b300 import api, native as N

    w = H.workload(name, L=None if name != "city32" else 16, log2_T=None if name != "city32" else 16)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m)
    o, d = _edge_rays(w, 2048)
    R = len(o)
    samp = dataclasses.replace(H.sampling(w), flags=api.SAVE_FEATURES)
    g = sy.rng(91, "misc")
    adj = [torch.from_numpy(a.astype(np.float32)).cuda() for a in
           (g.standard_normal((R, 3)), g.standard_normal(R), g.standard_normal(R), g.standard_normal(R))]
    lib = N.lib()
    runs = []
    try:
        for min_bytes in (0, 1):  # 0: the default threshold (tiled here); 1: every table is "large"
            N.check(lib.nerfxl_set_gather_groups(min_bytes, 0, 0, 0), "threshold")
            ws = api.alloc_workspace(gf, samp, R, for_backward=True)
            out = api.render_fwd(gf, samp, o, d, workspace=ws)
            gt, gm = api.render_bwd(gf, samp, o, d, ws, *adj)  # from the records this forward wrote
            api.check(ws)
            runs.append(({k: v.clone() for k, v in out.items()}, gt.cpu().numpy(), gm.cpu().numpy()))
    finally:
        N.check(lib.nerfxl_set_gather_groups(0, 0, 0, 0), "threshold reset")
    (a, ta, ma), (b, tb, mb) = runs
    for k in a:
        assert torch.equal(a[k], b[k]), k
    for x, y in ((ta, tb), (ma, mb)):
        assert np.abs(x).max() > 0
        assert np.abs(x - y).max() <= 1e-5 * np.abs(x).max()
    of = H.oracle_field(w, t, m)
    ref = oracle.render(of, w.S, o, d, 1)
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    H.assert_forward_close({k: v.cpu().numpy() for k, v in a.items()}, ref, t_far)
