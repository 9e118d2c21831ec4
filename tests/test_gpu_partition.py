"""Rendering on regions from the spatial partitioning (Sec. 4.4): the boxes are
no longer a uniform grid, and the renderer must still match the oracle and
the partitioned render must still equal the single pass; the partition spreads
samples over the regions more evenly than the uniform grid."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import synthetic as sy

import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _kd_workload(name, levels, L=None, log2_T=None):
    from paper_2404_16221_b300 import api

    w = H.workload(name, L=L, log2_T=log2_T)
    root = sy.scene_root(w)
    pts = sy.content_points(w, 100000, seed=17)
    boxes, counts = api.partition_boxes(pts, root, levels)
    w = dataclasses.replace(w, boxes=boxes, max_segments=min(len(boxes), 32))
    return w, counts


@pytest.mark.parametrize("name,levels,L,log2_T", [("grid8", 3, 16, 14), ("city32", 5, 12, 15)])
def test_forward_on_partitioned_regions_matches_oracle(name, levels, L, log2_T):
    from paper_2404_16221_b300 import api

    w, _ = _kd_workload(name, levels, L, log2_T)
    t, m = H.params(w)
    of = H.oracle_field(w, t, m)
    gf = H.gpu_field(w, t, m)
    o, d = sy.workload_rays(w, 2048, seed=41)
    samp = H.sampling(w)
    ws = api.alloc_workspace(gf, samp, len(o))
    out = api.render_fwd(gf, samp, o, d, workspace=ws)
    api.check(ws)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.render(of, w.S, o, d, 1)    # Algorithm 1-2 over the segments
    ref0 = oracle.render(of, w.S, o, d, 0)   # single pass over all samples
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    errs = H.assert_forward_close(out, ref, t_far)
    H.assert_forward_close(out, ref0, t_far)
    assert nseg.max() >= 2  # rays do cross partition planes
    print(name, levels, errs, "max segments", int(nseg.max()))


def test_mixed_forward_on_partitioned_regions():
    from paper_2404_16221_b300 import api

    w, _ = _kd_workload("grid8", 3, 16, 14)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    tq = torch.from_numpy(t).to(torch.float16).float().numpy()
    mq = torch.from_numpy(m).to(torch.bfloat16).float().numpy()
    o, d = sy.workload_rays(w, 2048, seed=43)
    out = api.render_fwd(gf, H.sampling(w), o, d)
    ref = oracle.render(H.oracle_field(w, tq, mq), w.S, o, d, 1)
    assert np.abs(out["rgb"].cpu().numpy() - ref["rgb"]).max() <= 2e-3


def test_partition_balances_region_samples():
    """Per-region chunk counts of held-out rays of an uneven city32 trajectory:
    boxes from the CDF splits of training-ray samples spread the work far more
    evenly than the uniform 8 x 4 x 1 slabs."""
    from paper_2404_16221_b300 import api

    w = sy.workload("city32")
    root = sy.scene_root(w)
    o_tr, d_tr = sy.one_sided_rays(w, 4096, 51)
    kd_boxes, _ = api.partition_boxes(sy.ray_sample_points(o_tr, d_tr, root, 64, 3), root, 5)
    o, d = sy.one_sided_rays(w, 1 << 15, 52)
    stats = {}
    for label, boxes in (("grid", w.boxes), ("cdf", kd_boxes)):
        wk = dataclasses.replace(w, boxes=boxes, level_res=w.level_res[:4], log2_T=12, max_segments=32)
        t, m = H.params(wk)
        gf = H.gpu_field(wk, t, m)
        samp = H.sampling(wk)
        ws = api.alloc_workspace(gf, samp, len(o))
        api.render_fwd(gf, samp, o, d, workspace=ws)
        api.check(ws)
        chunks = api.region_chunks(ws, wk.K)
        _, n_chunks = api.workspace_stats(ws)
        assert int(chunks.sum()) == n_chunks
        stats[label] = float(chunks.max() / max(int(chunks.min()), 1))
    print("max/min chunks per region:", stats)
    assert stats["cdf"] < 0.5 * stats["grid"]
