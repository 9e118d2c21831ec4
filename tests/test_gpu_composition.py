"""Sample-level composition (the naive scheme of Sec. 4.2) against the
segment-level composition of Eq. 3-8 / Algorithm 1-2: both equal the
single-pass render of the oracle; the segment-level scheme moves a small
fraction of the bytes between the field kernel and the composite."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import synthetic as sy

import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n", [("unit", 1024), ("grid8", 2048), ("city32", 1024)])
def test_sample_level_composition_matches_single_pass(name, n):
    from paper_2404_16221_b300 import api

    w = H.workload(name, L=None if name != "city32" else 12, log2_T=None if name != "city32" else 15)
    t, m = H.params(w)
    of = H.oracle_field(w, t, m)
    gf = H.gpu_field(w, t, m)
    o, d = sy.workload_rays(w, n)
    samp_s = dataclasses.replace(H.sampling(w), flags=api.SAMPLE_COMPOSITE)
    ws = api.alloc_workspace(gf, samp_s, len(o))
    out_s = api.render_fwd(gf, samp_s, o, d, workspace=ws)
    api.check(ws)
    out_s = {k: v.cpu().numpy() for k, v in out_s.items()}
    out_c = {k: v.cpu().numpy() for k, v in api.render_fwd(gf, H.sampling(w), o, d).items()}
    ref = oracle.render(of, w.S, o, d, 0)  # single pass, O(N^2) distortion
    nseg, region, t0, t1, nint = oracle.segments(of, w.S, o, d)
    t_far = np.array([t1[r, nseg[r] - 1] if nseg[r] else 0.0 for r in range(len(o))])
    errs = H.assert_forward_close(out_s, ref, t_far)
    H.assert_forward_close(out_c, ref, t_far)
    print(name, "sample-level vs single pass", errs)


def test_sample_level_composition_is_forward_only_and_fp32_only():
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("grid8", L=8, log2_T=14)
    t, m = H.params(w)
    samp = dataclasses.replace(H.sampling(w), flags=api.SAMPLE_COMPOSITE)
    o, d = sy.workload_rays(w, 64)
    gm = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    with pytest.raises(N.NerfxlError) as e:
        api.render_fwd(gm, samp, o, d)
    assert e.value.status == N.E_UNSUPPORTED
    g32 = H.gpu_field(w, t, m)
    ws = api.alloc_workspace(g32, samp, len(o), for_backward=True)
    api.render_fwd(g32, samp, o, d, workspace=ws)
    z = torch.zeros(len(o), 3, device="cuda")
    with pytest.raises(N.NerfxlError) as e:
        api.render_bwd(g32, samp, o, d, ws, z)
    assert e.value.status == N.E_UNSUPPORTED
