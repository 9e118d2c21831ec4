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
