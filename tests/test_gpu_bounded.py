"""Bounded-memory training steps: nerfxl_step under a workspace cap runs in
ray sub-batches (forward, loss adjoints normalised by the whole batch,
backward per sub-batch; one Adam step). The capped step must equal the
one-pass step (the loss bit for bit, the gradients up to the order of the FP32
sums) and, in FP32, the FP64 oracle within the stated bounds."""
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


def _cap_for(trainer, R, rays_per_batch):
    """A workspace cap that gives sub-batches of about rays_per_batch rays."""
    from paper_2404_16221_b300 import api, native as N

    fd, sd = trainer.field.desc(), trainer.samp.desc()
    return int(N.lib().nerfxl_step_workspace_bytes(api.C_ref(fd), api.C_ref(sd), rays_per_batch)) + (1 << 16)


def test_capped_fp32_step_matches_oracle_and_one_pass():
    from paper_2404_16221_b300 import api

    w = H.workload("grid8", L=16, log2_T=14)
    t, m = H.params(w)
    o, d = sy.workload_rays(w, 4096)
    sel = sy.subset(4096, 2600, 91)
    o, d = o[sel], d[sel]
    keep = H.kink_free(H.oracle_field(w, t, m), w.S, o, d)
    o, d = o[keep].copy(), d[keep].copy()
    R = len(o)
    tgt = sy.rng(92, "misc").uniform(0, 1, (R, 3)).astype(np.float32)
    runs = []
    for capped in (False, True):
        gf = H.gpu_field(w, t.copy(), m.copy())
        tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01)
        if capped:
            tr.workspace_cap = _cap_for(tr, R, 600)
            Rb = tr.sub_batch(R)
            assert 256 <= Rb < R and Rb % 256 == 0, Rb
        L = tr.step(o, d, tgt).cpu().numpy().copy()
        runs.append((L, tr.grad_tables.cpu().numpy(), tr.grad_mlp.cpu().numpy(), gf.tables.cpu().numpy(),
                     gf.mlp.cpu().numpy()))
    (L1, gt1, gm1, _, _), (L2, gt2, gm2, t2, m2) = runs
    assert np.array_equal(L1, L2)
    for a, b in ((gt1, gt2), (gm1, gm2)):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    L_ref, gt_ref, gm_ref = oracle.loss_grad(H.oracle_field(w, t, m), w.S, o, d, tgt, 0.01)
    assert abs(L2[0] - L_ref) <= 1e-5 * L_ref
    for g, ref in ((gt2, gt_ref), (gm2, gm_ref)):
        ok, e = H.grad_close(g, ref)
        assert ok, e
    H.assert_first_adam_step(t2, t, gt_ref, 1e-2, 1e-4)
    H.assert_first_adam_step(m2, m, gm_ref, 1e-2, 1e-4)


def test_capped_mixed_city_step_equals_one_pass():
    """The street/city field (K=32, L=16, S=256) with FP16 tables, BF16 MLP
    and the forward's records: 2^14 rays in one pass and under a cap that
    splits them into sub-batches of about 3000 rays."""
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("city32", L=16, log2_T=16)
    t, m = H.params(w)
    o, d = sy.workload_rays(w, 1 << 14)
    tgt = sy.rng(93, "misc").uniform(0, 1, (len(o), 3)).astype(np.float32)
    runs = []
    for capped in (False, True):
        gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
        tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=t, master_mlp=m)
        if capped:
            tr.workspace_cap = _cap_for(tr, len(o), 3000)
            Rb = tr.sub_batch(len(o))
            assert 256 <= Rb < len(o), Rb
        L = tr.step(o, d, tgt).cpu().numpy().copy()
        runs.append((L, tr.grad_tables.cpu().numpy(), tr.grad_mlp.cpu().numpy()))
    (L1, gt1, gm1), (L2, gt2, gm2) = runs
    assert np.array_equal(L1, L2)
    for a, b in ((gt1, gt2), (gm1, gm2)):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_full_size_city_step_under_4gb():
    """The street/city training step at its full size (2^20 rays, S=256,
    K=32, T=2^21, FP16 tables, BF16 MLP, FP32 Adam) runs with a 4 GB
    workspace (its one-pass workspace is far larger), and its loss equals the
    loss of a separate forward render of the same rays."""
    from paper_2404_16221_b300 import api, native as N

    w = sy.workload("city32")
    dev = torch.device("cuda")
    E = N.table_entries(w.level_res, w.log2_T)
    tt, mm = sy.field_params_device(w, E, N.mlp_params(w.mlp_in, w.W), dev)
    gf = api.PartitionedField(w.boxes, w.level_res, w.log2_T, tt.to(torch.float16), mm.to(torch.bfloat16), device=dev)
    o, d = (torch.from_numpy(a).to(dev) for a in sy.workload_rays(w))
    tgt = torch.rand(len(o), 3, generator=torch.Generator().manual_seed(94)).to(dev)
    cap = 4 << 30
    tr = api.Trainer(gf, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=tt, master_mlp=mm,
                     workspace_cap=cap)
    fd, sd = gf.desc(), tr.samp.desc()
    full = int(N.lib().nerfxl_step_workspace_bytes(api.C_ref(fd), api.C_ref(sd), len(o)))
    Rb = tr.sub_batch(len(o))
    print("city32 step: one-pass workspace %.1f GB, sub-batch %d rays under 4 GB" % (full / 2 ** 30, Rb))
    assert full > 2 * cap and 0 < Rb < len(o)
    out = api.render_fwd(gf, H.sampling(w), o, d)  # the parameters before the step
    loss = tr.step(o, d, tgt).cpu().numpy()
    assert tr._ws.numel() <= cap
    rgb, dist = out["rgb"].double(), out["dist"].double()
    ref = float(((rgb - tgt.double()) ** 2).mean() + 0.01 * dist.mean())
    assert np.isfinite(loss).all() and abs(loss[0] - ref) <= 1e-5 * ref, (loss[0], ref)
    assert torch.isfinite(tr.grad_tables).all() and float(tr.grad_tables.abs().max()) > 0
