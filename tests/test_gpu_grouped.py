"""Level-grouped gather of the tensor-core forward (fields whose region table
outgrows the L2's reach for random gathers): the features are gathered one
group of levels at a time over a region's samples into feature tiles, then the
MLP and render read them. The result must equal the one-pass gather bit for
bit, whatever the grouping and the window of tiles, in the plain forward, the
split representation and the record-writing forward of a training step. The
grouping thresholds are a process-wide setting; each test forces them and
restores the defaults."""
import ctypes

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


@pytest.fixture
def groups():
    """set(min_bytes, group_bytes, window): force the grouped gather; defaults restored after."""
    from paper_2404_16221_b300 import native as N

    def set_(min_bytes, group_bytes, window):
        N.check(N.lib().nerfxl_set_gather_groups(int(min_bytes), int(group_bytes), int(window), 1), "groups")

    yield set_
    N.check(N.lib().nerfxl_set_gather_groups(0, 0, 0, 0), "groups")


def _render(field, samp, o, d):
    from paper_2404_16221_b300 import api

    ws = api.alloc_workspace(field, samp, len(o))
    out = {k: v.cpu().numpy() for k, v in api.render_fwd(field, samp, o, d, workspace=ws).items()}
    api.check(ws)
    return out, ws.numel()


@pytest.mark.parametrize("tab", [torch.float16, torch.float32])
@pytest.mark.parametrize("group_bytes,window", [(1, 7), (300 << 10, 1 << 16), (2 << 20, 64)])
def test_grouped_forward_equals_one_pass(groups, tab, group_bytes, window):
    """city32 shapes (K=32, S=256) with 2^16-entry tables: one level per group
    (group_bytes = 1), a few levels per group, whole-batch and tiny windows
    (many launches, regions cut by window ends)."""
    w = H.workload("city32", L=16, log2_T=16)
    t, m = H.params(w)
    field = H.gpu_field(w, t, m, table_dtype=tab, mlp_dtype=torch.bfloat16)
    o, d = sy.workload_rays(w, 3000)
    samp = H.sampling(w)
    ref, ws_plain = _render(field, samp, o, d)
    groups(1, group_bytes, window)
    got, ws_grouped = _render(field, samp, o, d)
    assert ws_grouped > ws_plain  # the feature-tile window
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    # and against the oracle on the rounded parameters
    tq = torch.from_numpy(t).to(tab).float().numpy()
    mq = torch.from_numpy(m).bfloat16().float().numpy()
    orf = oracle.render(H.oracle_field(w, tq, mq), w.S, o, d, 1)
    assert np.abs(got["rgb"] - orf["rgb"]).max() <= 2e-3


def test_grouped_split_forward_equals_one_pass(groups):
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("grid8", L=16, log2_T=15)
    t, _ = H.params(w)
    n = api.split_mlp_params(w.K, w.mlp_in, w.W)
    m = sy.split_mlp_params(w, n)
    field = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.from_numpy(t).half(),
                                 torch.from_numpy(m).bfloat16(), arch=N.ARCH_SPLIT)
    o, d = sy.workload_rays(w, 2048)
    samp = H.sampling(w)
    ref, _ = _render(field, samp, o, d)
    groups(1, 1 << 20, 50)
    got, _ = _render(field, samp, o, d)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("window", [0, 9])
def test_grouped_training_step_equals_one_pass(groups, window):
    """The record-writing forward of nerfxl_step with the grouped gather
    (the default window, or 9 tiles: many windows, regions cut by window
    ends) writes the records from the feature words: loss bit for bit,
    gradients up to the order of the FP32 sums."""
    from paper_2404_16221_b300 import api

    w = H.workload("city32", L=16, log2_T=16)
    t, m = H.params(w)
    o, d = sy.workload_rays(w, 4096)
    tgt = sy.rng(95, "misc").uniform(0, 1, (len(o), 3)).astype(np.float32)
    runs = []
    for grouped in (False, True):
        if grouped:
            groups(1, 1 << 20, window)
        field = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
        tr = api.Trainer(field, H.sampling(w), lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=t, master_mlp=m)
        L = tr.step(o, d, tgt).cpu().numpy().copy()
        runs.append((L, tr.grad_tables.cpu().numpy(), tr.grad_mlp.cpu().numpy()))
    (L1, gt1, gm1), (L2, gt2, gm2) = runs
    assert np.array_equal(L1, L2)
    for a, b in ((gt1, gt2), (gm1, gm2)):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_set_gather_groups_rejects_bad_window():
    from paper_2404_16221_b300 import native as N

    assert N.lib().nerfxl_set_gather_groups(0, 0, -1, 0) == N.E_INVALID
    assert N.lib().nerfxl_set_gather_groups(0, 0, 0, -1) == N.E_INVALID
