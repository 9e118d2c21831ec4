"""Failure detection without a GPU fault: bounded device waits give up with
an error status the host reads, and the context stays usable afterwards."""
import numpy as np
import pytest

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


def test_bounded_wait_times_out_and_context_survives():
    from paper_2404_16221_b300 import api, native as N

    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    lib = N.lib()
    # a barrier nobody arrives on: the wait gives up after 2^16 polls
    st = lib.nerfxl_debug_wait_probe(N._ptr(status), 1 << 16, 0, N._stream(None))
    assert st == N.E_TIMEOUT and int(status.item()) == 0
    assert b"expired" in lib.nerfxl_last_error()
    # the same wait with an arrival completes
    assert lib.nerfxl_debug_wait_probe(N._ptr(status), 1 << 16, 1, N._stream(None)) == N.OK
    assert int(status.item()) == 1
    # and the context still renders
    w = H.workload("grid8", L=4, log2_T=12)
    t, m = H.params(w)
    gf = H.gpu_field(w, t, m, table_dtype=torch.float16, mlp_dtype=torch.bfloat16)
    o, d = sy.workload_rays(w, 128)
    ws = api.alloc_workspace(gf, H.sampling(w), len(o))
    out = api.render_fwd(gf, H.sampling(w), o, d, workspace=ws)
    api.check(ws)
    assert torch.isfinite(out["rgb"]).all()


def test_invalid_arguments_launch_nothing():
    from paper_2404_16221_b300 import native as N

    assert N.lib().nerfxl_debug_wait_probe(None, 16, 0, N._stream(None)) == N.E_INVALID
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert N.lib().nerfxl_debug_wait_probe(N._ptr(status), 0, 0, N._stream(None)) == N.E_INVALID
