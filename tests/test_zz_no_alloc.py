"""The allocation-free forward entry point, through the C ABI.

nerfxl_render_fwd_static is for callers that cannot allocate device memory
(a C program or plug-in without an allocator, a host that owns the device
memory pool, a frame loop where cudaMalloc would stall). It must give the
same image as nerfxl_render_fwd with a caller workspace, call after call,
although every call reuses one fixed scratch array that still holds the
previous call's contents. This file is collected last on purpose.
"""
import ctypes

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


def _static_call(field, samp, o, d):
    from paper_2404_16221_b300 import native as N

    R = o.shape[0]
    out = {"rgb": torch.full((R, 3), -1.0, device="cuda"), "depth": torch.full((R,), -1.0, device="cuda"),
           "opacity": torch.full((R,), -1.0, device="cuda"), "dist": torch.full((R,), -1.0, device="cuda")}
    fd, sd = field.desc(), samp.desc()
    st = N.lib().nerfxl_render_fwd_static(ctypes.byref(fd), ctypes.byref(sd), R, N._ptr(o), N._ptr(d),
                                          N._ptr(out["rgb"]), N._ptr(out["depth"]), N._ptr(out["opacity"]),
                                          N._ptr(out["dist"]), N._stream(None))
    N.check(st, "nerfxl_render_fwd_static")
    torch.cuda.synchronize()
    return out


def test_static_scratch_matches_workspace_entry_point():
    from paper_2404_16221_b300 import api, native as N

    w = H.workload("grid8")
    t, m = H.params(w)
    field = H.gpu_field(w, t, m)
    samp = H.sampling(w)
    # two different batches, so the second call starts from the first call's leftovers
    o1, d1 = sy.workload_rays(w, 8192)
    o2, d2 = o1[4096:] * np.float32(1.1), d1[4096:].copy()
    for o, d in ((o1, d1), (o2, d2)):
        o_t = torch.from_numpy(np.ascontiguousarray(o)).cuda()
        d_t = torch.from_numpy(np.ascontiguousarray(d)).cuda()
        ref = api.render_fwd(field, samp, o_t, d_t)
        got = _static_call(field, samp, o_t, d_t)
        for k in ref:
            # the same kernels on the same inputs: the same bits
            assert torch.equal(got[k], ref[k]), k
        assert N.lib().nerfxl_static_check(N._stream(None)) == N.OK


def test_static_scratch_reports_device_side_overflow():
    """A ray crossing more regions than max_segments is flagged on the device;
    the static caller reads that flag with nerfxl_static_check, and the next
    call starts clean."""
    import dataclasses

    from paper_2404_16221_b300 import native as N

    w = H.workload("grid8", L=8, log2_T=14)
    t, m = H.params(w)
    field = H.gpu_field(w, t, m)
    o, d = sy.workload_rays(w, 2048)
    o_t, d_t = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    _static_call(field, dataclasses.replace(H.sampling(w), max_segments=1), o_t, d_t)
    assert N.lib().nerfxl_static_check(N._stream(None)) == N.E_OVERFLOW
    assert b"max_segments" in N.lib().nerfxl_last_error()
    _static_call(field, H.sampling(w), o_t, d_t)
    assert N.lib().nerfxl_static_check(N._stream(None)) == N.OK


def test_static_scratch_refuses_oversized_batch():
    from paper_2404_16221_b300 import native as N

    w = H.workload("grid8", L=4, log2_T=12)
    t, m = H.params(w)
    field = H.gpu_field(w, t, m)
    samp = H.sampling(w)
    R = 1 << 20  # far beyond the 32 MiB scratch
    fd, sd = field.desc(), samp.desc()
    st = N.lib().nerfxl_render_fwd_static(ctypes.byref(fd), ctypes.byref(sd), R, None, None, None, None, None, None,
                                          None)
    assert st == N.E_WORKSPACE
    assert b"split the batch" in N.lib().nerfxl_last_error()
