"""The reduction-rate probe that measures the backward scatter's ceiling
does the work it claims: every one of the reported reductions lands (each
adds 1.0 to four floats, so the buffer sums to exactly 4 x ops), all inside
the buffer, and bad arguments launch nothing."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_16221_b300 import build

    build.build()


def test_reduction_probe_counts_every_reduction():
    from paper_2404_16221_b300 import native as N

    lib = N.lib()
    nbytes = 1 << 20
    # guard words around the probed range must stay zero
    buf = torch.zeros(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    inner = buf[32:32 + nbytes // 4]
    ops = ctypes.c_int64(0)
    assert lib.nerfxl_probe_reduction_rate(N._ptr(inner), nbytes, 3, ctypes.byref(ops), N._stream(None)) == N.OK
    torch.cuda.synchronize()
    assert ops.value > 0 and ops.value % 3 == 0
    a = buf.cpu().numpy().astype(np.float64)
    assert a[:32].sum() == 0 and a[32 + nbytes // 4:].sum() == 0
    assert a.sum() == 4 * ops.value  # small integer counts: exact in FP32
    assert np.all(a == np.round(a))


def test_reduction_probe_rejects_bad_arguments():
    from paper_2404_16221_b300 import native as N

    lib = N.lib()
    ops = ctypes.c_int64(-1)
    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")
    for p, nbytes, iters, o in ((None, 4096, 1, ctypes.byref(ops)), (N._ptr(buf), 8, 1, ctypes.byref(ops)),
                                (N._ptr(buf), 4096, 0, ctypes.byref(ops)), (N._ptr(buf), 4096, 1, None)):
        assert lib.nerfxl_probe_reduction_rate(p, nbytes, iters, o, N._stream(None)) == N.E_INVALID
    assert ops.value == -1


def test_load_probe_reads_only_and_counts():
    from paper_2404_16221_b300 import native as N

    lib = N.lib()
    nbytes = 1 << 20
    buf = torch.arange(nbytes // 4, dtype=torch.int32, device="cuda")
    before = buf.clone()
    ops = ctypes.c_int64(0)
    assert lib.nerfxl_probe_load_rate(N._ptr(buf), nbytes, 2, ctypes.byref(ops), N._stream(None)) == N.OK
    torch.cuda.synchronize()
    assert ops.value > 0 and ops.value % (2 * 16) == 0
    assert torch.equal(buf, before)  # only read
    bad = ctypes.c_int64(-1)
    for p, nb, it, o in ((None, 4096, 1, ctypes.byref(bad)), (N._ptr(buf), 4, 1, ctypes.byref(bad)),
                         (N._ptr(buf), 4096, 0, ctypes.byref(bad)), (N._ptr(buf), 4096, 1, None)):
        assert lib.nerfxl_probe_load_rate(p, nb, it, o, N._stream(None)) == N.E_INVALID
    assert bad.value == -1
