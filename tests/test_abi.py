"""The C-ABI library loads, exports every declared symbol, and validates its
arguments on the host (no GPU needed: nothing here launches a kernel)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2404_16221_b300 import build, native as N
from paper_2404_16221_b300 import synthetic as sy


@pytest.fixture(scope="module")
def lib():
    build.build()
    return N.lib()


def test_every_declared_symbol_is_exported(lib):
    names = N.header_functions()
    assert "nerfxl_render_fwd" in names and len(names) >= 8
    raw = ctypes.CDLL(N.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name
        assert name in N.SIGNATURES, "binding misses " + name


@pytest.mark.parametrize("name", ["unit", "grid8", "city32"])
def test_table_layout_agrees_with_oracle(lib, name):
    # Two independent implementations of the level layout must agree.
    w = sy.workload(name)
    assert N.table_entries(w.level_res, w.log2_T) == oracle.table_entries(w.level_res, w.log2_T)
    assert N.mlp_params(32, 64) == oracle.mlp_params(32, 64)


def _desc(K=8, F=2, mlp_in=32, width=64, L=16):
    d = N.FieldDesc()
    d.K, d.L, d.F, d.log2_T, d.mlp_in, d.mlp_width = K, L, F, 19, mlp_in, width
    for i in range(L):
        d.level_res[i] = 16 + 8 * i
    d.boxes = d.tables = d.mlp = 1  # never dereferenced: validation fails or no launch happens
    return d


def test_host_validation_rejects_bad_arguments(lib):
    s = N.SamplingDesc(128, 4, 0.0, 0)
    for kw, want in ((dict(K=0), N.E_INVALID), (dict(F=4), N.E_UNSUPPORTED), (dict(width=128), N.E_UNSUPPORTED),
                     (dict(L=0), N.E_INVALID)):
        d = _desc(**kw)
        st = lib.nerfxl_render_fwd(ctypes.byref(d), ctypes.byref(s), 16, None, None, None, None, None, None, None, 0,
                                   None)
        assert st == want, (kw, st)
        assert lib.nerfxl_last_error()
    bad_s = N.SamplingDesc(0, 4, 0.0, 0)
    d = _desc()
    assert lib.nerfxl_render_fwd(ctypes.byref(d), ctypes.byref(bad_s), 16, None, None, None, None, None, None, None,
                                 0, None) == N.E_INVALID
    # workspace too small is refused before any launch
    st = lib.nerfxl_render_fwd(ctypes.byref(d), ctypes.byref(s), 16, 1, 1, 1, 1, 1, 1, 1, 16, None)
    assert st == N.E_WORKSPACE


def test_workspace_size_grows_with_rays(lib):
    d = _desc()
    s = N.SamplingDesc(128, 4, 0.0, 0)
    a = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0)
    b = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 2000, 0)
    c = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 2000, 1)
    assert 0 < a < b < c
    assert lib.nerfxl_max_chunks(ctypes.byref(s), 8) == 4 + 127 // 32


def test_occupancy_and_split_arguments_on_the_host(lib):
    """Host-side checks of the occupancy grid and the split representation:
    grid resolution, representation code, dtype combinations, workspace
    sizes and parameter counts (no kernel is launched)."""
    s = N.SamplingDesc(128, 4, 0.0, 0)
    d = _desc()
    base = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0)
    assert base > 0
    # an occupancy grid adds the per-segment kept counts and the kept-interval lists
    d.occupancy, d.occ_res = 1, 64
    grown = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0)
    assert grown >= base + 1000 * 4 * 4 + 1000 * 2 * (128 + 4 - 1)
    for bad in (0, 1025):
        d.occ_res = bad
        assert lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0) == 0
        st = lib.nerfxl_render_fwd(ctypes.byref(d), ctypes.byref(s), 16, 1, 1, 1, 1, 1, 1, 1, 1 << 30, None)
        assert st == N.E_INVALID
    # representations: fused and split counts, unknown code rejected
    d = _desc()
    assert lib.nerfxl_field_mlp_params(ctypes.byref(d)) == 8 * N.mlp_params(32, 64)
    d.arch = N.ARCH_SPLIT
    assert lib.nerfxl_field_mlp_params(ctypes.byref(d)) == \
        8 * oracle.density_params(32, 64) + oracle.color_params(64)
    d.mlp_dtype = N.E4M3
    assert lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0) == 0
    d.mlp_dtype = N.BF16
    # both representations keep the same records for the backward: the
    # tensor-core backward's per-tile records with a 16-bit MLP (about 116
    # bytes per sample row), the FP32 features (128 bytes) with an FP32 MLP
    with_rec = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 1)
    assert with_rec == lib.nerfxl_workspace_bytes(ctypes.byref(_fused_bf16()), ctypes.byref(s), 1000, 1)
    d.mlp_dtype = N.F32
    f32_rec = lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 1)
    assert f32_rec == lib.nerfxl_workspace_bytes(ctypes.byref(_desc()), ctypes.byref(s), 1000, 1)
    assert lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0) < f32_rec
    d.mlp_dtype = N.BF16
    d.arch = 7
    assert lib.nerfxl_field_mlp_params(ctypes.byref(d)) == -1
    assert lib.nerfxl_workspace_bytes(ctypes.byref(d), ctypes.byref(s), 1000, 0) == 0


def _fused_bf16():
    d = _desc()
    d.mlp_dtype = N.BF16
    return d


def test_occupancy_refresh_arguments_on_the_host(lib):
    d = _desc()
    d.level_res[15] = 16 + 8 * 15
    for G, decay, tdt, mdt in ((0, 0.9, N.F32, N.F32), (2048, 0.9, N.F32, N.F32), (8, 1.5, N.F32, N.F32),
                               (8, 0.9, N.F16, N.BF16)):
        d.table_dtype, d.mlp_dtype = tdt, mdt
        st = lib.nerfxl_occupancy_update(ctypes.byref(d), G, 0, 1, decay, 0.01, 1, 1, None)
        assert st in (N.E_INVALID, N.E_UNSUPPORTED), (G, decay, st)
    d.table_dtype, d.mlp_dtype = N.F32, N.F32
    assert lib.nerfxl_occupancy_update(ctypes.byref(d), 8, 0, 1, 0.9, 0.01, None, None, None) == N.E_INVALID


def test_backward_rejects_fp16_tables_with_fp32_mlp_before_any_launch(lib):
    """The FP32 MLP reads FP32 tables (forward and backward alike): FP16
    tables with an FP32 MLP are refused on the host for both representations,
    before the backward launches anything (no GPU needed)."""
    s = N.SamplingDesc(128, 4, 0.0, 0)
    for arch in (N.ARCH_FUSED, N.ARCH_SPLIT):
        d = _desc()
        d.arch = arch
        d.table_dtype, d.mlp_dtype = N.F16, N.F32
        st = lib.nerfxl_render_bwd(ctypes.byref(d), ctypes.byref(s), 16, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1 << 40, None)
        assert st == N.E_UNSUPPORTED, (arch, st)
        assert b"16-bit MLP" in lib.nerfxl_last_error()
        st = lib.nerfxl_render_fwd(ctypes.byref(d), ctypes.byref(s), 16, 1, 1, 1, 1, 1, 1, 1, 1 << 40, None)
        assert st == N.E_UNSUPPORTED, (arch, st)
