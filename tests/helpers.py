"""Shared set-up for parity tests: one seeded workload, handed both to the
oracle (float64 copies) and to the CUDA library (device tensors)."""
import numpy as np

import oracle
from paper_2404_16221_b300 import synthetic as sy


def workload(name, L=None, log2_T=None, S=None):
    w = sy.workload(name)
    if L is not None:
        w.level_res = w.level_res[:L]
    if log2_T is not None:
        w.log2_T = log2_T
    if S is not None:
        w.S = S
    return w


def params(w, table_std=1.0, mlp_std=0.1):
    E = oracle.table_entries(w.level_res, w.log2_T)
    P = oracle.mlp_params(w.mlp_in, w.W)
    return sy.field_params(w, E, P, table_std, mlp_std)


def oracle_field(w, tables, mlp):
    return oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, tables.astype(np.float64),
                        mlp.astype(np.float64))


def gpu_field(w, tables, mlp, table_dtype=None, mlp_dtype=None):
    import torch

    from paper_2404_16221_b300 import api

    t = torch.from_numpy(tables)
    m = torch.from_numpy(mlp)
    if table_dtype is not None:
        t = t.to(table_dtype)
    if mlp_dtype is not None:
        m = m.to(mlp_dtype)
    return api.PartitionedField(w.boxes, w.level_res, w.log2_T, t, m, F=w.F, mlp_in=w.mlp_in, width=w.W)


def sampling(w):
    from paper_2404_16221_b300 import api

    return api.Sampling(w.S, w.max_segments)


def rel_err(gpu, ref, s):
    """max |gpu - ref| / (|ref| + s), the relative measure with floor s."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(gpu - ref) / (np.abs(ref) + s))) if gpu.size else 0.0


def assert_forward_close(out, ref, t_far, tol=1e-5):
    """Tolerance of the FP32 forward: |gpu - ref| <= tol * (|ref| + s), with
    s = 1 for colour and opacity, s = t_far of the ray for depth and s = the
    largest distortion of the batch for the distortion loss."""
    errs = {
        "rgb": rel_err(out["rgb"], ref["rgb"], 1.0),
        "opacity": rel_err(out["opacity"], ref["opacity"], 1.0),
        # a missed ray has t_far = 0 and must render depth 0 exactly
        "depth": float(np.max(np.abs(np.asarray(out["depth"], np.float64) - ref["depth"]) /
                              (np.abs(ref["depth"]) + np.where(t_far > 0, t_far, 1.0)))) if len(t_far) else 0.0,
        "dist": rel_err(out["dist"], ref["dist"], max(float(np.max(np.abs(ref["dist"]))), 1e-30)),
    }
    bad = {k: v for k, v in errs.items() if not v <= tol}  # NaN counts as a failure
    assert not bad, errs
    return errs
