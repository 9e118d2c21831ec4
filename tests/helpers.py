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


# FP32 gradients take each hidden unit's ReLU decision from an FP32
# pre-activation. Where the FP64 pre-activation lies within the FP32 rounding
# of zero the two can decide differently, and either decision is a correct
# FP32 result. The oracle measures, per ray, the smallest |z| / s over the
# hidden units of its evaluated samples (s: the sum of the magnitudes that
# form z, carried through the layers; an FP32 evaluation of z errs by at most
# about n u s, u = 6e-8, n <= 64, and typically sqrt(n) u s = 5e-7 s). Rays
# within KINK_MARGIN of a kink are left out of the FP32 gradient checks, which
# then hold every entry of every gradient to the stated bound with no
# exception.
KINK_MARGIN = 1e-6


def kink_free(of, S, o, d, margin=KINK_MARGIN):
    """Boolean mask of the rays whose evaluated samples keep every hidden unit
    more than `margin` of its error scale away from the ReLU kink."""
    import oracle

    return oracle.relu_margin(of, S, o, d) > margin


def grad_close(g, ref, tol=1e-4):
    """The FP32 gradient bound: |g - ref| <= tol * max|ref| for every entry
    (FP32 atomics only reorder the sums). Returns (ok, max relative error)."""
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    err = float(np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-30)) if g.size else 0.0
    return err <= tol, err


def kinkless_params(w, seed=22):
    """A network without ReLU kinks for the 16-bit gradient checks: positive
    table entries U[0.1, 1] and hidden weights U[0, 0.05] make every hidden
    pre-activation a sum of positive terms, far above zero, so a 16-bit
    rounding cannot flip a ReLU decision; output weights N(0, 0.1)."""
    import oracle
    from paper_2404_16221_b300 import synthetic as sy

    E = oracle.table_entries(w.level_res, w.log2_T)
    g = sy.rng(seed, "misc")
    t = g.uniform(0.1, 1.0, (w.K, E, w.F)).astype(np.float32)
    m = np.concatenate([g.uniform(0.0, 0.05, (w.K, w.mlp_in * w.W)), g.uniform(0.0, 0.05, (w.K, w.W * w.W)),
                        g.normal(0.0, 0.1, (w.K, w.W * 4))], 1).astype(np.float32)
    return t, m


def assert_first_adam_step(new, old, g_ref, lr, tol):
    """The first bias-corrected Adam step with a negligible eps moves every
    parameter by lr g / |g| = -lr sign(g) ... up to FP32 rounding. Checked on
    every entry: where |g_ref| > 2 tol max|g_ref| the computed gradient has
    g_ref's sign (it is within tol max|g_ref| of it), so the move is -lr
    sign(g_ref); where g_ref is exactly zero (no sample reads the entry) the
    parameter does not move; elsewhere the move is at most lr."""
    new = np.asarray(new, np.float64).reshape(-1)
    old = np.asarray(old, np.float64).reshape(-1)
    g_ref = np.asarray(g_ref, np.float64).reshape(-1)
    delta = new - old
    scale = np.abs(g_ref).max()
    sure = np.abs(g_ref) > 2 * tol * scale
    assert sure.sum() > 0
    e_sure = np.abs(delta[sure] + lr * np.sign(g_ref[sure])).max()
    assert e_sure <= 1e-6, ("signed steps", e_sure)
    zero = g_ref == 0
    assert not delta[zero].any(), ("untouched entries moved", int((delta[zero] != 0).sum()))
    rest = ~sure & ~zero
    if rest.any():
        assert np.abs(delta[rest]).max() <= lr * (1 + 1e-6) + 1e-6


MLP_LAYER_SIZES = (32 * 64, 64 * 64, 64 * 4)  # W1, W2, W3 of one fused region block


def e4m3_definition(mlp):
    """The E4M3 weight quantisation written out in torch on the CPU (the
    definition the library's nerfxl_quantize_e4m3 is checked against): per
    region and layer scale = max(max|W|, 1e-30) / 448, W_q = e4m3(W / scale)
    (round to nearest even). Returns (bytes [K][P] uint8, scales [K][3])."""
    import torch

    m = torch.as_tensor(mlp, dtype=torch.float32).cpu()
    q = torch.empty(m.shape, dtype=torch.uint8)
    scales = torch.empty(m.shape[0], 3, dtype=torch.float32)
    off = 0
    for li, n in enumerate(MLP_LAYER_SIZES):
        blk = m[:, off:off + n]
        s = blk.abs().amax(dim=1).clamp_min(1e-30) / 448.0
        q[:, off:off + n] = (blk / s[:, None]).to(torch.float8_e4m3fn).view(torch.uint8)
        scales[:, li] = s
        off += n
    return q, scales


def e4m3_dequantize(q, scales):
    """W = scale * e4m3 value, FP32 [K][P] (host)."""
    import torch

    q = torch.as_tensor(q).cpu()
    out = q.view(torch.float8_e4m3fn).float()
    sc = torch.as_tensor(scales).cpu()
    off = 0
    for li, n in enumerate(MLP_LAYER_SIZES):
        out[:, off:off + n] *= sc[:, li:li + 1]
        off += n
    return out
