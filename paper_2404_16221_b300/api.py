"""Python front end of the NeRF-XL C ABI: field blocks on the GPU and calls.

A ``PartitionedField`` holds the K region parameter blocks (boxes, hash
tables, MLPs) as device tensors; ``Sampling`` holds the per-ray sampling
settings. The functions below only marshal arguments into the C ABI
(``native.py``); all work happens in libnerfxl's CUDA kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import torch

from . import native as N

_DTYPE_CODE = {torch.float32: N.F32, torch.float16: N.F16, torch.bfloat16: N.BF16, torch.uint8: N.E4M3}


SAVE_FEATURES = 1  # forward writes the tensor-core backward's records (NERFXL_SAVE_FEATURES)
SAMPLE_COMPOSITE = 2  # sample-level composition, FP32 forward only (NERFXL_SAMPLE_COMPOSITE)


@dataclasses.dataclass
class Sampling:
    n_samples: int
    max_segments: int = 0
    t_min: float = 0.0
    flags: int = 0

    def desc(self) -> N.SamplingDesc:
        return N.SamplingDesc(int(self.n_samples), int(self.max_segments), float(self.t_min), int(self.flags))


class PartitionedField:
    """K disjoint regions, each with its own hash grid and MLP (App. A.1).

    boxes [K][6] float32; tables [K][E][F] float32 (or float16);
    mlp [K][P] float32 (or bf16/fp16; uint8 holding e4m3 with mlp_scales).
    occupancy: optional [K][ceil(G^3/32)] int32/uint32 cell bits of a G^3 grid
    per region (G = occ_res); samples in cells with a clear bit are skipped.
    """

    def __init__(self, boxes, level_res, log2_T: int, tables, mlp, F: int = 2, mlp_in: int = 32, width: int = 64,
                 mlp_scales=None, device="cuda", occupancy=None, occ_res: int = 0, arch: int = N.ARCH_FUSED):
        self.device = torch.device(device)
        self.boxes = torch.as_tensor(boxes, dtype=torch.float32).reshape(-1, 6).contiguous().to(self.device)
        self.level_res = [int(v) for v in level_res]
        self.K = int(self.boxes.shape[0])
        self.L = len(self.level_res)
        self.F, self.log2_T, self.mlp_in, self.width = int(F), int(log2_T), int(mlp_in), int(width)
        self.E = N.table_entries(self.level_res, self.log2_T)
        self.P = N.mlp_params(self.mlp_in, self.width)
        self.tables = torch.as_tensor(tables).to(self.device).reshape(self.K, self.E, self.F).contiguous()
        self.arch = int(arch)
        if self.arch == N.ARCH_SPLIT:
            # per-region density blocks, then the shared colour block (flat)
            self.P = split_mlp_params(self.K, self.mlp_in, self.width)
            self.mlp = torch.as_tensor(mlp).to(self.device).reshape(self.P).contiguous()
        else:
            self.mlp = torch.as_tensor(mlp).to(self.device).reshape(self.K, self.P).contiguous()
        self.mlp_scales = None if mlp_scales is None else torch.as_tensor(
            mlp_scales, dtype=torch.float32).to(self.device).reshape(self.K, 3).contiguous()
        self.set_occupancy(occupancy, occ_res)

    def set_occupancy(self, occupancy, occ_res: int = 0):
        """Attach (or, with None, drop) an occupancy bitfield [K][words]."""
        self.occ_res = int(occ_res) if occupancy is not None else 0
        self.occupancy = None
        if occupancy is not None:
            occ = torch.as_tensor(occupancy)
            if occ.dtype != torch.int32:  # uint32 bit patterns travel as int32
                occ = torch.from_numpy(np.ascontiguousarray(np.asarray(occ.cpu().numpy(), np.uint32).view(np.int32)))
            self.occupancy = occ.to(self.device).reshape(self.K, occupancy_words(self.occ_res)).contiguous()

    def desc(self) -> N.FieldDesc:
        d = N.FieldDesc()
        d.K, d.L, d.F, d.log2_T, d.mlp_in, d.mlp_width = self.K, self.L, self.F, self.log2_T, self.mlp_in, self.width
        for i, v in enumerate(self.level_res):
            d.level_res[i] = v
        d.boxes = self.boxes.data_ptr()
        d.tables = self.tables.data_ptr()
        d.mlp = self.mlp.data_ptr()
        d.table_dtype = _DTYPE_CODE[self.tables.dtype]
        d.mlp_dtype = _DTYPE_CODE[self.mlp.dtype]
        d.mlp_scales = None if self.mlp_scales is None else self.mlp_scales.data_ptr()
        d.occupancy = None if self.occupancy is None else self.occupancy.data_ptr()
        d.occ_res = self.occ_res
        d.arch = self.arch
        return d


def split_mlp_params(K: int, mlp_in: int = 32, width: int = 64) -> int:
    """MLP values of the split representation: K density blocks (mlp_in x W +
    W x 16) and the shared colour block (32 x W + W x W + W x 4)."""
    return K * (mlp_in * width + width * 16) + (32 * width + width * width + width * 4)


def occupancy_words(G: int) -> int:
    """32-bit words of one region's G^3-cell occupancy bitfield."""
    return (int(G) ** 3 + 31) // 32


class OccupancyGrid:
    """Per-region G^3 occupancy grid (Sec. 5.1's spatial skipping, the cited
    Instant-NGP grid): a density estimate per cell and the bitfield the
    renderer skips by. Starts with density 0 and every cell occupied;
    ``update`` refreshes it from an FP32 field (nerfxl_occupancy_update)."""

    def __init__(self, K: int, G: int, device="cuda", decay: float = 0.95, threshold: float = 0.01, seed: int = 0):
        self.K, self.G = int(K), int(G)
        self.decay, self.threshold, self.seed = float(decay), float(threshold), int(seed)
        self.density = torch.zeros(self.K, self.G ** 3, dtype=torch.float32, device=device)
        self.bits = torch.full((self.K, occupancy_words(self.G)), -1, dtype=torch.int32, device=device)
        tail = self.G ** 3 % 32
        if tail:
            self.bits[:, -1] = (1 << tail) - 1
        self.updates = 0

    def attach(self, field: PartitionedField):
        """Make ``field`` render with this grid (shares the bit tensor)."""
        field.occupancy, field.occ_res = self.bits, self.G

    def update(self, fp32_field: PartitionedField, stream=None):
        """One refresh from an FP32 field (tables and MLP, e.g. the training masters)."""
        st = N.lib().nerfxl_occupancy_update(C_ref(fp32_field.desc()), self.G, self.updates, self.seed, self.decay,
                                             self.threshold, N._ptr(self.density), N._ptr(self.bits),
                                             N._stream(stream))
        N.check(st, "nerfxl_occupancy_update")
        self.updates += 1

    def occupied_fraction(self) -> float:
        bits = self.bits.cpu().numpy().view(np.uint32)
        return float(np.unpackbits(bits.view(np.uint8), bitorder="little").sum()) / (self.K * self.G ** 3)


def _rays(rays_o, rays_d, device):
    o = torch.as_tensor(rays_o, dtype=torch.float32).reshape(-1, 3).to(device).contiguous()
    d = torch.as_tensor(rays_d, dtype=torch.float32).reshape(-1, 3).to(device).contiguous()
    if o.shape != d.shape:
        raise ValueError("rays_o and rays_d differ in shape")
    return o, d


def workspace_bytes(field: PartitionedField, samp: Sampling, n_rays: int, for_backward: bool = False) -> int:
    fd, sd = field.desc(), samp.desc()
    n = int(N.lib().nerfxl_workspace_bytes(C_ref(fd), C_ref(sd), int(n_rays), int(for_backward)))
    if n == 0:
        N.check(N.E_INVALID, "nerfxl_workspace_bytes")
    return n


def C_ref(x):
    import ctypes

    return ctypes.byref(x)


def alloc_workspace(field, samp, n_rays, for_backward=False):
    return torch.empty(workspace_bytes(field, samp, n_rays, for_backward), dtype=torch.uint8, device=field.device)


def render_fwd(field: PartitionedField, samp: Sampling, rays_o, rays_d, workspace=None, want_dist: bool = True,
               stream=None, out=None):
    """Forward render: returns dict rgb [R][3], depth, opacity, dist [R]."""
    o, d = _rays(rays_o, rays_d, field.device)
    R = o.shape[0]
    if workspace is None:
        workspace = alloc_workspace(field, samp, R)
    if out is None:
        out = {"rgb": torch.empty(R, 3, device=field.device), "depth": torch.empty(R, device=field.device),
               "opacity": torch.empty(R, device=field.device),
               "dist": torch.empty(R, device=field.device) if want_dist else None}
    fd, sd = field.desc(), samp.desc()
    st = N.lib().nerfxl_render_fwd(C_ref(fd), C_ref(sd), R, N._ptr(o), N._ptr(d), N._ptr(out["rgb"]),
                                   N._ptr(out["depth"]), N._ptr(out["opacity"]), N._ptr(out.get("dist")),
                                   N._ptr(workspace), workspace.numel(), N._stream(stream))
    N.check(st, "nerfxl_render_fwd")
    return out


def check(workspace, stream=None):
    """Report device-side flags of the last call on this workspace (syncs)."""
    N.check(N.lib().nerfxl_check(N._ptr(workspace), workspace.numel(), N._stream(stream)), "nerfxl_check")


def debug_segments(field: PartitionedField, samp: Sampling, rays_o, rays_d, max_seg: int):
    o, d = _rays(rays_o, rays_d, field.device)
    R = o.shape[0]
    dev = field.device
    nseg = torch.zeros(R, dtype=torch.int32, device=dev)
    region = torch.full((R, max_seg), -1, dtype=torch.int32, device=dev)
    t0 = torch.zeros(R, max_seg, device=dev)
    t1 = torch.zeros(R, max_seg, device=dev)
    nint = torch.zeros(R, max_seg, dtype=torch.int32, device=dev)
    ws = alloc_workspace(field, samp, R)
    fd, sd = field.desc(), samp.desc()
    st = N.lib().nerfxl_debug_segments(C_ref(fd), C_ref(sd), R, N._ptr(o), N._ptr(d), int(max_seg), N._ptr(nseg),
                                       N._ptr(region), N._ptr(t0), N._ptr(t1), N._ptr(nint), N._ptr(ws), ws.numel(),
                                       N._stream(None))
    N.check(st, "nerfxl_debug_segments")
    return nseg, region, t0, t1, nint


def debug_samples(field: PartitionedField, samp: Sampling, rays_o, rays_d, max_int: int, want_idx=False,
                  want_feat=False, want_raw=False):
    o, d = _rays(rays_o, rays_d, field.device)
    R = o.shape[0]
    dev = field.device
    count = torch.zeros(R, dtype=torch.int32, device=dev)
    a = torch.zeros(R, max_int, device=dev)
    b = torch.zeros(R, max_int, device=dev)
    region = torch.full((R, max_int), -1, dtype=torch.int32, device=dev)
    idx = torch.zeros(R, max_int, field.L, 8, dtype=torch.int32, device=dev) if want_idx else None
    feat = torch.zeros(R, max_int, field.mlp_in, device=dev) if want_feat else None
    raw = torch.zeros(R, max_int, 4, device=dev) if want_raw else None
    fd, sd = field.desc(), samp.desc()
    st = N.lib().nerfxl_debug_samples(C_ref(fd), C_ref(sd), R, N._ptr(o), N._ptr(d), int(max_int), N._ptr(count),
                                      N._ptr(a), N._ptr(b), N._ptr(region), N._ptr(idx), N._ptr(feat), N._ptr(raw),
                                      N._stream(None))
    N.check(st, "nerfxl_debug_samples")
    return count, a, b, region, idx, feat, raw


def render_bwd(field: PartitionedField, samp: Sampling, rays_o, rays_d, workspace, d_rgb=None, d_depth=None,
               d_opacity=None, d_dist=None, grad_tables=None, grad_mlp=None, stream=None):
    """Adjoint render. ``workspace`` must come from the matching render_fwd
    (allocated with for_backward=True). Gradients are accumulated into
    grad_tables [K][E][F] and grad_mlp (the field's mlp shape; FP32; zero-filled if None)."""
    o, d = _rays(rays_o, rays_d, field.device)
    R = o.shape[0]
    if grad_tables is None:
        grad_tables = torch.zeros(field.K, field.E, field.F, dtype=torch.float32, device=field.device)
    if grad_mlp is None:
        grad_mlp = torch.zeros(field.mlp.shape, dtype=torch.float32, device=field.device)

    def c(t):
        return None if t is None else t.contiguous()

    d_rgb, d_depth, d_opacity, d_dist = c(d_rgb), c(d_depth), c(d_opacity), c(d_dist)
    fd, sd = field.desc(), samp.desc()
    st = N.lib().nerfxl_render_bwd(C_ref(fd), C_ref(sd), R, N._ptr(o), N._ptr(d), N._ptr(d_rgb), N._ptr(d_depth),
                                   N._ptr(d_opacity), N._ptr(d_dist), N._ptr(grad_tables), N._ptr(grad_mlp),
                                   N._ptr(workspace), workspace.numel(), N._stream(stream))
    N.check(st, "nerfxl_render_bwd")
    return grad_tables, grad_mlp


def loss(rgb, dist, target, lam: float, want_grads: bool = True, stream=None):
    """Returns (loss[3] device tensor, d_rgb, d_dist)."""
    R = rgb.shape[0]
    dev = rgb.device
    out = torch.empty(3, dtype=torch.float32, device=dev)
    d_rgb = torch.empty_like(rgb) if want_grads else None
    d_dist = torch.empty(R, dtype=torch.float32, device=dev) if want_grads else None
    scratch = torch.empty(max(1, (R + 255) // 256) * 8, dtype=torch.uint8, device=dev)
    tgt = torch.as_tensor(target, dtype=torch.float32).to(dev).contiguous()
    st = N.lib().nerfxl_loss(R, N._ptr(rgb.contiguous()), N._ptr(None if dist is None else dist.contiguous()),
                             N._ptr(tgt), float(lam), N._ptr(d_rgb), N._ptr(d_dist), N._ptr(out), N._ptr(scratch),
                             scratch.numel(), N._stream(stream))
    N.check(st, "nerfxl_loss")
    return out, d_rgb, d_dist


def adam_update(params, grads, m, v, step: int, lr: float, beta1=0.9, beta2=0.99, eps=1e-15, compute_copy=None,
                stream=None):
    """In-place Adam on FP32 tensors; refreshes an fp16/bf16 compute copy if given."""
    opt = N.AdamDesc(float(lr), float(beta1), float(beta2), float(eps), int(step))
    code = N.F32 if compute_copy is None else _DTYPE_CODE[compute_copy.dtype]
    st = N.lib().nerfxl_adam_update(params.numel(), N._ptr(params), N._ptr(grads), N._ptr(m), N._ptr(v),
                                    ctypes_addr(opt), N._ptr(compute_copy), code, N._stream(stream))
    N.check(st, "nerfxl_adam_update")


def ctypes_addr(x):
    import ctypes

    return ctypes.cast(ctypes.pointer(x), ctypes.c_void_p)


class Trainer:
    """FP32 master parameters + Adam moments; nerfxl_step does fwd, loss, bwd
    and the update in one call. If the field holds 16-bit compute copies
    (FP16 tables, BF16/FP16 MLP), the masters live here and every step
    refreshes the copies from them."""

    def __init__(self, field: PartitionedField, samp: Sampling, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15,
                 lambda_dist=0.01, master_tables=None, master_mlp=None, save_features: bool = True,
                 workspace_cap: int | None = None):
        """workspace_cap (bytes): bound the step's workspace; a batch whose
        one-pass workspace is larger runs in ray sub-batches (nerfxl_step)."""
        self.field = field
        self.workspace_cap = workspace_cap
        if save_features:
            # keep the forward's records (features, and for a 16-bit MLP the
            # tensor-core backward's geometry) instead of encoding again
            samp = dataclasses.replace(samp, flags=samp.flags | SAVE_FEATURES)
        self.samp = samp
        self.lr, self.beta1, self.beta2, self.eps, self.lambda_dist = lr, beta1, beta2, eps, lambda_dist

        def master(copy, given):
            if copy.dtype == torch.float32:
                return copy  # renders straight from the master
            m = given if given is not None else copy.float()
            return torch.as_tensor(m, dtype=torch.float32).to(field.device).reshape(copy.shape).contiguous()

        self.tables = master(field.tables, master_tables)
        self.mlp = master(field.mlp, master_mlp)
        z = torch.zeros_like
        self.grad_tables, self.grad_mlp = z(self.tables), z(self.mlp)
        self.m_tables, self.v_tables = z(self.tables), z(self.tables)
        self.m_mlp, self.v_mlp = z(self.mlp), z(self.mlp)
        self.step_count = 0
        self._ws = None
        self.loss = torch.zeros(3, dtype=torch.float32, device=field.device)

    def master_field(self) -> PartitionedField:
        """The FP32 masters as a field (shares their memory; no copy), e.g. for
        refreshing an occupancy grid while training with 16-bit copies."""
        f = self.field
        return PartitionedField(f.boxes, f.level_res, f.log2_T, self.tables, self.mlp, F=f.F, mlp_in=f.mlp_in,
                                width=f.width, device=f.device, arch=f.arch)

    def sub_batch(self, n_rays: int) -> int:
        """Rays per sub-batch of a step over n_rays under the workspace cap
        (n_rays itself when the one-pass workspace fits)."""
        fd, sd = self.field.desc(), self.samp.desc()
        need = int(N.lib().nerfxl_step_workspace_bytes(C_ref(fd), C_ref(sd), int(n_rays)))
        if self.workspace_cap is not None:
            need = min(need, int(self.workspace_cap))
        return int(N.lib().nerfxl_step_sub_batch(C_ref(fd), C_ref(sd), int(n_rays), need))

    def state_desc(self) -> N.TrainStateDesc:
        return N.TrainStateDesc(self.tables.data_ptr(), self.mlp.data_ptr(), self.grad_tables.data_ptr(),
                                self.grad_mlp.data_ptr(), self.m_tables.data_ptr(), self.v_tables.data_ptr(),
                                self.m_mlp.data_ptr(), self.v_mlp.data_ptr())

    def step(self, rays_o, rays_d, target, stream=None):
        o, d = _rays(rays_o, rays_d, self.field.device)
        tgt = torch.as_tensor(target, dtype=torch.float32).to(self.field.device).reshape(-1, 3).contiguous()
        R = o.shape[0]
        fd, sd = self.field.desc(), self.samp.desc()
        need = int(N.lib().nerfxl_step_workspace_bytes(C_ref(fd), C_ref(sd), R))
        if need == 0:
            N.check(N.E_INVALID, "nerfxl_step_workspace_bytes")
        if self.workspace_cap is not None:
            need = min(need, int(self.workspace_cap))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.field.device)
        self.step_count += 1
        opt = N.AdamDesc(float(self.lr), float(self.beta1), float(self.beta2), float(self.eps), self.step_count)
        stt = self.state_desc()
        st = N.lib().nerfxl_step(C_ref(fd), C_ref(sd), R, N._ptr(o), N._ptr(d), N._ptr(tgt), float(self.lambda_dist),
                                 ctypes_addr(stt), ctypes_addr(opt), N._ptr(self.loss), N._ptr(self._ws),
                                 self._ws.numel(), N._stream(stream))
        N.check(st, "nerfxl_step")
        return self.loss


def quantize_mlp_e4m3(mlp, mlp_in: int = 32, width: int = 64, device=None):
    """FP32 fused MLP blocks [K][P] -> (E4M3 bytes [K][P] uint8, scales [K][3]),
    on the device, by nerfxl_quantize_e4m3 (per region and layer: scale =
    max|W| / 448, W_q = e4m3(W / scale), so W ~= scale * W_q)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    m = torch.as_tensor(mlp, dtype=torch.float32).to(dev).contiguous()
    K = m.shape[0]
    q = torch.empty(m.shape, dtype=torch.uint8, device=dev)
    scales = torch.empty(K, 3, dtype=torch.float32, device=dev)
    N.check(N.lib().nerfxl_quantize_e4m3(K, int(mlp_in), int(width), N._ptr(m), N._ptr(q), N._ptr(scales),
                                         N._stream(torch.cuda.current_stream(dev))), "nerfxl_quantize_e4m3")
    return q, scales


def partition_boxes(points, root, levels: int):
    """Spatial partitioning (Sec. 4.4): 2^levels disjoint boxes [K][6] with
    balanced point counts, and the counts (host numpy arrays)."""
    pts = np.ascontiguousarray(np.asarray(points, np.float32).reshape(-1, 3))
    root = np.ascontiguousarray(np.asarray(root, np.float32).reshape(6))
    K = 1 << min(max(int(levels), 0), 10)  # out-of-range levels are refused by the library
    boxes = np.zeros((K, 6), np.float32)
    counts = np.zeros(K, np.int64)
    st = N.lib().nerfxl_partition(pts.ctypes.data, len(pts), root.ctypes.data, int(levels), boxes.ctypes.data,
                                  counts.ctypes.data)
    N.check(st, "nerfxl_partition")
    return boxes, counts


def region_chunks(workspace, K: int, stream=None):
    """Per-region chunk counts of the last sampling in a workspace (syncs)."""
    out = np.zeros(int(K), np.int32)
    N.check(N.lib().nerfxl_region_chunks(N._ptr(workspace), workspace.numel(), int(K), out.ctypes.data,
                                         N._stream(stream)), "nerfxl_region_chunks")
    return out


def workspace_stats(workspace, stream=None):
    """(samples, chunks) of the last sampling in a workspace (syncs)."""
    import ctypes

    ns, nc = ctypes.c_int64(0), ctypes.c_int64(0)
    N.check(N.lib().nerfxl_workspace_stats(N._ptr(workspace), workspace.numel(), ctypes.byref(ns), ctypes.byref(nc),
                                           N._stream(stream)), "nerfxl_workspace_stats")
    return int(ns.value), int(nc.value)
