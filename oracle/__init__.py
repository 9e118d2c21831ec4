"""NeRF-XL CPU oracle: ctypes front end of ``nerfxl_oracle.cpp``.

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product package
never imports this module, and this module never imports the product package.

Every function takes plain numpy arrays. Field parameters are handed over as
float64 (the values a GPU run uses, promoted exactly), rays and boxes as
float32, because the geometry/index path is prescribed in FP32 (Sec. 4.2:
samples are assigned by tile box and must agree bit for bit).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nerfxl_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


class _Field(C.Structure):
    _fields_ = [("K", C.c_int32), ("L", C.c_int32), ("F", C.c_int32), ("log2_T", C.c_int32),
                ("mlp_in", C.c_int32), ("W", C.c_int32), ("level_res", C.c_void_p),
                ("boxes", C.c_void_p), ("tables", C.c_void_p), ("mlp", C.c_void_p),
                ("occupancy", C.c_void_p), ("occ_res", C.c_int32), ("arch", C.c_int32)]


class _Sampling(C.Structure):
    _fields_ = [("S", C.c_int32), ("t_min", C.c_float)]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, IEEE semantics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        fp, sp = C.POINTER(_Field), C.POINTER(_Sampling)
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_threads.restype = C.c_int
        L.oracle_table_entries.restype = C.c_int64
        L.oracle_table_entries.argtypes = [C.c_int32, _i32p, C.c_int32]
        L.oracle_level_offset.restype = C.c_int64
        L.oracle_level_offset.argtypes = [C.c_int32, _i32p, C.c_int32, C.c_int32]
        L.oracle_level_dense.restype = C.c_int32
        L.oracle_level_dense.argtypes = [C.c_int32, _i32p, C.c_int32, C.c_int32]
        L.oracle_mlp_params.restype = C.c_int64
        L.oracle_mlp_params.argtypes = [C.c_int32, C.c_int32]
        L.oracle_segments.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, _i32p, _i32p, _f32p, _f32p, _i32p]
        L.oracle_intervals.restype = C.c_int
        L.oracle_intervals.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, C.c_int32, _i32p, _f32p, _f32p, _i32p]
        L.oracle_hash_indices.restype = C.c_int
        L.oracle_hash_indices.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, C.c_int32, _u32p]
        L.oracle_encode_points.argtypes = [fp, C.c_int64, _i32p, _f32p, _f64p, C.c_void_p]
        L.oracle_mlp.argtypes = [fp, C.c_int64, _i32p, _f64p, C.c_void_p, _f64p]
        L.oracle_density_params.restype = C.c_int64
        L.oracle_density_params.argtypes = [C.c_int32, C.c_int32]
        L.oracle_color_params.restype = C.c_int64
        L.oracle_color_params.argtypes = [C.c_int32]
        L.oracle_sh4.argtypes = [C.c_int64, _f64p, _f64p]
        L.oracle_render_samples.argtypes = [C.c_int64, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.oracle_render_local.argtypes = [C.c_int64, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.oracle_composite.argtypes = [C.c_int64, _f64p, _f64p]
        L.oracle_render.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, C.c_int32, _f64p, _f64p, _f64p, _f64p,
                                    _f64p, _i32p]
        L.oracle_loss.restype = C.c_double
        L.oracle_loss.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, _f32p, C.c_double]
        L.oracle_render_grad.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                         _f64p]
        L.oracle_loss_grad.restype = C.c_double
        L.oracle_loss_grad.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, _f32p, C.c_double, _f64p, _f64p]
        L.oracle_fd_grad.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, _f32p, C.c_double, _f64p, _f64p,
                                     C.c_int64, _i32p, _i64p, C.c_double, _f64p]
        L.oracle_adam.argtypes = [C.c_int64, _f64p, _f64p, _f64p, _f64p, C.c_int64, C.c_double, C.c_double,
                                  C.c_double, C.c_double]
        L.oracle_blob_render.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, C.c_int64, _f64p, _f64p, _f64p, _f64p]
        L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.oracle_relu_margin.argtypes = [fp, sp, C.c_int64, _f32p, _f32p, _f64p]
        L.oracle_camera_rays.argtypes = [_f32p, C.c_int32, C.c_int32, C.c_int64, C.c_int64, _f32p, _f32p]
        L.oracle_occupancy_update.argtypes = [fp, C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_double, _f64p,
                                              _u32p, C.c_void_p]
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def threads() -> int:
    return int(lib().oracle_threads())


def table_entries(level_res, log2_T: int) -> int:
    r = np.ascontiguousarray(level_res, dtype=np.int32)
    return int(lib().oracle_table_entries(len(r), r, int(log2_T)))


def level_offset(level_res, log2_T: int, l: int) -> int:
    r = np.ascontiguousarray(level_res, dtype=np.int32)
    return int(lib().oracle_level_offset(len(r), r, int(log2_T), int(l)))


def level_dense(level_res, log2_T: int, l: int) -> bool:
    r = np.ascontiguousarray(level_res, dtype=np.int32)
    return bool(lib().oracle_level_dense(len(r), r, int(log2_T), int(l)))


def mlp_params(mlp_in: int, W: int) -> int:
    return int(lib().oracle_mlp_params(int(mlp_in), int(W)))


class Field:
    """A host-side field description the oracle reads.

    boxes [K][6] float32; tables [K][E][F] and mlp [K][P] promoted to float64.
    """

    def __init__(self, boxes, level_res, log2_T, F, mlp_in, W, tables, mlp, occupancy=None, occ_res: int = 0,
                 arch: int = 0):
        self.boxes = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 6)
        self.level_res = np.ascontiguousarray(level_res, dtype=np.int32)
        self.K = self.boxes.shape[0]
        self.L = len(self.level_res)
        self.F, self.log2_T, self.mlp_in, self.W = int(F), int(log2_T), int(mlp_in), int(W)
        self.E = table_entries(self.level_res, self.log2_T)
        self.arch = int(arch)
        self.P = mlp_params(self.mlp_in, self.W)
        self.tables = np.ascontiguousarray(tables, dtype=np.float64).reshape(self.K, self.E, self.F)
        if self.arch == 1:
            # split representation: [K][density block] then the shared colour block, flat
            self.Pd = density_params(self.mlp_in, self.W)
            self.Pc = color_params(self.W)
            self.mlp = np.ascontiguousarray(mlp, dtype=np.float64).reshape(self.K * self.Pd + self.Pc)
        else:
            self.mlp = np.ascontiguousarray(mlp, dtype=np.float64).reshape(self.K, self.P)
        # optional occupancy grid: [K][ceil(G^3/32)] uint32 cell bits, G = occ_res
        self.occ_res = int(occ_res)
        self.occupancy = None
        if occupancy is not None:
            self.occupancy = np.ascontiguousarray(occupancy, dtype=np.uint32).reshape(self.K, occupancy_words(occ_res))

    def with_params(self, tables, mlp) -> "Field":
        return Field(self.boxes, self.level_res, self.log2_T, self.F, self.mlp_in, self.W, tables, mlp,
                     self.occupancy, self.occ_res, self.arch)

    def with_occupancy(self, occupancy, occ_res: int) -> "Field":
        return Field(self.boxes, self.level_res, self.log2_T, self.F, self.mlp_in, self.W, self.tables, self.mlp,
                     occupancy, occ_res, self.arch)

    def struct(self, tables=None, mlp=None) -> _Field:
        t = self.tables if tables is None else tables
        m = self.mlp if mlp is None else mlp
        occ = None if self.occupancy is None else self.occupancy.ctypes.data
        return _Field(self.K, self.L, self.F, self.log2_T, self.mlp_in, self.W, self.level_res.ctypes.data,
                      self.boxes.ctypes.data, t.ctypes.data, m.ctypes.data, occ, self.occ_res, self.arch)


def occupancy_words(G: int) -> int:
    """32-bit words of one region's G^3-cell occupancy bitfield."""
    return (int(G) ** 3 + 31) // 32


def _samp(S: int, t_min: float = 0.0) -> _Sampling:
    return _Sampling(int(S), float(t_min))


def _rays(o, d):
    o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
    assert o.shape == d.shape
    return o, d


def segments(field: Field, S: int, o, d):
    """Per ray: nseg, and region/t0/t1/n_intervals of each segment ([R][K])."""
    o, d = _rays(o, d)
    R, K = o.shape[0], field.K
    nseg = np.zeros(R, np.int32)
    region = np.full((R, K), -1, np.int32)
    t0 = np.zeros((R, K), np.float32)
    t1 = np.zeros((R, K), np.float32)
    nint = np.zeros((R, K), np.int32)
    fs = field.struct()
    lib().oracle_segments(C.byref(fs), C.byref(_samp(S)), R, o, d, nseg, region, t0, t1, nint)
    return nseg, region, t0, t1, nint


def intervals(field: Field, S: int, o, d, max_int: int):
    o, d = _rays(o, d)
    R = o.shape[0]
    count = np.zeros(R, np.int32)
    a = np.zeros((R, max_int), np.float32)
    b = np.zeros((R, max_int), np.float32)
    region = np.full((R, max_int), -1, np.int32)
    fs = field.struct()
    rc = lib().oracle_intervals(C.byref(fs), C.byref(_samp(S)), R, o, d, max_int, count, a, b, region)
    if rc != 0:
        raise ValueError("a ray has more intervals than max_int")
    return count, a, b, region


def hash_indices(field: Field, S: int, o, d, max_int: int):
    o, d = _rays(o, d)
    R = o.shape[0]
    idx = np.zeros((R, max_int, field.L, 8), np.uint32)
    fs = field.struct()
    rc = lib().oracle_hash_indices(C.byref(fs), C.byref(_samp(S)), R, o, d, max_int, idx)
    if rc != 0:
        raise ValueError("a ray has more intervals than max_int")
    return idx


def encode_points(field: Field, region, x, want_idx: bool = False):
    region = np.ascontiguousarray(region, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    n = x.shape[0]
    feat = np.zeros((n, field.mlp_in), np.float64)
    idx = np.zeros((n, field.L, 8), np.uint32) if want_idx else None
    fs = field.struct()
    lib().oracle_encode_points(C.byref(fs), n, region, x, feat, None if idx is None else idx.ctypes.data)
    return (feat, idx) if want_idx else feat


def mlp(field: Field, region, feat, dirs=None):
    """Raw outputs [n][4] (log density, three colour logits); the split
    representation's colour also takes the unit view directions dirs [n][3]."""
    region = np.ascontiguousarray(region, dtype=np.int32)
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    n = feat.shape[0]
    o = np.zeros((n, 4), np.float64)
    dv = None
    if dirs is not None:
        dv = np.ascontiguousarray(dirs, dtype=np.float32).reshape(n, 3)
    fs = field.struct()
    lib().oracle_mlp(C.byref(fs), n, region, feat, None if dv is None else dv.ctypes.data, o)
    return o


def density_params(mlp_in: int, W: int) -> int:
    return int(lib().oracle_density_params(int(mlp_in), int(W)))


def color_params(W: int) -> int:
    return int(lib().oracle_color_params(int(W)))


def sh4(dirs):
    """Real spherical harmonics of degrees 0..3 (16 per direction)."""
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(d), 16))
    lib().oracle_sh4(len(d), d, out)
    return out


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def render_samples(seg_of, sigma, rgb, tbar, delta):
    """Render explicit interval values: (single-pass out[7], partitioned out[7]).

    out = C[3], D, A, L_dist, T_final."""
    seg_of = np.ascontiguousarray(seg_of, dtype=np.int32)
    sigma, rgb, tbar, delta = _f64(sigma), _f64(rgb).reshape(-1, 3), _f64(tbar), _f64(delta)
    s1 = np.zeros(7)
    s2 = np.zeros(7)
    lib().oracle_render_samples(len(sigma), seg_of, sigma, rgb, tbar, delta, s1, s2)
    return s1, s2


def render_local(sigma, rgb, tbar, delta):
    """Segment partial {tau, C[3], A, D, L}."""
    sigma, rgb, tbar, delta = _f64(sigma), _f64(rgb).reshape(-1, 3), _f64(tbar), _f64(delta)
    p = np.zeros(7)
    lib().oracle_render_local(len(sigma), sigma, rgb, tbar, delta, p)
    return p


def composite(parts):
    parts = _f64(parts).reshape(-1, 7)
    out = np.zeros(7)
    lib().oracle_composite(parts.shape[0], parts, out)
    return out


def render(field: Field, S: int, o, d, mode: int = 0):
    """mode 0: single pass; mode 1: partitioned (Algorithm 1/2).

    Returns dict rgb [R][3], depth, opacity, dist, tfinal, n_samples [R]."""
    o, d = _rays(o, d)
    R = o.shape[0]
    out = {k: np.zeros(R) for k in ("depth", "opacity", "dist", "tfinal")}
    out["rgb"] = np.zeros((R, 3))
    out["n_samples"] = np.zeros(R, np.int32)
    fs = field.struct()
    lib().oracle_render(C.byref(fs), C.byref(_samp(S)), R, o, d, int(mode), out["rgb"], out["depth"],
                        out["opacity"], out["dist"], out["tfinal"], out["n_samples"])
    return out


def loss(field: Field, S: int, o, d, target, lam: float) -> float:
    o, d = _rays(o, d)
    target = np.ascontiguousarray(target, dtype=np.float32).reshape(-1, 3)
    fs = field.struct()
    return float(lib().oracle_loss(C.byref(fs), C.byref(_samp(S)), o.shape[0], o, d, target, float(lam)))


def loss_grad(field: Field, S: int, o, d, target, lam: float):
    """Returns (loss, g_tables [K][E][F], g_mlp [K][P]) in float64."""
    o, d = _rays(o, d)
    target = np.ascontiguousarray(target, dtype=np.float32).reshape(-1, 3)
    gt = np.zeros_like(field.tables)
    gm = np.zeros_like(field.mlp)
    fs = field.struct()
    L = lib().oracle_loss_grad(C.byref(fs), C.byref(_samp(S)), o.shape[0], o, d, target, float(lam), gt, gm)
    return float(L), gt, gm


def render_grad(field: Field, S: int, o, d, gC, gD, gA, gL):
    """Adjoint of render for output adjoints; returns (g_tables, g_mlp)."""
    o, d = _rays(o, d)
    R = o.shape[0]
    f = lambda a, shp: np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shp))
    gC, gD, gA, gL = f(gC, (R, 3)), f(gD, (R,)), f(gA, (R,)), f(gL, (R,))
    gt = np.zeros_like(field.tables)
    gm = np.zeros_like(field.mlp)
    fs = field.struct()
    lib().oracle_render_grad(C.byref(fs), C.byref(_samp(S)), R, o, d, gC, gD, gA, gL, gt, gm)
    return gt, gm


def fd_grad(field: Field, S: int, o, d, target, lam: float, which, idx, eps: float = 1e-3):
    """Central differences of the loss at the listed coordinates.

    which[c] = 0 -> flat index into tables, 1 -> flat index into mlp."""
    o, d = _rays(o, d)
    target = np.ascontiguousarray(target, dtype=np.float32).reshape(-1, 3)
    which = np.ascontiguousarray(which, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    t = field.tables.copy()
    m = field.mlp.copy()
    out = np.zeros(len(idx))
    fs = field.struct(t, m)
    lib().oracle_fd_grad(C.byref(fs), C.byref(_samp(S)), o.shape[0], o, d, target, float(lam), t, m, len(idx),
                         which, idx, float(eps), out)
    return out


def adam(p, m, v, g, step: int, lr: float, b1: float, b2: float, eps: float):
    """One Adam step in place on float64 arrays."""
    for a in (p, m, v, g):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oracle_adam(p.size, p, m, v, g, int(step), float(lr), float(b1), float(b2), float(eps))


def blob_render(field: Field, S: int, o, d, blobs):
    """Target colours of the Gaussian-blob field; returns (rgb, depth, opacity)."""
    o, d = _rays(o, d)
    R = o.shape[0]
    blobs = _f64(blobs).reshape(-1, 8)
    rgb = np.zeros((R, 3))
    depth = np.zeros(R)
    op = np.zeros(R)
    fs = field.struct()
    lib().oracle_blob_render(C.byref(fs), C.byref(_samp(S)), R, o, d, blobs.shape[0], blobs, rgb, depth, op)
    return rgb, depth, op


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 128-bit counter and 64-bit key (4 and 2 uint32 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(c, k, out)
    return out


def occupancy_update(field: Field, G: int, step: int, seed: int, decay: float, threshold: float, density,
                     want_points: bool = False):
    """One refresh of every region's G^3 occupancy grid from the field.

    density [K][G^3] float64 is updated in place to max(decay * density,
    sigma(point)); returns the new bits [K][words] (and the drawn region
    coordinates [K][G^3][3] if asked)."""
    assert density.dtype == np.float64 and density.flags.c_contiguous and density.size == field.K * G ** 3
    bits = np.zeros((field.K, occupancy_words(G)), np.uint32)
    pts = np.zeros((field.K, G ** 3, 3), np.float32) if want_points else None
    fs = field.struct()
    lib().oracle_occupancy_update(C.byref(fs), int(G), int(step), int(seed), float(decay), float(threshold), density,
                                  bits, None if pts is None else pts.ctypes.data)
    return (bits, pts) if want_points else bits


def relu_margin(field: Field, S: int, o, d):
    """Per ray, the smallest distance of any evaluated sample's hidden unit
    from its ReLU kink, relative to the scale that unit's rounding error
    grows with (see relu_margin_sample in the C source); +inf for a ray
    without evaluated samples. A test diagnostic: rays whose margin is within
    a few orders of magnitude of the FP32 unit roundoff may take the other
    ReLU decision in FP32."""
    o, d = _rays(o, d)
    out = np.zeros(o.shape[0])
    fs = field.struct()
    lib().oracle_relu_margin(C.byref(fs), C.byref(_samp(S)), o.shape[0], o, d, out)
    return out


def camera_rays(origin, right, up, forward, tan_half_fov: float, width: int, height: int, first: int = 0,
                count: int | None = None):
    """Pinhole rays of pixels first..first+count-1 (row-major) in the
    prescribed FP32 operation order; returns (o, d) [count][3] float32."""
    cam = np.concatenate([np.asarray(v, np.float32).reshape(3) for v in (origin, right, up, forward)] +
                         [np.asarray([tan_half_fov], np.float32)])
    cam = np.ascontiguousarray(cam, dtype=np.float32)
    count = int(width) * int(height) - int(first) if count is None else int(count)
    o = np.zeros((count, 3), np.float32)
    d = np.zeros((count, 3), np.float32)
    lib().oracle_camera_rays(cam, int(width), int(height), int(first), count, o, d)
    return o, d
