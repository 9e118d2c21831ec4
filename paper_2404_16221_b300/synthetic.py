"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module holds no arithmetic of the method itself: it only draws rays,
region boxes, parameter blocks, blob targets and render requests, with the
shapes of the paper's captures (object-centric, aerial and street-height
cameras; Table 1 lists the captures, whose data are not available here).
Every stream is a separate numpy ``Generator`` keyed by (seed, purpose), so a
change to one stream never shifts another.

Workloads (seed = 1000 + workload index):
  * ``unit``   -- K=1 over [-0.5,0.5]^3, L=8 F=2 T=2^14, 16->256, 4096 rays from
    a radius-2 sphere towards random points of the box, S=64.
  * ``grid8``  -- K=8 (2x2x2 over [-1,1]^3), L=16 F=2 T=2^19, 16->2048, 64
    pinhole cameras (64x64 px, FOV 50 deg) on a radius-3 Fibonacci sphere, S=128.
  * ``train8`` -- the grid8 scene trained towards 200 Gaussian blobs.
  * ``city32`` -- K=32 (8x4x1 slabs over [-4,4]x[-2,2]x[0,0.5]), L=16 F=2
    T=2^21, 16->8192, 2^20 rays (half aerial, half street height), S=256.
  * ``serve32`` -- the city32 field with a Poisson stream of render requests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_STREAMS = {"rays": 1, "tables": 2, "mlp": 3, "blobs": 4, "batch": 5, "requests": 6, "subset": 7, "misc": 8,
            "content": 9, "ray_samples": 10, "split_mlp": 11}


def rng(seed: int, purpose: str) -> np.random.Generator:
    """Independent PCG64 stream for (seed, purpose)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), _STREAMS[purpose]])))


def level_resolutions(n_min: int, n_max: int, levels: int) -> np.ndarray:
    """Per-level grid resolution N_l = floor(N_min * b^l), b = (N_max/N_min)^(1/(L-1)).

    This is the geometric level schedule of the cited Instant-NGP encoding (the
    paper adopts that encoding per tile, App. A.1); a 1e-9 guard keeps exact
    powers (128, 1024, 8192, ...) from rounding down. The result is passed to
    both the oracle and the CUDA library as an explicit array.
    """
    if levels == 1:
        return np.array([n_min], np.int32)
    b = math.exp((math.log(n_max) - math.log(n_min)) / (levels - 1))
    return np.array([int(math.floor(n_min * b ** l + 1e-9)) for l in range(levels)], np.int32)


def grid_boxes(lo, hi, counts) -> np.ndarray:
    """Disjoint axis-aligned boxes tiling [lo, hi] as counts[0] x counts[1] x counts[2].

    Shared faces are written from the same float32 values, so neighbouring
    boxes agree on them bit for bit. Region id = x + nx*(y + ny*z).
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    edges = [np.linspace(lo[a], hi[a], counts[a] + 1).astype(np.float32) for a in range(3)]
    boxes = []
    for z in range(counts[2]):
        for y in range(counts[1]):
            for x in range(counts[0]):
                boxes.append([edges[0][x], edges[1][y], edges[2][z], edges[0][x + 1], edges[1][y + 1],
                              edges[2][z + 1]])
    return np.array(boxes, np.float32)


def max_segments_for_grid(counts) -> int:
    """Largest number of boxes a straight ray can cross in a regular grid."""
    return int(sum(counts) - 2)


def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def sphere_rays(n: int, radius: float, box_lo, box_hi, seed: int):
    """Origins uniform on a sphere, directions towards uniform points of a box."""
    g = rng(seed, "rays")
    o = radius * _normalize(g.standard_normal((n, 3)))
    tgt = g.uniform(box_lo, box_hi, size=(n, 3))
    d = _normalize(tgt - o)
    return o.astype(np.float32), d.astype(np.float32)


def look_at(eye, target, up=(0.0, 0.0, 1.0)):
    f = _normalize(np.asarray(target, np.float64) - eye)
    upv = np.asarray(up, np.float64)
    if abs(float(np.dot(f, upv))) > 0.999:
        upv = np.array([0.0, 1.0, 0.0])
    r = _normalize(np.cross(f, upv))
    u = np.cross(r, f)
    return r, u, f


def pinhole_rays(eye, target, H: int, W: int, fov_deg: float, up=(0.0, 0.0, 1.0)):
    """Row-major pixel-centre rays of one pinhole camera (vertical FOV)."""
    eye = np.asarray(eye, np.float64)
    r, u, f = look_at(eye, target, up)
    tan = math.tan(math.radians(fov_deg) / 2.0)
    js, is_ = np.meshgrid(np.arange(W), np.arange(H))
    x = ((js + 0.5) / W * 2.0 - 1.0) * tan * (W / H)
    y = (1.0 - (is_ + 0.5) / H * 2.0) * tan
    d = x[..., None] * r + y[..., None] * u + f
    d = _normalize(d.reshape(-1, 3))
    o = np.broadcast_to(eye, d.shape)
    return o.astype(np.float32), d.astype(np.float32)


def fibonacci_sphere(n: int, radius: float):
    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    theta = math.pi * (1.0 + 5.0 ** 0.5) * i
    return radius * np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], -1)


def orbit_cameras(n_cams: int, radius: float, H: int, W: int, fov_deg: float, first: int = 0, total: int = 0):
    """Rays of cameras first..first+n_cams-1 of a total-camera Fibonacci sphere
    (total defaults to n_cams), each looking at the origin."""
    total = total or n_cams
    os_, ds = [], []
    eyes = fibonacci_sphere(total, radius)
    for eye in eyes[first:first + n_cams]:
        o, d = pinhole_rays(eye, (0.0, 0.0, 0.0), H, W, fov_deg)
        os_.append(o)
        ds.append(d)
    return np.concatenate(os_), np.concatenate(ds)


def city_rays(n: int, seed: int, extent=(4.0, 2.0, 0.5)):
    """Half aerial rays (origins at z in [2,3] over the footprint, towards random
    ground points), half street-height rays (origins inside the slab at z=0.1,
    near-horizontal directions)."""
    g = rng(seed, "rays")
    ex, ey, ez = extent
    na = n // 2
    ns = n - na
    oa = np.stack([g.uniform(-ex, ex, na), g.uniform(-ey, ey, na), g.uniform(2.0, 3.0, na)], -1)
    ta = np.stack([g.uniform(-ex, ex, na), g.uniform(-ey, ey, na), g.uniform(0.0, 0.1 * ez, na)], -1)
    da = _normalize(ta - oa)
    os_ = np.stack([g.uniform(-0.95 * ex, 0.95 * ex, ns), g.uniform(-0.95 * ey, 0.95 * ey, ns), np.full(ns, 0.1)],
                   -1)
    az = g.uniform(0.0, 2.0 * math.pi, ns)
    el = g.uniform(-0.05, 0.15, ns)
    ds = np.stack([np.cos(az) * np.cos(el), np.sin(az) * np.cos(el), np.sin(el)], -1)
    o = np.concatenate([oa, os_]).astype(np.float32)
    d = _normalize(np.concatenate([da, ds])).astype(np.float32)
    return o, d


def gaussian_params(shape, std: float, seed: int, purpose: str) -> np.ndarray:
    return (std * rng(seed, purpose).standard_normal(shape)).astype(np.float32)


def uniform_params(shape, scale: float, seed: int, purpose: str) -> np.ndarray:
    return rng(seed, purpose).uniform(-scale, scale, size=shape).astype(np.float32)


def blobs(n: int, seed: int, lo=-0.8, hi=0.8, s_range=(0.05, 0.2), a_range=(5.0, 50.0)):
    """[n][8] = mu xyz ~ U[lo,hi]^3, s ~ logU[s_range], a ~ U[a_range], rgb ~ U[0,1]^3."""
    g = rng(seed, "blobs")
    mu = g.uniform(lo, hi, (n, 3))
    s = np.exp(g.uniform(math.log(s_range[0]), math.log(s_range[1]), n))
    a = g.uniform(a_range[0], a_range[1], n)
    rgb = g.uniform(0.0, 1.0, (n, 3))
    return np.concatenate([mu, s[:, None], a[:, None], rgb], 1)


def sparse_blobs(seed: int):
    """A sparse blob scene: 24 small dense blobs in [-0.6, 0.6]^3 (s in
    [0.04, 0.1], a in [20, 100]); about 10% of the [-1, 1]^3 volume has
    density above 0.4, the share of empty space of real captures."""
    return blobs(24, seed, -0.6, 0.6, (0.04, 0.1), (20.0, 100.0))


def blob_occupancy(boxes, blob_params, G: int, threshold: float) -> np.ndarray:
    """A stand-in for the occupancy grid of a field trained on a blob scene:
    per region [K][ceil(G^3/32)] uint32 words whose bit c % 32 of word c / 32
    is set where the blob density at the centre of cell c = x + G (y + G z)
    exceeds threshold."""
    boxes = np.asarray(boxes, np.float64).reshape(-1, 6)
    K = len(boxes)
    c = (np.arange(G) + 0.5) / G
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")  # x fastest in C order
    u = np.stack([cx, cy, cz], -1).reshape(-1, 3)
    words = (G ** 3 + 31) // 32
    out = np.zeros((K, words), np.uint32)
    for k in range(K):
        x = boxes[k, :3] + u * (boxes[k, 3:] - boxes[k, :3])
        sig = np.zeros(len(x))
        for q in blob_params:
            sig += q[4] * np.exp(-((x - q[:3]) ** 2).sum(-1) / (2.0 * q[3] ** 2))
        on = np.zeros(words * 32, bool)
        on[:G ** 3] = sig > threshold
        out[k] = np.packbits(on.reshape(-1, 32), axis=-1, bitorder="little").view(np.uint32).reshape(-1)
    return out


@dataclasses.dataclass
class Workload:
    name: str
    seed: int
    boxes: np.ndarray
    level_res: np.ndarray
    log2_T: int
    F: int
    mlp_in: int
    W: int
    S: int
    max_segments: int
    n_rays: int

    @property
    def K(self) -> int:
        return int(self.boxes.shape[0])

    @property
    def L(self) -> int:
        return int(len(self.level_res))


def workload(name: str, n_rays: int | None = None) -> Workload:
    if name == "unit":
        return Workload("unit", 1000, grid_boxes([-0.5] * 3, [0.5] * 3, (1, 1, 1)), level_resolutions(16, 256, 8), 14,
                        2, 32, 64, 64, 1, n_rays or 4096)
    if name in ("grid8", "train8"):
        seed = 1001 if name == "grid8" else 1002
        return Workload(name, seed, grid_boxes([-1.0] * 3, [1.0] * 3, (2, 2, 2)), level_resolutions(16, 2048, 16),
                        19, 2, 32, 64, 128, max_segments_for_grid((2, 2, 2)), n_rays or (1 << 18))
    if name in ("city32", "serve32"):
        seed = 1003 if name == "city32" else 1004
        return Workload(name, seed, grid_boxes([-4.0, -2.0, 0.0], [4.0, 2.0, 0.5], (8, 4, 1)),
                        level_resolutions(16, 8192, 16), 21, 2, 32, 64, 256, max_segments_for_grid((8, 4, 1)),
                        n_rays or (1 << 20))
    raise KeyError(name)


def workload_rays(w: Workload, n: int | None = None, seed: int | None = None):
    """Rays of a workload (the first n of its ray set)."""
    n = n or w.n_rays
    seed = w.seed if seed is None else seed
    if w.name == "unit":
        return sphere_rays(n, 2.0, [-0.5] * 3, [0.5] * 3, seed)
    if w.name in ("grid8", "train8"):
        n_cams = max(1, -(-n // 4096))
        o, d = orbit_cameras(n_cams, 3.0, 64, 64, 50.0, 0, max(64, n_cams))
        return o[:n].copy(), d[:n].copy()
    return city_rays(n, seed)


def field_params(w: Workload, E: int, P: int, table_std: float = 1.0, mlp_std: float = 0.1,
                 table_init: str = "normal"):
    """Tables [K][E][F] and MLP blocks [K][P] (float32).

    E (entries per region) and P (MLP parameters per region) are layout facts
    the caller obtains from the library that consumes the arrays. MLP blocks
    are W1 [mlp_in][W], W2 [W][W], W3 [W][4], row-major.
    """
    if table_init == "normal":
        tables = gaussian_params((w.K, E, w.F), table_std, w.seed, "tables")
    else:
        tables = uniform_params((w.K, E, w.F), table_std, w.seed, "tables")
    mlp = gaussian_params((w.K, P), mlp_std, w.seed, "mlp")
    return tables, mlp


def split_mlp_params(w: Workload, n_params: int, mlp_std: float = 0.1):
    """MLP parameters of the split representation (per-region density blocks
    followed by the shared colour block, flat float32 of n_params values, the
    size the consuming library reports), N(0, mlp_std)."""
    return gaussian_params((n_params,), mlp_std, w.seed, "split_mlp")


def subset(n_total: int, n: int, seed: int) -> np.ndarray:
    """Sorted seeded subset of ray indices."""
    g = rng(seed, "subset")
    return np.sort(g.choice(n_total, size=n, replace=False))


def request_stream(n_requests: int, rate_hz: float, seed: int, h_min=64, h_max=1080, w_min=64, w_max=1920):
    """Poisson render requests: (arrival_s, H, W, eye [n][3], target [n][3]).

    H ~ logU[h_min, h_max], W = clamp(round(H * U[1, 16/9]), w_min, w_max);
    poses: half aerial, half street height over the city footprint.
    """
    g = rng(seed, "requests")
    gaps = g.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    H = np.exp(g.uniform(math.log(h_min), math.log(h_max), n_requests)).round().astype(np.int64)
    Wd = np.clip((H * g.uniform(1.0, 16.0 / 9.0, n_requests)).round(), w_min, w_max).astype(np.int64)
    aerial = g.uniform(size=n_requests) < 0.5
    eye_a = np.stack([g.uniform(-4, 4, n_requests), g.uniform(-2, 2, n_requests), g.uniform(2, 3, n_requests)], -1)
    eye_s = np.stack([g.uniform(-3.8, 3.8, n_requests), g.uniform(-1.9, 1.9, n_requests),
                      np.full(n_requests, 0.1)], -1)
    eye = np.where(aerial[:, None], eye_a, eye_s)
    tgt = np.stack([g.uniform(-4, 4, n_requests), g.uniform(-2, 2, n_requests), g.uniform(0.0, 0.3, n_requests)], -1)
    return t, H, Wd, eye, tgt


def field_params_device(w: Workload, E: int, P: int, device, table_std: float = 1.0, mlp_std: float = 0.1):
    """Large parameter blocks drawn directly on the GPU (seeded torch Philox),
    for full-size throughput runs; tables [K][E][F] and MLP [K][P] float32."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(w.seed) * 7919 + _STREAMS["tables"])
    tables = torch.randn((w.K, E, w.F), generator=g, device=device) * table_std
    g.manual_seed(int(w.seed) * 7919 + _STREAMS["mlp"])
    mlp = torch.randn((w.K, P), generator=g, device=device) * mlp_std
    return tables, mlp


# ---------------------------------------------------------------------------
# Scene content for the spatial partitioning (Sec. 4.4): an SfM-like point
# cloud, or samples of training rays when no point cloud is available.

def scene_root(w: Workload) -> np.ndarray:
    """The scene's bounding box [6] (min xyz, max xyz): the union of the
    workload's grid boxes."""
    b = np.asarray(w.boxes, np.float32)
    return np.concatenate([b[:, :3].min(0), b[:, 3:].max(0)]).astype(np.float32)


def content_points(w: Workload, n: int, seed: int | None = None, clusters: int = 24) -> np.ndarray:
    """SfM-like point cloud [n][3] float32: a mixture of anisotropic Gaussian
    clusters (centres uniform in the scene box, per-axis sizes log-uniform in
    2%..20% of the box extent, weights uniform in [0.2, 1]) clipped to the
    box, so content is uneven across space as in real captures."""
    g = rng(w.seed if seed is None else seed, "content")
    root = scene_root(w)
    lo, hi = root[:3].astype(np.float64), root[3:].astype(np.float64)
    ext = hi - lo
    centres = lo + g.uniform(0.0, 1.0, (clusters, 3)) * ext
    sizes = np.exp(g.uniform(np.log(0.02), np.log(0.2), (clusters, 3))) * ext
    weights = g.uniform(0.2, 1.0, clusters)
    which = g.choice(clusters, size=n, p=weights / weights.sum())
    pts = centres[which] + g.standard_normal((n, 3)) * sizes[which]
    return np.clip(pts, lo, hi).astype(np.float32)


def ray_sample_points(rays_o, rays_d, root, n_per_ray: int, seed: int) -> np.ndarray:
    """Samples of training rays inside the scene box: per ray, n_per_ray
    stratified samples (one uniform draw per stratum) of the ray's overlap
    [t0, t1] with the box; rays that miss the box give none."""
    o = np.asarray(rays_o, np.float64)
    d = np.asarray(rays_d, np.float64)
    root = np.asarray(root, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta = (root[:3] - o) * inv
        tb = (root[3:] - o) * inv
    t0 = np.nanmax(np.minimum(ta, tb), axis=1)
    t1 = np.nanmin(np.maximum(ta, tb), axis=1)
    t0 = np.maximum(t0, 0.0)
    hit = t1 > t0
    o, d, t0, t1 = o[hit], d[hit], t0[hit], t1[hit]
    g = rng(seed, "ray_samples")
    j = (np.arange(n_per_ray)[None, :] + g.uniform(0.0, 1.0, (len(o), n_per_ray))) / n_per_ray
    t = t0[:, None] + j * (t1 - t0)[:, None]
    pts = o[:, None, :] + t[..., None] * d[:, None, :]
    return np.clip(pts.reshape(-1, 3), root[:3], root[3:]).astype(np.float32)


def one_sided_rays(w: Workload, n: int, seed: int, x_max: float = -1.0):
    """Rays of a trajectory that covers one side of the scene: the workload's
    rays whose origin has x < x_max (uneven training-view coverage, the case
    the spatial partitioning balances)."""
    o, d = workload_rays(w, 4 * n, seed=seed)
    keep = np.nonzero(o[:, 0] < x_max)[0][:n]
    return o[keep].copy(), d[keep].copy()
