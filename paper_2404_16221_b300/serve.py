"""Continuous-batching render server over the C ABI (nerfxl_render_cameras).

Requests (a pinhole camera and an image size) arrive over time. The engine
keeps the field and every admitted request's state on the device: its camera
in a device camera table and its output image in a fixed-capacity device
arena. A request is admitted when its image fits in the arena (admission by
memory). Each iteration forms a batch of up to ``max_batch_rays`` pixels from
the admitted requests, by default those with the fewest pixels left first
(policy "srpt"; "fifo" takes them in arrival order, "fair" splits the batch
evenly by water-filling), so a large image does not hold the small requests
admitted behind it; a large request spans several batches. The batch is
rendered with one call,
whose field kernel is a persistent launch over the whole batch. At most two
batches are in flight, so requests that arrive while the GPU works are
admitted into the next batch. Completion times are device times (CUDA events
aligned to the host clock at start), so latency = device completion - arrival.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import time
from collections import deque

import numpy as np
import torch

from . import api
from . import native as N


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    height: int
    width: int
    eye: tuple
    target: tuple
    fov_deg: float = 60.0
    # filled by the engine
    slot: int = -1          # first pixel slot in the arena
    cam: int = -1           # camera table entry
    next_pixel: int = 0
    done_s: float = math.nan
    result: dict | None = None

    @property
    def pixels(self) -> int:
        return int(self.height) * int(self.width)


class Arena:
    """First-fit allocator of pixel slots (the device image memory)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free = [(0, self.capacity)]  # sorted (start, length)

    def alloc(self, n: int) -> int:
        for i, (s, l) in enumerate(self.free):
            if l >= n:
                if l == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (s + n, l - n)
                return s
        return -1

    def release(self, s: int, n: int):
        self.free.append((s, n))
        self.free.sort()
        merged = []
        for a, l in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + l)
            else:
                merged.append((a, l))
        self.free = merged

    @property
    def used(self) -> int:
        return self.capacity - sum(l for _, l in self.free)


def camera_desc(req: Request) -> N.CameraDesc:
    eye = np.asarray(req.eye, np.float64)
    f = np.asarray(req.target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(float(f @ up)) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    c = N.CameraDesc()
    for i in range(3):
        c.origin[i], c.right[i], c.up[i], c.forward[i] = eye[i], r[i], u[i], f[i]
    c.tan_half_fov = math.tan(math.radians(req.fov_deg) / 2.0)
    c.width, c.height, c.reserved = int(req.width), int(req.height), 0
    return c


def camera_rays(req: Request, device=None):
    """The rays nerfxl_render_cameras renders for a request, generated by the
    library's own ray generator (nerfxl_debug_camera_rays); returns host
    (o, d) [H*W][3] float32. Used to check a served image against a plain
    render of the same rays."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    n = req.pixels
    cam = camera_desc(req)
    item = N.RayItemDesc(0, 0, 0, 0, n)
    cam_d = torch.frombuffer(bytearray(bytes(cam)), dtype=torch.uint8).to(dev)
    item_d = torch.frombuffer(bytearray(bytes(item)), dtype=torch.uint8).to(dev)
    o = torch.empty(n, 3, device=dev)
    d = torch.empty(n, 3, device=dev)
    N.check(N.lib().nerfxl_debug_camera_rays(n, 1, N._ptr(item_d), N._ptr(cam_d), 1, N._ptr(o), N._ptr(d),
                                             N._stream(torch.cuda.current_stream(dev))), "nerfxl_debug_camera_rays")
    return o.cpu().numpy(), d.cpu().numpy()


class ServeEngine:
    def __init__(self, field: api.PartitionedField, samp: api.Sampling, max_batch_rays: int = 1 << 20,
                 arena_pixels: int = 1 << 26, max_cameras: int = 4096, max_inflight: int = 2,
                 one_at_a_time: bool = False, keep_results: bool = False, policy: str = "srpt"):
        self.field, self.samp = field, samp
        self.dev = field.device
        self.max_batch = int(max_batch_rays)
        self.one_at_a_time = one_at_a_time
        if policy not in ("fair", "fifo", "srpt"):
            raise ValueError("policy must be fair, fifo or srpt")
        self.policy = policy
        self.max_inflight = 1 if one_at_a_time else int(max_inflight)
        self.keep_results = keep_results
        self.arena = Arena(arena_pixels)
        self.rgb = torch.empty(arena_pixels, 3, device=self.dev)
        self.depth = torch.empty(arena_pixels, device=self.dev)
        self.opacity = torch.empty(arena_pixels, device=self.dev)
        self.max_cameras = max_cameras
        self.cams_host = (N.CameraDesc * max_cameras)()
        self.cams_dev = torch.empty(max_cameras * ctypes.sizeof(N.CameraDesc), dtype=torch.uint8, device=self.dev)
        self.free_cams = deque(range(max_cameras))
        fd, sd = field.desc(), samp.desc()
        wsb = int(N.lib().nerfxl_render_cameras_workspace_bytes(ctypes.byref(fd), ctypes.byref(sd), self.max_batch))
        if wsb == 0:
            N.check(N.E_INVALID, "nerfxl_render_cameras_workspace_bytes")
        nbuf = self.max_inflight
        self.ws = [torch.empty(wsb, dtype=torch.uint8, device=self.dev) for _ in range(nbuf)]
        self.max_items = 4096
        isz = ctypes.sizeof(N.RayItemDesc)
        self.items_host = [torch.empty(self.max_items * isz, dtype=torch.uint8, pin_memory=True) for _ in range(nbuf)]
        self.items_dev = [torch.empty(self.max_items * isz, dtype=torch.uint8, device=self.dev) for _ in range(nbuf)]
        self.stream = torch.cuda.current_stream(self.dev)

    # -- device state of a request
    def _admit(self, req: Request) -> bool:
        if req.pixels > self.arena.capacity:
            raise ValueError("request %d needs %d pixel slots, the arena holds %d" % (req.rid, req.pixels,
                                                                                      self.arena.capacity))
        if not self.free_cams:
            return False
        s = self.arena.alloc(req.pixels)
        if s < 0:
            return False
        req.slot = s
        req.cam = self.free_cams.popleft()
        self.cams_host[req.cam] = camera_desc(req)
        csz = ctypes.sizeof(N.CameraDesc)
        src = torch.frombuffer(bytearray(bytes(self.cams_host[req.cam])), dtype=torch.uint8)
        self.cams_dev[req.cam * csz:(req.cam + 1) * csz].copy_(src, non_blocking=False)
        req.next_pixel = 0
        return True

    def _release(self, req: Request):
        if self.keep_results:
            s, n = req.slot, req.pixels
            req.result = {"rgb": self.rgb[s:s + n].clone(), "depth": self.depth[s:s + n].clone(),
                          "opacity": self.opacity[s:s + n].clone()}
        self.arena.release(req.slot, req.pixels)
        self.free_cams.append(req.cam)

    def _shares(self, active: deque):
        """Pixels each admitted request renders in the next batch. Fair share
        by water-filling: requests that need less than an equal share of the
        batch get all they need, and the rest is split evenly among the
        others (in arrival order for the remainder), so a large image never
        holds the small requests admitted behind it for more than one batch.
        With one_at_a_time, the first request alone (FIFO). Other policies:
        "fifo" fills the batch in arrival order; "srpt" in order of fewest
        remaining pixels (ties by arrival)."""
        if self.one_at_a_time:
            r = active[0]
            return [(r, min(r.pixels - r.next_pixel, self.max_batch))]
        if self.policy in ("fifo", "srpt"):
            order = list(active)
            if self.policy == "srpt":
                order.sort(key=lambda r: (r.pixels - r.next_pixel, r.arrival_s))
            out, budget = [], self.max_batch
            for r in order[:self.max_items]:
                if budget == 0:
                    break
                t = min(r.pixels - r.next_pixel, budget)
                out.append((r, t))
                budget -= t
            return out
        reqs = list(active)[:self.max_items]
        need = {id(r): r.pixels - r.next_pixel for r in reqs}
        take = {id(r): 0 for r in reqs}
        budget = self.max_batch
        left = sorted(reqs, key=lambda r: need[id(r)])
        while left and budget > 0:
            share = budget // len(left)
            if share == 0:  # fewer pixels than requests: one each, in arrival order
                for r in sorted(left, key=lambda r: r.arrival_s)[:budget]:
                    take[id(r)] += 1
                break
            r = left[0]
            t = min(need[id(r)] - take[id(r)], share)
            if t == need[id(r)] - take[id(r)]:
                take[id(r)] += t
                budget -= t
                left.pop(0)
            else:  # everyone left needs at least a share
                for q in left:
                    take[id(q)] += share
                budget -= share * len(left)
                for q in left[:budget]:  # the remainder, one pixel each
                    take[id(q)] += 1
                budget = 0
        return [(r, take[id(r)]) for r in reqs if take[id(r)] > 0]

    def _launch(self, active: deque, buf: int):
        """One batch: each admitted request's next pixel range (fair share)."""
        items = (N.RayItemDesc * self.max_items).from_buffer(self.items_host[buf].numpy())
        n_items = 0
        n_rays = 0
        finished = []
        for req, take in self._shares(active):
            it = items[n_items]
            it.batch_offset, it.first_pixel, it.out_offset = n_rays, req.next_pixel, req.slot + req.next_pixel
            it.camera, it.count = req.cam, take
            n_items += 1
            n_rays += take
            req.next_pixel += take
            if req.next_pixel == req.pixels:
                finished.append(req)
        for r in finished:
            active.remove(r)
        nbytes = n_items * ctypes.sizeof(N.RayItemDesc)
        self.items_dev[buf][:nbytes].copy_(self.items_host[buf][:nbytes], non_blocking=True)
        fd, sd = self.field.desc(), self.samp.desc()
        st = N.lib().nerfxl_render_cameras(ctypes.byref(fd), ctypes.byref(sd), n_rays, n_items,
                                           N._ptr(self.items_dev[buf]), N._ptr(self.cams_dev), self.max_cameras,
                                           N._ptr(self.rgb), N._ptr(self.depth), N._ptr(self.opacity),
                                           N._ptr(self.ws[buf]), self.ws[buf].numel(), N._stream(self.stream))
        N.check(st, "nerfxl_render_cameras")
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        return ev, finished, n_rays

    def run(self, requests, realtime: bool = True):
        """Serve the requests (sorted by arrival). Returns metrics; fills
        each request's done_s (and result if keep_results)."""
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        active = deque()
        inflight = deque()
        torch.cuda.synchronize()
        t0_ev = torch.cuda.Event(enable_timing=True)
        t0_ev.record(self.stream)
        t0_ev.synchronize()
        t0 = time.perf_counter()
        done = []
        total_rays = 0
        n_batches = 0
        buf = 0
        peak_arena = 0
        while pending or active or inflight:
            now = time.perf_counter() - t0
            # admission by memory (FIFO: a request waits until it fits)
            while pending and (not realtime or pending[0].arrival_s <= now):
                if not self._admit(pending[0]):
                    break
                active.append(pending.popleft())
            peak_arena = max(peak_arena, self.arena.used)
            progressed = False
            if active and len(inflight) < self.max_inflight:
                ev, fin, nr = self._launch(active, buf)
                inflight.append((ev, fin))
                buf = (buf + 1) % len(self.ws)
                total_rays += nr
                n_batches += 1
                progressed = True
            while inflight and (inflight[0][0].query() or (len(inflight) >= self.max_inflight and not active
                                                          and not pending)):
                ev, fin = inflight.popleft()
                ev.synchronize()
                t_dev = t0_ev.elapsed_time(ev) / 1000.0
                for r in fin:
                    r.done_s = t_dev
                    self._release(r)
                    done.append(r)
                progressed = True
            if not progressed:
                if inflight:
                    time.sleep(20e-6)
                elif pending and realtime:
                    time.sleep(max(0.0, min(1e-3, pending[0].arrival_s - (time.perf_counter() - t0))))
        lat = np.array([r.done_s - r.arrival_s for r in done]) * 1000.0
        span = max(r.done_s for r in done) - min(r.arrival_s for r in done) if done else 0.0
        return {"requests": len(done), "rays": int(total_rays), "batches": n_batches,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None,
                "rays_per_s": total_rays / span if span > 0 else None, "span_s": span,
                "peak_arena_pixels": int(peak_arena)}


def requests_from_stream(n: int, rate_hz: float, seed: int, **kw):
    from . import synthetic as sy

    t, H, W, eye, tgt = sy.request_stream(n, rate_hz, seed, **kw)
    return [Request(i, float(t[i]), int(H[i]), int(W[i]), tuple(eye[i]), tuple(tgt[i])) for i in range(n)]
