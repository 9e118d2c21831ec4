"""Throughput benchmark of the one-GPU NeRF-XL hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

The headline step is one training step of the grid8 workload (K=8 regions,
2x2x2 over [-1,1]^3, L=16 F=2 T=2^19 levels 16->2048, 2^18 rays from 64
pinhole cameras, 128 samples per ray) through the C ABI, in the training
configuration: FP16 hash tables, BF16 MLP on the tensor cores, FP32 Adam
masters: sampling, gather, MLP, local render, composite, loss, backward, Adam.
Beside it, under "forms": forward renders (FP32 and FP16 tables + BF16 MLP),
the FP32 plain training step, the city32 MLP precision variants (K=32,
2^20 rays, 256 samples) and the serving loop (Poisson 200 req/s) next to
one-request-at-a-time FP32 rendering. Under torchrun each rank works on its
own batch on its own GPU (rays are independent: weak scaling, no data-path
collective). Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s (render fwd; train fwd+bwd) vs FP32 plain at stated error; p50/p99 serve ms"
WORKLOAD = "grid8"
L2_BYTES = 126 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-rays", type=int, default=1 << 14, help="oracle sample size for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-city", action="store_true", help="skip the city32 precision and serving forms")
    ap.add_argument("--profile-rays", type=int, default=0,
                    help="ncu captures only: use the first N rays of the workload per step (a smaller device "
                         "footprint); 0, the default, keeps the full batch")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-sweep", type=str, default="",
                    help="comma-separated arrival rates (req/s): run only the city32 serving sweep")
    ap.add_argument("--only", type=str, default="",
                    choices=["", "city32_fwd", "city32_train", "grid8_fwd", "grid8_train", "grid8_train_fp32",
                             "grid8_split_train", "grid8_split_train_fp32", "grid8_fwd_fp32",
                             "grid8_split_fwd_fp32"],
                    help="profiler captures: run one form alone and print its own line")
    ap.add_argument("--log2-t", type=int, default=0, help="--only: override the hash table size (log2 entries)")
    ap.add_argument("--group-min-mb", type=float, default=0.0,
                    help="--only: region-table size above which the forward gathers by level groups (0: default)")
    ap.add_argument("--group-mb", type=float, default=0.0, help="--only: table bytes per level group (0: default)")
    ap.add_argument("--window-tiles", type=int, default=0, help="--only: tiles per gather window (0: default)")
    ap.add_argument("--serve-policies", type=str, default="srpt", help="serving sweep: batching policies")
    ap.add_argument("--serve-batches", type=str, default=str(1 << 18), help="serving sweep: max rays per batch")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def rank_rays(w, rank: int):
    """Rays of one rank: rank 0 gets the workload's own rays; rank r > 0 the
    same camera ring rotated by 0.37 r rad about z (same size and
    distribution, different rays: each replica renders its own batch)."""
    from paper_2404_16221_b300 import synthetic as sy

    o, d = sy.workload_rays(w)
    if rank:
        ang = 0.37 * rank
        Rz = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]], np.float32)
        o, d = (o @ Rz.T).astype(np.float32), (d @ Rz.T).astype(np.float32)
    return o, d


def max_over_ranks(values, device=None):
    """Timing reduction across replicas: the slowest rank sets the job time."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def setup_workload(rank: int = 0, sizes=None):
    """The headline workload's field and rays. sizes(w) -> (E, P) gives the
    table entries and MLP parameters per region; by default the library's
    own layout functions (the reference arm passes the oracle's, so that it
    never loads the library)."""
    from paper_2404_16221_b300 import synthetic as sy

    w = sy.workload(WORKLOAD)
    if sizes is None:
        from paper_2404_16221_b300 import native as N

        E, P = N.table_entries(w.level_res, w.log2_T), N.mlp_params(w.mlp_in, w.W)
    else:
        E, P = sizes(w)
    tables, mlp = sy.field_params(w, E, P)
    o, d = rank_rays(w, rank)
    return w, tables, mlp, o, d


def oracle_sizes(w):
    import oracle

    return oracle.table_entries(w.level_res, w.log2_T), oracle.mlp_params(w.mlp_in, w.W)


def cpu_baseline(w, tables, mlp, o, d, n_rays: int, batch: int = 2048):
    """The oracle's training step on the host cores, on a bounded sample: FP64
    loss and gradient (render, Algorithm 1/2 and their adjoint) on n_rays
    seeded rays, in batches, and one FP64 Adam step over every parameter. The
    full step is extrapolated as per-ray time x rays per step + Adam time."""
    import oracle

    from paper_2404_16221_b300 import synthetic as sy

    f = oracle.Field(w.boxes, w.level_res, w.log2_T, w.F, w.mlp_in, w.W, tables.astype(np.float64),
                     mlp.astype(np.float64))
    sel = sy.subset(len(o), min(n_rays, len(o)), 1234)
    tgt = sy.rng(1002, "misc").uniform(0.0, 1.0, (len(sel), 3)).astype(np.float32)
    gt = np.zeros_like(f.tables)
    gm = np.zeros_like(f.mlp)
    t0 = time.perf_counter()
    for b in range(0, len(sel), batch):
        idx = sel[b:b + batch]
        _, bt, bm = oracle.loss_grad(f, w.S, o[idx], d[idx], tgt[b:b + batch], 0.01)
        gt += bt
        gm += bm
    t1 = time.perf_counter()
    for p_, g_ in ((f.tables.reshape(-1), gt.reshape(-1)), (f.mlp.reshape(-1), gm.reshape(-1))):
        oracle.adam(np.ascontiguousarray(p_), np.zeros_like(p_), np.zeros_like(p_), np.ascontiguousarray(g_), 1, 1e-2,
                    0.9, 0.99, 1e-15)
    t2 = time.perf_counter()
    step_s = (t1 - t0) / len(sel) * w.n_rays + (t2 - t1)
    n_params = f.tables.size + f.mlp.size
    return {"value": w.n_rays / step_s, "unit": "rays/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d seeded rays of the %s training step: FP64 loss + gradient (render, Algorithm 1/2 and their "
                      "adjoint) %.1f s, one FP64 Adam step over all %d parameters %.1f s; a full step of %d rays "
                      "extrapolated as per-ray time x rays + Adam time" % (len(sel), w.name, t1 - t0, n_params,
                                                                           t2 - t1, w.n_rays)}


def run_reference(args, rank, world):
    """The oracle's training step on the host cores. Each step is a bounded
    sample of the headline workload (cpu_rays / 8 of its rays, at least 256,
    plus one FP64 Adam step over every parameter), timed as it runs; rays/s
    is the sample's rays over the measured time of its ray part."""
    if rank != 0:
        return
    w, tables, mlp, o, d = setup_workload(sizes=oracle_sizes)
    n = max(256, args.cpu_rays // 8)
    for _ in range(max(0, args.warmup)):
        cpu_baseline(w, tables, mlp, o, d, 256)
    vals, secs = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(w, tables, mlp, o, d, n)
        secs.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grid8 training step (loss L2 + 0.01 distortion, gradient, Adam): K=8 2x2x2 over "
                                   "[-1,1]^3, L=16 F=2 T=2^19 (16->2048), 2^18 rays from 64 cameras, S=128. Each "
                                   "timed step is a bounded sample: the FP64 loss and gradient of %d seeded rays "
                                   "and one FP64 Adam step over all parameters; ms_per_step is that sample's "
                                   "measured time, value = rays/s of the full 2^18-ray step extrapolated from "
                                   "the sample's per-ray time plus the Adam time" % n,
                       "rays_per_step": n},
            "cpu_baseline": {"value": v, "unit": "rays/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(step, steps, flush, stream, prof=True):
    """Per-step CUDA events around each step (L2 flushed before each step,
    outside the events); the library's profile events bracket the dominant
    kernel of each step. Returns (step_ms, kernel_ms) lists."""
    import torch

    from paper_2404_16221_b300 import native as N

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for pair in kev:  # torch creates the CUDA event on first record
        for e in pair:
            e.record(stream)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        if prof:
            N.check(N.lib().nerfxl_set_profile_events(C_void(kev[i][0].cuda_event), C_void(kev[i][1].cuda_event)),
                    "profile events")
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    N.lib().nerfxl_set_profile_events(None, None)
    return [a.elapsed_time(b) for a, b in ev], ([a.elapsed_time(b) for a, b in kev] if prof else [])


# Table-gradient reduction requests (32-byte sectors per instruction) per
# sample of the headline backward's scatter, from the same ncu capture as
# BWD_TC_DRAM (l1tex__t_sectors_pipe_lsu_mem_global_op_red.sum / samples). One
# lane per sample and level, with a 16-byte vector on the aligned entry pair
# holding the first corner of each x-pair plus an 8-byte one when the second
# corner is not in that pair, takes 16 levels x 4 x-pairs x 1.5 = 96; runs of
# samples in the same cell share one set (76), and two lanes per run, one per
# x-half, send both halves of an x-pair in one instruction, one request when
# they share a sector (three x-pairs in four): 63.5.
BWD_TC_RED = {"sectors": 1860324857, "samples": 29292644}
RED_PROBE_BYTES = 48 << 20  # about one grid8 region's FP32 gradient table (49 MB)
LD_PROBE_BYTES = 24 << 20  # about one grid8 region's FP16 table (24 MB)
# Table-read sectors per sample of the mixed forward's gather (FP16 tables),
# from one ncu capture of the plain grid8 forward at full size
# (l1tex__t_sectors_pipe_lsu_mem_global_op_ld.sum / samples), valid while the
# forward's sources are unchanged.
FWD_TC_LD = {"sectors": 2144803190, "samples": 29292644, "sources_sha16": "15c0a93433dfff2f"}
FWD_TC_SOURCES = ("nerfxl_fwd_tc.cu", "nerfxl_field.cuh", "nerfxl_tc.cuh", "nerfxl_half.cuh", "nerfxl_device.cuh")


def _probe_rate(entry: str, nbytes: int, iters: int, stream, reps: int = 5) -> float:
    import torch

    from paper_2404_16221_b300 import native as N

    buf = torch.zeros(nbytes // 4, dtype=torch.float32, device="cuda")
    ops = C_int64()
    fn = getattr(N.lib(), entry)
    N.check(fn(N._ptr(buf), nbytes, iters, ctypes_byref(ops), N._stream(stream)), entry)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        N.check(fn(N._ptr(buf), nbytes, iters, ctypes_byref(ops), N._stream(stream)), entry)
    b.record(stream)
    torch.cuda.synchronize()
    return reps * ops.value / (a.elapsed_time(b) / 1000.0)


def reduction_ceiling(stream) -> float:
    """Measured ceiling of scattered 16-byte FP32 reductions (per second) on
    this GPU: nerfxl_probe_reduction_rate into a 48 MB buffer, CUDA events."""
    return _probe_rate("nerfxl_probe_reduction_rate", RED_PROBE_BYTES, 256, stream)


def load_ceiling(stream) -> float:
    """Measured ceiling of scattered 8-byte loads (per second) on this GPU:
    nerfxl_probe_load_rate over a 24 MB buffer (one grid8 region's FP16
    table), CUDA events."""
    return _probe_rate("nerfxl_probe_load_rate", LD_PROBE_BYTES, 64, stream)


def ctypes_byref(x):
    import ctypes

    return ctypes.byref(x)


def fp32_alu_peak_tflops(sm_count: int = 148, mhz: float = 2032.0) -> float:
    """CUDA-core FP32 peak: SMs x 128 FMA lanes x 2 FLOP x max SM clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


# Algorithmic FLOPs of the MLP per sample (32-64-64-4, multiply-add = 2 FLOP):
# forward 2 (32*64 + 64*64 + 64*4) = 12,800; the backward recomputes the
# forward, then dX (12,800) and dW (12,800): 38,400 per sample.
MLP_FWD_FLOP = 2 * (32 * 64 + 64 * 64 + 64 * 4)
BWD_FLOP_PER_SAMPLE = 3 * MLP_FWD_FLOP
# split representation: density 32-64-16 + colour 32-64-64-3 (Wc3 counted as stored, 64 x 4)
SPLIT_FWD_FLOP = 2 * (32 * 64 + 64 * 16) + 2 * (32 * 64 + 64 * 64 + 64 * 4)
SPLIT_BWD_FLOP = 3 * SPLIT_FWD_FLOP
# Algorithmic bytes of the tensor-core backward field kernel per sample (L=16
# levels, F=2, 8 corners): its per-tile records (16-bit features 32 x 2 B, the
# 12 geometry floats of a record row 48 B, chunk adjoints 32 B per 32 samples)
# and the read-modify-write of the FP32 gradient entries the sample touches
# (2 x 8 x 2 x 4 B x 16 = 2048 B).
TRAIN_BYTES_PER_SAMPLE_F16 = 32 * 2 + 12 * 4 + 1 + 2 * 8 * 2 * 4 * 16
# DRAM bytes (read + write) of one k_field_bwd_tc launch on this workload from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), with a hash
# of the kernel's sources at the time of the capture: the figure is reported
# only while the sources are unchanged (None: not captured for this build).
BWD_TC_DRAM = {"bytes": 3.991044e9 + 0.339015e9, "sources_sha16": "38b3437278130f0d"}
BWD_TC_SOURCES = ("nerfxl_bwd_tc.cu", "nerfxl_scatter.cuh", "nerfxl_tc.cuh", "nerfxl_field.cuh", "nerfxl_half.cuh",
                  "nerfxl_device.cuh")


def sources_sha16(names=BWD_TC_SOURCES):
    import hashlib

    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2404_16221_b300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def bwd_tc_traffic():
    if BWD_TC_DRAM["bytes"] is None or BWD_TC_DRAM["sources_sha16"] != sources_sha16():
        return None
    return BWD_TC_DRAM["bytes"]


def fwd_tc_sectors_per_sample():
    """Measured table-read sectors per sample of the mixed forward's gather
    (None once the kernel's sources differ from the captured build)."""
    if FWD_TC_LD["sources_sha16"] != sources_sha16(FWD_TC_SOURCES):
        return None
    return FWD_TC_LD["sectors"] / FWD_TC_LD["samples"]


def bwd_tc_reductions_per_sample():
    """Measured reduction requests per sample of the headline backward's scatter
    (None once the kernel's sources differ from the captured build)."""
    if BWD_TC_DRAM["sources_sha16"] != sources_sha16():
        return None
    return BWD_TC_RED["sectors"] / BWD_TC_RED["samples"]


def single_form(args, dev):
    """One form alone, for profiler captures (--only): its steps timed with
    CUDA events and one JSON line printed. city32_fwd: the street/city
    forward with FP16 tables and a BF16 MLP; grid8_fwd / grid8_train: the
    mixed grid8 forward and training step; grid8_split_train(_fp32): the
    split representation's mixed (FP32) training step; grid8_fwd_fp32 /
    grid8_split_fwd_fp32: the FP32 forward of either representation.
    --profile-rays keeps the first N rays (a smaller device footprint for
    captures)."""
    import torch

    from paper_2404_16221_b300 import api, native as N, synthetic as sy

    name = args.only
    if args.group_min_mb > 0 or args.group_mb > 0 or args.window_tiles > 0:
        N.check(N.lib().nerfxl_set_gather_groups(int(args.group_min_mb * (1 << 20)), int(args.group_mb * (1 << 20)),
                                                 args.window_tiles, 0), "gather groups")
    w = sy.workload("city32" if name.startswith("city32") else "grid8")
    if args.log2_t:
        w.log2_T = args.log2_t
    E = N.table_entries(w.level_res, w.log2_T)
    fp32 = name.endswith("_fp32")
    forward = "_fwd" in name
    if name.startswith("grid8_split"):
        n_split = api.split_mlp_params(w.K, w.mlp_in, w.W)
        t, _ = sy.field_params_device(w, E, N.mlp_params(w.mlp_in, w.W), dev)
        g = torch.Generator(device=dev)
        g.manual_seed(int(w.seed) * 7919 + 11)
        m = torch.randn(n_split, generator=g, device=dev) * 0.1
        field = api.PartitionedField(w.boxes, w.level_res, w.log2_T, t if fp32 else t.to(torch.float16),
                                     m if fp32 else m.to(torch.bfloat16), device=dev, arch=N.ARCH_SPLIT)
    elif fp32:
        t, m = sy.field_params_device(w, E, N.mlp_params(w.mlp_in, w.W), dev)
        field = api.PartitionedField(w.boxes, w.level_res, w.log2_T, t, m, device=dev)
    else:
        t, m = sy.field_params_device(w, E, N.mlp_params(w.mlp_in, w.W), dev)
        field = api.PartitionedField(w.boxes, w.level_res, w.log2_T, t.to(torch.float16), m.to(torch.bfloat16),
                                     device=dev)
    if forward:
        del t, m  # a forward holds only the field it reads
        torch.cuda.empty_cache()
    o, d = sy.workload_rays(w)
    if args.profile_rays > 0:
        o, d = o[:args.profile_rays].copy(), d[:args.profile_rays].copy()
    o, d = torch.from_numpy(o).to(dev), torch.from_numpy(d).to(dev)
    samp = api.Sampling(w.S, w.max_segments)
    if forward:
        ws = api.alloc_workspace(field, samp, len(o))
        step = lambda: api.render_fwd(field, samp, o, d, workspace=ws)
    else:
        tgt = torch.rand(len(o), 3, generator=torch.Generator().manual_seed(1002)).to(dev)
        masters = {} if fp32 else {"master_tables": t, "master_mlp": m}
        tr = api.Trainer(field, samp, **masters,
                         workspace_cap=(4 << 30) if name == "city32_train" else None)
        step = lambda: tr.step(o, d, tgt)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    step_ms, kern_ms = time_steps(step, args.steps, flush, stream)
    print(json.dumps({"only": name, "rays": len(o), "ms_per_step": statistics.mean(step_ms),
                      "rays_per_s": len(o) / (statistics.mean(step_ms) / 1000.0),
                      "dominant_kernel_ms": statistics.mean(kern_ms)}), flush=True)


def serve_sweep(args, dev, rates):
    """p50/p99 latency and served rays/s of the city32 serving loop (FP16
    tables + BF16 MLP) at several Poisson arrival rates, args.serve_requests
    requests each; prints one JSON line."""
    import torch

    from paper_2404_16221_b300 import api, native as N, serve, synthetic as sy

    ws_ = sy.workload("serve32")
    E = N.table_entries(ws_.level_res, ws_.log2_T)
    t, m = sy.field_params_device(ws_, E, N.mlp_params(ws_.mlp_in, ws_.W), dev)
    field = api.PartitionedField(ws_.boxes, ws_.level_res, ws_.log2_T, t.to(torch.float16), m.to(torch.bfloat16),
                                 device=dev)
    del t, m
    samp = api.Sampling(ws_.S, ws_.max_segments)
    serve.ServeEngine(field, samp).run(serve.requests_from_stream(4, 100.0, ws_.seed + 17), realtime=False)
    rows = []
    for policy, batch in [(p_, int(b_)) for p_ in args.serve_policies.split(",")
                          for b_ in args.serve_batches.split(",")]:
        for rate in rates:
            reqs = serve.requests_from_stream(args.serve_requests, rate, ws_.seed)
            px = sum(r.pixels for r in reqs)
            m_ = serve.ServeEngine(field, samp, max_batch_rays=batch, arena_pixels=1 << 26, policy=policy).run(reqs)
            m_.update({"rate_req_s": rate, "offered_rays_per_s": px / max(reqs[-1].arrival_s, 1e-9),
                       "policy": policy, "max_batch_rays": batch,
                       "largest_request_pixels": max(r.pixels for r in reqs)})
            rows.append(m_)
    print(json.dumps({"serve_sweep": rows, "workload": "serve32: K=32 city field, FP16 tables + BF16 MLP, "
                      "log-uniform 64x64..1920x1080 requests, Poisson arrivals, %d requests per rate"
                      % args.serve_requests}), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2404_16221_b300 import api, build, native as N, serve, synthetic as sy

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    if args.only:
        single_form(args, dev)
        return
    if args.serve_sweep:
        serve_sweep(args, dev, [float(r) for r in args.serve_sweep.split(",")])
        return
    w, tables, mlp, o, d = setup_workload(rank)
    if args.profile_rays > 0:
        o, d = o[:args.profile_rays].copy(), d[:args.profile_rays].copy()
    samp = api.Sampling(w.S, w.max_segments)
    R = len(o)
    o_dev = torch.from_numpy(o).to(dev)
    d_dev = torch.from_numpy(d).to(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    steps, warm = args.steps, max(3, args.warmup)

    def mk_field(wl, t, m, tab_dtype, mlp_dtype):
        return api.PartitionedField(wl.boxes, wl.level_res, wl.log2_T, torch.as_tensor(t).to(dev, tab_dtype),
                                    torch.as_tensor(m).to(dev, mlp_dtype), device=dev)

    def out_bufs(n):
        return {"rgb": torch.empty(n, 3, device=dev), "depth": torch.empty(n, device=dev),
                "opacity": torch.empty(n, device=dev), "dist": torch.empty(n, device=dev)}

    def fwd_form(wl, field, sp, ro, rd, kernel, bytes_per_sample):
        n = ro.shape[0]
        ws = api.alloc_workspace(field, sp, n)
        out = out_bufs(n)
        step = lambda: api.render_fwd(field, sp, ro, rd, workspace=ws, out=out)
        for _ in range(warm):
            step()
        api.check(ws)
        ns, nc = C_int64(), C_int64()
        N.check(N.lib().nerfxl_workspace_stats(N._ptr(ws), ws.numel(), ns, nc, N._stream(None)), "stats")
        with Clocks(local) as clk:
            step_ms, kern_ms = time_steps(step, steps, flush, stream)
        return {"rays": n, "step_ms": step_ms, "kern_ms": kern_ms, "samples": ns.value, "chunks": nc.value,
                "clocks": clk.summary(), "kernel": kernel, "bytes_per_sample": bytes_per_sample,
                "field": field, "ws": ws, "out": out, "step": step}

    forms = {}
    # ---- grid8 (K=8): forward forms
    f32 = mk_field(w, tables, mlp, torch.float32, torch.float32)
    forms["grid8_fwd_fp32"] = fwd_form(w, f32, samp, o_dev, d_dev, "k_field_fwd_f32", 8 * w.F * 4 * w.L)
    fmix = mk_field(w, tables, mlp, torch.float16, torch.bfloat16)
    forms["grid8_fwd_f16tab_bf16mlp"] = fwd_form(w, fmix, samp, o_dev, d_dev, "k_field_fwd_tc", 8 * w.F * 2 * w.L)
    # sample-level composition (the naive scheme of Sec. 4.2) vs the segment-level one, FP32 forward:
    # bytes between the field kernel and the composite (written once, read once) and rays/s
    samp_s = dataclasses.replace(samp, flags=api.SAMPLE_COMPOSITE)
    fs = fwd_form(w, f32, samp_s, o_dev, d_dev, "k_field_fwd_f32", 8 * w.F * 4 * w.L)
    seg = forms["grid8_fwd_fp32"]
    seg_bytes = 2 * 32 * seg["chunks"] / R          # one 32-byte partial per 32-sample chunk
    smp_bytes = 2 * 24 * 32 * fs["chunks"] / R      # 24 bytes per sample slot
    forms["grid8_composition"] = {
        "composition": {
            "segment_level": {"rays_per_s": R / (statistics.mean(seg["step_ms"]) / 1000.0),
                              "bytes_per_ray": seg_bytes},
            "sample_level": {"rays_per_s": R / (statistics.mean(fs["step_ms"]) / 1000.0),
                             "bytes_per_ray": smp_bytes},
            "bytes_ratio": smp_bytes / seg_bytes},
        "note": "FP32 field; bytes written by the field kernel and read by the composite, per ray "
                "(the one-GPU analogue of the paper's per-sample vs per-tile exchange)"}
    for k in ("field", "ws", "out", "step"):
        fs.pop(k)
    for k in ("grid8_fwd_fp32", "grid8_fwd_f16tab_bf16mlp"):
        forms[k].pop("field"), forms[k].pop("ws"), forms[k].pop("out"), forms[k].pop("step")
    del fmix
    # ---- grid8 training steps: FP16 tables + BF16 MLP + FP32 Adam (the headline, configs c3) and FP32 plain
    tgt = torch.rand(R, 3, generator=torch.Generator().manual_seed(1002)).to(dev)
    mfield = mk_field(w, tables, mlp, torch.float16, torch.bfloat16)
    mtrainer = api.Trainer(mfield, samp, lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=torch.from_numpy(tables),
                           master_mlp=torch.from_numpy(mlp))
    mstep = lambda: mtrainer.step(o_dev, d_dev, tgt)
    for _ in range(warm):
        mstep()
    torch.cuda.synchronize()
    launches0 = int(N.lib().nerfxl_launch_count())
    with Clocks(local) as clk:
        step_ms, kern_ms = time_steps(mstep, steps, flush, stream)
    head_launches = int(N.lib().nerfxl_launch_count()) - launches0
    forms["grid8_train_f16tab_bf16mlp"] = {"rays": R, "step_ms": step_ms, "kern_ms": kern_ms,
                                           "clocks": clk.summary(), "kernel": "k_field_bwd_tc",
                                           "samples": forms["grid8_fwd_fp32"]["samples"],
                                           "bytes_per_sample": TRAIN_BYTES_PER_SAMPLE_F16}
    # end to end through host buffers: rays and targets in, the loss out
    def pinned(a):
        # page-locked buffer allocated pinned (torch.empty(pin_memory=True)):
        # its host-to-device copies ran at 53 GB/s here, those of a tensor
        # pinned after the fact (.pin_memory()) at 13 GB/s
        h = torch.empty(a.shape, dtype=a.dtype, pin_memory=True)
        h.copy_(a)
        return h

    o_h, d_h = pinned(torch.from_numpy(o)), pinned(torch.from_numpy(d))
    t_h = pinned(tgt.cpu())
    loss_h = torch.empty(3, pin_memory=True)

    def e2e_step():
        o_dev.copy_(o_h, non_blocking=True)
        d_dev.copy_(d_h, non_blocking=True)
        tgt.copy_(t_h, non_blocking=True)
        loss = mtrainer.step(o_dev, d_dev, tgt)
        loss_h.copy_(loss, non_blocking=True)

    for _ in range(warm):
        e2e_step()
    e2e_ms, _ = time_steps(e2e_step, steps, flush, stream, prof=False)
    del mtrainer, mfield
    trainer = api.Trainer(f32, samp, lr=1e-2, eps=1e-15, lambda_dist=0.01)
    tstep = lambda: trainer.step(o_dev, d_dev, tgt)
    for _ in range(warm):
        tstep()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        step_ms, kern_ms = time_steps(tstep, steps, flush, stream)
    forms["grid8_train_fp32"] = {"rays": R, "step_ms": step_ms, "kern_ms": kern_ms, "clocks": clk.summary(),
                                 "kernel": "k_field_bwd_f32", "samples": forms["grid8_fwd_fp32"]["samples"],
                                 "flop_per_sample": BWD_FLOP_PER_SAMPLE}
    del trainer
    # ---- occupancy-grid skipping (the spatial-skipping structure of Sec. 5.1) on the grid8 shapes: the
    #      grid a field trained on the sparse blob scene would hold (11% of cells), throughput with and
    #      without it, and the cost of one full refresh of a 128^3-per-region grid
    G_occ = 64
    occ_bits = sy.blob_occupancy(w.boxes, sy.sparse_blobs(w.seed), G_occ, 0.4)
    occ = {"grid": "%d^3 cells per region, %.1f%% occupied" % (G_occ, 100.0 * float(
        np.unpackbits(occ_bits.view(np.uint8)).sum()) / (w.K * G_occ ** 3))}
    fmix = mk_field(w, tables, mlp, torch.float16, torch.bfloat16)
    for label, bits in (("no_grid", None), ("grid", occ_bits)):
        fmix.set_occupancy(bits, G_occ)
        r = fwd_form(w, fmix, samp, o_dev, d_dev, "k_field_fwd_tc", 8 * w.F * 2 * w.L)
        km = statistics.mean(r["kern_ms"])
        occ["fwd_f16tab_bf16mlp_" + label] = {
            "rays_per_s": R / (statistics.mean(r["step_ms"]) / 1000.0), "samples_per_ray": r["samples"] / R,
            "field_kernel_ms": km, "chunk_fill": r["samples"] / (32.0 * max(r["chunks"], 1)),
            "field_gbs_algorithmic": r["samples"] * 8 * w.F * 2 * w.L / (km / 1000.0) / 1e9}
        del r
        otrainer = api.Trainer(fmix, samp, lr=1e-2, eps=1e-15, lambda_dist=0.01,
                               master_tables=torch.from_numpy(tables), master_mlp=torch.from_numpy(mlp))
        ostep = lambda: otrainer.step(o_dev, d_dev, tgt)
        for _ in range(warm):
            ostep()
        o_ms, _ = time_steps(ostep, steps, flush, stream, prof=False)
        occ["train_f16tab_bf16mlp_" + label] = {"rays_per_s": R / (statistics.mean(o_ms) / 1000.0)}
        del otrainer
    del fmix
    grid = api.OccupancyGrid(w.K, 128, decay=0.95, threshold=0.4)
    grid.update(f32)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(3):
        grid.update(f32)
    ev1.record(stream)
    torch.cuda.synchronize()
    occ["refresh_ms_128cubed_per_region"] = ev0.elapsed_time(ev1) / 3
    forms["grid8_occupancy"] = {
        "occupancy": occ,
        "note": "FP16 tables + BF16 MLP, random-init grid8 field; the bits are those of the sparse blob scene's "
                "density > 0.4 at cell centres (a trained field's grid stand-in); the refresh evaluates the FP32 "
                "field at one Philox point per cell"}
    del grid, f32
    torch.cuda.empty_cache()
    # ---- the split representation (App. A.1): per-region density MLP + one shared view-dependent colour
    #      MLP, FP32 forward and training step on the grid8 shapes, next to the fused FP32 forms above
    n_split = api.split_mlp_params(w.K, w.mlp_in, w.W)
    gsm = torch.Generator(device=dev)
    gsm.manual_seed(int(w.seed) * 7919 + 11)
    m_split = torch.randn(n_split, generator=gsm, device=dev) * 0.1
    fsplit = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.as_tensor(tables).to(dev), m_split, device=dev,
                                  arch=N.ARCH_SPLIT)
    r = fwd_form(w, fsplit, samp, o_dev, d_dev, "k_field_fwd_persample_f32", 8 * w.F * 4 * w.L)
    km = statistics.mean(r["kern_ms"])
    split = {"fwd_fp32": {"rays_per_s": R / (statistics.mean(r["step_ms"]) / 1000.0), "kernel_ms": km,
                          "mlp_tflops_algorithmic": r["samples"] * SPLIT_FWD_FLOP / (km / 1000.0) / 1e12,
                          "fp32_alu_peak_tflops": fp32_alu_peak_tflops()}}
    r_samples = r["samples"]
    del r
    fsplit16 = api.PartitionedField(w.boxes, w.level_res, w.log2_T, torch.as_tensor(tables).to(dev, torch.float16),
                                    m_split.to(torch.bfloat16), device=dev, arch=N.ARCH_SPLIT)
    r = fwd_form(w, fsplit16, samp, o_dev, d_dev, "k_field_fwd_tc", 8 * w.F * 2 * w.L)
    km = statistics.mean(r["kern_ms"])
    split["fwd_f16tab_bf16mlp"] = {"rays_per_s": R / (statistics.mean(r["step_ms"]) / 1000.0), "kernel_ms": km,
                                   "mlp_tflops_algorithmic": r["samples"] * SPLIT_FWD_FLOP / (km / 1000.0) / 1e12}
    del r
    # mixed training of the split form: tensor-core forward and backward, FP32 Adam masters
    mtr = api.Trainer(fsplit16, samp, lr=1e-2, eps=1e-15, lambda_dist=0.01,
                      master_tables=torch.as_tensor(tables), master_mlp=m_split.float().cpu())
    mst = lambda: mtr.step(o_dev, d_dev, tgt)
    for _ in range(warm):
        mst()
    torch.cuda.synchronize()
    m_ms, m_kern = time_steps(mst, steps, flush, stream)
    split["train_f16tab_bf16mlp"] = {"rays_per_s": R / (statistics.mean(m_ms) / 1000.0),
                                     "kernel_ms": statistics.mean(m_kern), "kernel": "k_field_bwd_split_tc",
                                     "mlp_tflops_algorithmic": r_samples * SPLIT_BWD_FLOP
                                     / (statistics.mean(m_kern) / 1000.0) / 1e12}
    del mtr, fsplit16
    strainer = api.Trainer(fsplit, samp, lr=1e-2, eps=1e-15, lambda_dist=0.01)
    sstep = lambda: strainer.step(o_dev, d_dev, tgt)
    for _ in range(warm):
        sstep()
    torch.cuda.synchronize()
    s_ms, s_kern = time_steps(sstep, steps, flush, stream)
    split["train_fp32"] = {"rays_per_s": R / (statistics.mean(s_ms) / 1000.0), "kernel_ms": statistics.mean(s_kern),
                           "kernel": "k_field_bwd_split_f32",
                           "mlp_tflops_algorithmic": r_samples * SPLIT_BWD_FLOP / (statistics.mean(s_kern) / 1000.0)
                           / 1e12}
    forms["grid8_split"] = {
        "split": split,
        "note": "FP32 tables and MLPs; density MLP 32-64-16 per region, colour MLP 32-64-64-3 shared, on "
                "[density features, degree-0..3 SH of the view direction]; compare grid8_fwd_fp32 / grid8_train_fp32"}
    del strainer, fsplit, m_split
    torch.cuda.empty_cache()
    # ---- city32 (K=32, 8x4x1 slabs, 2^20 rays, S=256): MLP precision variants
    if not args.skip_city:
        wc = sy.workload("city32")
        Ec = N.table_entries(wc.level_res, wc.log2_T)
        tc_, mc_ = sy.field_params_device(wc, Ec, N.mlp_params(wc.mlp_in, wc.W), dev)
        oc, dc = sy.workload_rays(wc)
        oc_d, dc_d = torch.from_numpy(oc).to(dev), torch.from_numpy(dc).to(dev)
        sc = api.Sampling(wc.S, wc.max_segments)
        for name, td, md, kern in (("city32_fwd_fp32", torch.float32, torch.float32, "k_field_fwd_persample_f32"),
                                   ("city32_fwd_bf16mlp", torch.float32, torch.bfloat16, "k_field_fwd_tc"),
                                   ("city32_fwd_fp16mlp", torch.float32, torch.float16, "k_field_fwd_tc"),
                                   ("city32_fwd_f16tab_bf16mlp", torch.float16, torch.bfloat16, "k_field_fwd_tc")):
            fc = mk_field(wc, tc_, mc_, td, md)
            forms[name] = fwd_form(wc, fc, sc, oc_d, dc_d, kern, 8 * wc.F * (4 if td == torch.float32 else 2) * wc.L)
            for k in ("field", "ws", "out", "step"):
                forms[name].pop(k)
            del fc
            torch.cuda.empty_cache()
        # ---- city32 training step (FP16 tables, BF16 MLP, records, FP32 Adam) under a 4 GB workspace cap:
        #      the step runs in ray sub-batches (its one-pass workspace is several times larger)
        tgt_c = torch.rand(len(oc), 3, generator=torch.Generator().manual_seed(1003)).to(dev)
        fcm = mk_field(wc, tc_, mc_, torch.float16, torch.bfloat16)
        cap = 4 << 30
        ctr = api.Trainer(fcm, sc, lr=1e-2, eps=1e-15, lambda_dist=0.01, master_tables=tc_, master_mlp=mc_,
                          workspace_cap=cap)
        cstep = lambda: ctr.step(oc_d, dc_d, tgt_c)
        for _ in range(warm):
            cstep()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            c_ms, _ = time_steps(cstep, max(2, steps // 4), flush, stream, prof=False)
        fdc, sdc = fcm.desc(), ctr.samp.desc()
        forms["city32_train_f16tab_bf16mlp"] = {
            "train_capped": {
                "rays_per_s": len(oc) / (statistics.mean(c_ms) / 1000.0), "ms_per_step": statistics.mean(c_ms),
                "clocks": clk.summary(), "cap_bytes": cap, "used_bytes": int(ctr._ws.numel()),
                "one_pass_bytes": int(N.lib().nerfxl_step_workspace_bytes(api.C_ref(fdc), api.C_ref(sdc), len(oc))),
                "sub_batch_rays": ctr.sub_batch(len(oc))},
            "note": "K=32 city field, 2^20 rays, S=256, FP16 tables + BF16 MLP + FP32 Adam masters, uniform random "
                    "target; the step's workspace capped at 4 GB, so it runs in ray sub-batches"}
        del ctr, fcm
        torch.cuda.empty_cache()
        # ---- spatial partitioning (Sec. 4.4) on an uneven trajectory: 32 regions from the CDF splits of
        #      training-ray samples vs the uniform 8x4x1 slabs, held-out rays of the same trajectory
        root = sy.scene_root(wc)
        o_tr, d_tr = sy.one_sided_rays(wc, 1 << 14, 61)
        cdf_boxes, _ = api.partition_boxes(sy.ray_sample_points(o_tr, d_tr, root, 64, 62), root, 5)
        o1, d1 = sy.one_sided_rays(wc, 1 << 18, 63)
        o1_d, d1_d = torch.from_numpy(o1).to(dev), torch.from_numpy(d1).to(dev)
        part = {}
        for label, boxes in (("uniform_grid", wc.boxes), ("cdf_partition", cdf_boxes)):
            fc = api.PartitionedField(boxes, wc.level_res, wc.log2_T, tc_.to(torch.float16), mc_.to(torch.bfloat16),
                                      device=dev)
            sp1 = api.Sampling(wc.S, 32)
            r = fwd_form(wc, fc, sp1, o1_d, d1_d, "k_field_fwd_tc", 8 * wc.F * 2 * wc.L)
            chunks = api.region_chunks(r["ws"], wc.K)
            part[label] = {"rays_per_s": r["rays"] / (statistics.mean(r["step_ms"]) / 1000.0),
                           "chunks_max_over_min": float(chunks.max() / max(int(chunks.min()), 1)),
                           "chunks_max_over_mean": float(chunks.max() / chunks.mean())}
            del fc, r
            torch.cuda.empty_cache()
        forms["city32_partition_balance"] = {
            "partition": part,
            "note": "FP16 tables + BF16 MLP; 2^18 held-out rays of a trajectory covering x < -1 only; 32 boxes "
                    "from recursive CDF = 0.5 splits of samples of 2^14 training rays of the same trajectory"}
        # ---- serving (K=32 field resident, FP16 tables + BF16 MLP), Poisson arrivals at 200 req/s
        ws_ = sy.workload("serve32")
        reqs = serve.requests_from_stream(args.serve_requests, 200.0, ws_.seed)
        sfield = mk_field(ws_, tc_, mc_, torch.float16, torch.bfloat16)
        ss = api.Sampling(ws_.S, ws_.max_segments)
        warm_reqs = serve.requests_from_stream(4, 200.0, ws_.seed + 17)
        serve.ServeEngine(sfield, ss, max_batch_rays=1 << 20, arena_pixels=1 << 26).run(warm_reqs, realtime=False)
        with Clocks(local) as clk:
            m = serve.ServeEngine(sfield, ss, max_batch_rays=1 << 18, arena_pixels=1 << 26).run(reqs)
        m["clocks"] = clk.summary()
        forms["serve32_poisson200"] = {"serve": m, "requests": len(reqs),
                                       "note": "FP16 tables + BF16 MLP, batches of up to 2^18 rays (fewest remaining "
                                               "pixels first), 2 in flight, arena 2^26 pixel slots; latency = "
                                               "arrival to device completion"}
        del sfield
        torch.cuda.empty_cache()
        ffield = mk_field(ws_, tc_, mc_, torch.float32, torch.float32)
        reqs1 = serve.requests_from_stream(args.serve_requests, 200.0, ws_.seed)
        serve.ServeEngine(ffield, ss, max_batch_rays=1 << 20, one_at_a_time=True).run(warm_reqs[:2], realtime=False)
        m1 = serve.ServeEngine(ffield, ss, max_batch_rays=1 << 20, arena_pixels=1 << 26, one_at_a_time=True).run(reqs1)
        forms["serve32_one_at_a_time_fp32"] = {"serve": m1, "requests": len(reqs1),
                                               "note": "FP32 field, one request per launch, FIFO"}
        del ffield, tc_, mc_
        torch.cuda.empty_cache()

    head = forms["grid8_train_f16tab_bf16mlp"]
    red_ceiling = reduction_ceiling(torch.cuda.current_stream())
    ld_ceiling = load_ceiling(torch.cuda.current_stream())
    t_step = sum(head["step_ms"]) / 1000.0
    t_e2e = sum(e2e_ms) / 1000.0
    if world > 1:
        dist.barrier()
        t_step, t_e2e = max_over_ranks([t_step, t_e2e], dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    hbm, bf16, src = peaks()
    alu_peak = fp32_alu_peak_tflops()
    # fractions of the peaks for the occupancy and split forms' field kernels
    for v in forms.get("grid8_occupancy", {}).get("occupancy", {}).values():
        if isinstance(v, dict) and "field_gbs_algorithmic" in v:
            v["field_frac_of_hbm"] = v["field_gbs_algorithmic"] / hbm
    for name, v in forms.get("grid8_split", {}).get("split", {}).items():
        if "mlp_tflops_algorithmic" in v:
            if name.endswith("fp32"):
                v["frac_of_fp32_alu"] = v["mlp_tflops_algorithmic"] / alu_peak
            else:
                v["frac_of_bf16_tensor"] = v["mlp_tflops_algorithmic"] / bf16

    def summary(f):
        if any(k in f for k in ("serve", "partition", "composition", "occupancy", "split", "train_capped")):
            return {k: v for k, v in f.items()}
        ms = statistics.mean(f["step_ms"])
        r = {"rays_per_s": f["rays"] / (ms / 1000.0), "ms_per_step": ms}
        if f.get("kern_ms"):
            km = statistics.mean(f["kern_ms"])
            r["kernel"] = f["kernel"]
            r["kernel_ms"] = km
            if "bytes_per_sample" in f:
                r["gbs_algorithmic"] = f["samples"] * f["bytes_per_sample"] / (km / 1000.0) / 1e9
                r["frac_of_hbm"] = r["gbs_algorithmic"] / hbm
            if "flop_per_sample" in f:
                r["mlp_tflops_algorithmic"] = f["samples"] * f["flop_per_sample"] / (km / 1000.0) / 1e12
        r["samples_per_step"] = f.get("samples")
        r["clocks"] = f["clocks"]
        return r

    kern_s = statistics.mean(head["kern_ms"]) / 1000.0
    red_per_sample = bwd_tc_reductions_per_sample()
    achieved = head["samples"] * TRAIN_BYTES_PER_SAMPLE_F16 / kern_s / 1e9
    rays_total = R * world * steps
    line = {
        "metric": METRIC, "value": rays_total / t_step, "unit": "rays/s", "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": 1000.0 * t_step / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "grid8 training step (sampling, gather, MLP, local render, composite, loss "
                               "L2 + 0.01 distortion, backward, Adam): K=8 2x2x2 over [-1,1]^3, L=16 F=2 T=2^19 "
                               "(16->2048), FP16 hash tables, BF16 MLP 32-64-64-4 with FP32 accumulation on the "
                               "tensor cores, FP32 Adam masters, 2^18 rays from 64 pinhole cameras, S=128; "
                               "the target colours are uniform random instead of the 200-blob render (the "
                               "dense field's throughput does not depend on the target)",
                   "rays_per_gpu": R, "samples_per_step": int(head["samples"]),
                   **({"reduced_batch": "first %d rays of the workload (profiling capture, not a bench value)"
                       % R} if args.profile_rays > 0 else {}),
                   "l2": "flushed before every timed step (252 MB write, outside the step events)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "train_target": "uniform random colours (throughput does not depend on the target)",
                   "precision": "FP16 tables, BF16 MLP operands, FP32 accumulation, gradients and Adam"},
        "e2e": {"value": rays_total / t_e2e, "unit": "rays/s", "h2d_bytes_per_step": int(3 * R * 12),
                "d2h_bytes_per_step": 12},
        "gpu_launches": head_launches,
        "roofline": {"bound": "hbm", "kernel": head["kernel"], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": bwd_tc_traffic(),
                     "frac_kind": "notional: algorithmic bytes against the HBM copy peak; the kernel is not "
                                  "bound by HBM bandwidth (binding_resource)",
                     "basis": "%d B/sample algorithmic (records: 16-bit features 64 B + geometry 48 B + chunk "
                              "adjoints 1 B; FP32 gradient read-modify-write 2048 B) x %d samples / mean kernel time "
                              "%.3f ms (%s peak)"
                              % (TRAIN_BYTES_PER_SAMPLE_F16, head["samples"], 1000 * kern_s, src),
                     "binding_resource": "the table-gradient reductions: 63.5 sector requests per sample "
                                         "(runs of samples in the same cell merged, both halves of an x-pair "
                                         "in one instruction; 96 with neither), near the rate the reduction "
                                         "probe measures (binding); issue 52%, L1 throughput 63%, tensor "
                                         "pipe 9% (ncu, reduced batch); not HBM (DRAM traffic 0.07x the "
                                         "algorithmic bytes, the swept region's gradient lines stay in L2)",
                     "binding": {"resource": "scattered FP32 vector reductions (32-byte sector requests)",
                                 "per_sample": red_per_sample,
                                 "per_sample_kind": "measured by ncu on this build (l1tex__t_sectors_pipe_lsu_"
                                                    "mem_global_op_red); 96 without merging runs of samples in "
                                                    "the same cell and x-pair halves",
                                 "achieved_per_s": None if red_per_sample is None
                                 else head["samples"] * red_per_sample / kern_s,
                                 "ceiling_per_s": red_ceiling,
                                 "frac": None if red_per_sample is None
                                 else head["samples"] * red_per_sample / kern_s / red_ceiling,
                                 "ceiling_kind": "measured in this run: nerfxl_probe_reduction_rate, 4 CTAs x "
                                                 "256 threads per SM issuing red.global.add.v4.f32 (evict-last) "
                                                 "to random 16-byte slots of a 48 MB buffer, one sector request "
                                                 "per lane"}},
        "forms": {k: summary(v) for k, v in forms.items()},
        "clocks": head["clocks"],
    }
    fwd = line["forms"].get("grid8_fwd_f16tab_bf16mlp")
    sps = fwd_tc_sectors_per_sample()
    if fwd is not None and sps is not None and fwd.get("kernel_ms"):
        got = fwd["samples_per_step"] * sps / (fwd["kernel_ms"] / 1000.0)
        fwd["binding"] = {"resource": "scattered table reads (L1 sectors)", "per_sample": sps,
                          "per_sample_kind": "measured by ncu on this build (l1tex__t_sectors_pipe_lsu_mem_global_"
                                             "op_ld)",
                          "achieved_per_s": got, "ceiling_per_s": ld_ceiling, "frac": got / ld_ceiling,
                          "ceiling_kind": "measured in this run: nerfxl_probe_load_rate, 4 CTAs x 256 threads per "
                                          "SM, 16 independent random 8-byte loads per thread in flight, 24 MB "
                                          "buffer"}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, tables, mlp, o, d, args.cpu_rays)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def C_int64():
    import ctypes

    return ctypes.c_int64(0)


def C_void(x):
    import ctypes

    return ctypes.c_void_p(x)


if __name__ == "__main__":
    main()
