#!/usr/bin/env python
"""Benchmark of the GB300 sonar path on the single-frame seabed workload.

Workload (the single-frame configuration): a 1024 x 1024-cell fBm seabed over
100 x 100 m (2,097,152 triangles) with 48 pier piles and 24 boxes (2,100,512
triangles), 16 materials; a 512-beam x 64-elevation sonar (130 x 20 deg,
0.1-20 m, 1000 range x 512 azimuth bins) with a 1024 x 576 fan image.

One step = one batch of B frames (B sensor poses along a trajectory) through
the whole path: the batched persistent launch (ray cast, intensity, binning,
noise), normalisation + fan, and the adjoint (gradient of a fixed upstream
gradient image with respect to alpha, gain and the 16 reflectivities), each
replayed from a captured CUDA graph.  `value` = frames per second of that
forward+adjoint step with inputs resident in HBM; `e2e` = the same through
the public API with the step's inputs copied from pinned host memory and its
outputs (polar + fan images, gradient) copied back inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank renders its own B frames (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sonar frames/s & Mrays/s, batched vs single, fwd+adjoint; % of memory roofline"
UNIT = "frames/s"
WORKLOAD = ("single-frame seabed: 1024^2-cell fBm heightfield over 100 m (2,097,152 tris) + 48 piles "
            "+ 24 boxes = 2,100,512 tris, 16 materials; sonar 512 beams x 64 elevations (130 x 20 deg), "
            "0.1-20 m, 1000 x 512 polar bins, 1024 x 576 fan")
ALPHA, GAIN = 0.04, 1.5


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--frames", type=int, default=64, help="frames (sensor poses) per step and rank")
    p.add_argument("--ref-rays", type=int, default=4096, help="rays the reference arm (the oracle) casts per step")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the single-frame and e2e legs")
    p.add_argument("--small", action="store_true", help="a small case for profiler captures")
    p.add_argument("--tune", default=None, metavar="COLS,TB,BLOCK,OCC",
                   help="fixed launch configuration instead of autotuning (profiler captures, whose "
                        "replays distort the autotuner's timings)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other configurations (differentiable fit, heterogeneous batch, large, dense rays)")
    p.add_argument("--configs", action="store_true",
                   help="also measure the large scene with 1024 materials")
    return p.parse_args()


def rank_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


SEED = 1   # Philox key of every frame; the counter's frame word is the global frame index


def frame_shard(rank: int, world: int, frames: int):
    """Global frame indices rendered by `rank`: the job's world x frames frames
    (poses of one trajectory) are split into contiguous blocks, one per rank,
    so no frame is rendered twice and no rank needs another's data."""
    if not 0 <= rank < world or frames < 0:
        raise ValueError(f"bad shard: rank {rank}, world {world}, frames {frames}")
    return list(range(rank * frames, (rank + 1) * frames))


def max_over_ranks(x: float, device) -> float:
    """The maximum of `x` over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(frames_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job frames/s: the frames all ranks rendered over the slowest rank's time."""
    return frames_per_rank * steps * world / (max_ms / 1000.0)


def workload(rank: int, world: int, frames: int, small: bool):
    """The scene, its sonar, and this rank's share of a trajectory of
    world x frames poses (with their global frame indices)."""
    from paper_2503_01074_gb300 import scenes as S
    if small:
        mesh, mu, hfn = S.single_frame_scene(n_cells=512, extent=100.0)
    else:
        mesh, mu, hfn = S.single_frame_scene()
    base = S.sensor_single(hfn)
    fids = frame_shard(rank, world, frames)
    every = S.trajectory(base, hfn, world * frames, radius=20.0, seed=0)
    return mesh, mu, base, [every[f] for f in fids], fids


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    """SM clock and throttle reasons sampled while the timed region runs.

    A poller thread reads the NVIDIA driver's NVML library (through ctypes, read-only
    queries) every millisecond, since the timed region can be shorter than
    nvidia-smi's sampling period; where NVML does not load, nvidia-smi samples
    every 200 ms instead."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clocks-event reason bits
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self, gpu_index: int, uuid: str | None = None):
        self.proc = None
        self.path = None
        self.thread = None
        self.samples = []
        self.source = None
        if self._start_nvml(gpu_index, uuid):
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi, 200 ms"
        except Exception:
            self.proc = None

    def _start_nvml(self, gpu_index, uuid):
        import ctypes
        import threading
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            ok = False
            if uuid:
                ok = lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(h)) == 0
            if not ok:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(h)) == 0
            if not ok:
                return False
            reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0:   # 1 = SM clock
                return False
        except Exception:
            return False
        self.max_mhz = float(mx.value)
        self.stop_flag = threading.Event()

        def poll():
            clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
            while not self.stop_flag.is_set():
                if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and \
                        reasons_fn(h, ctypes.byref(rs)) == 0:
                    self.samples.append((float(clk.value), int(rs.value)))
                time.sleep(0.001)

        self.thread = threading.Thread(target=poll, daemon=True)
        self.thread.start()
        self.source = "NVML, 1 ms"
        return True

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            if not self.samples:
                return None
            reasons = sorted({n for _, r in self.samples for n, b in self.REASON_BITS.items() if r & b})
            return {"sm_mhz": float(np.median([c for c, _ in self.samples])), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.samples), "source": self.source}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def oracle_pass(mesh, mu, spec, n_rays, seed=0, tv=None):
    """One pass of the oracle over `n_rays` sampled rays of the frame (all of
    them when n_rays = the frame's rays): brute-force FP64 ray casting, then
    the whole per-bin pipeline on the full image (binning, noise,
    normalisation, fan).  Returns (seconds casting, seconds per-bin, threads,
    the per-ray results)."""
    import oracle as O
    tv = O.tri_verts(mesh) if tv is None else tv
    ids = None if n_rays >= spec.n_rays else \
        np.sort(np.random.default_rng(seed).choice(spec.n_rays, n_rays, replace=False))
    t0 = time.perf_counter()
    r = O.render(mesh, mu, ALPHA, GAIN, spec, O.Params(),
                 ray_ids=ids if ids is not None else np.arange(spec.n_rays), tv=tv)
    t1 = time.perf_counter()
    P = np.zeros(spec.n_range_bins * spec.n_az_bins)
    O.lib().oracle_accumulate(len(r["key"]), r["key"], r["score"], P.size, P)
    In = O.noise(spec, P.reshape(spec.n_range_bins, spec.n_az_bins), 0, 0, O.Params())
    N, _, _ = O.normalise(spec, In, 1)
    O.fan_image(spec, N, spec.fan_w, spec.fan_h)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, int(r["hits"]["threads"]), r


def cpu_baseline(mesh, mu, spec):
    """The oracle on one whole frame of the workload (every ray cast by brute
    force in FP64, then the per-bin pipeline), timed on this host's cores."""
    t_rays, t_bins, threads, r = oracle_pass(mesh, mu, spec, spec.n_rays)
    total = t_rays + t_bins
    return {"value": 1.0 / total, "unit": UNIT, "cores": threads, "kind": "oracle",
            "Mrays_s": spec.n_rays / total / 1e6,
            "sample": (f"one whole frame: all {spec.n_rays} rays cast by brute force in FP64 ({t_rays:.1f} s) "
                       f"+ binning, noise, normalisation and fan of the full image ({t_bins:.2f} s)")}, r, total


SMALL_WORKLOAD = ("profiling case: 512^2-cell fBm heightfield over 100 m (524,288 tris) + 48 piles + 24 boxes "
                  "= 527,648 tris, 16 materials; the single-frame sonar")


def arm_config(frames, rays_per_frame, world, small=False):
    """The workload description both arms print."""
    return {"workload": SMALL_WORKLOAD if small else WORKLOAD, "frames_per_step": frames,
            "rays_per_frame": rays_per_frame,
            "step": "batched forward (graph) + batched adjoint (graph)",
            "cast": "bounded at the sonar's maximum range r_max (returns beyond it are not searched)",
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"dp{world}"}


def run_reference(args):
    """The oracle as the reference arm: each step casts a seeded sample of
    `--ref-rays` rays of one frame of the workload by brute force in FP64 and
    runs the per-bin pipeline on the full image; the step counts as that
    share of a frame, so ms_per_step is the step's wall time and value the
    frames per second it sustains."""
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    mesh, mu, base, poses, _ = workload(0, 1, max(args.frames, 1), args.small)
    import oracle as O
    tv = O.tri_verts(mesh)
    n = min(args.ref_rays, base.n_rays)
    for k in range(args.warmup):
        oracle_pass(mesh, mu, poses[k % len(poses)], 256, seed=k, tv=tv)
    walls, threads = [], 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        _, _, threads, _ = oracle_pass(mesh, mu, poses[k % len(poses)], n, seed=100 + k, tv=tv)
        walls.append(time.perf_counter() - t0)
    share = n / base.n_rays
    value = share * args.steps / float(np.sum(walls))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": arm_config(args.frames, base.n_rays, 1, args.small),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(threads), "kind": "oracle",
                             "sample": f"each step: {n} of the {base.n_rays} rays of one frame ({share:.3f} "
                                       f"of the frame) cast by brute force in FP64, then binning, noise, "
                                       f"normalisation and fan of the full image; a step counts as "
                                       f"{share:.3f} frames"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def timed(fn, steps, stream):
    """Mean device milliseconds of fn() over `steps` runs (after one warm-up)."""
    import torch
    fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms))


WIDE = 16   # ray-cast variant flag of a tuning row: the 8-wide tree (256-byte nodes)


def shape_of(spec):
    return [spec.n_beams, spec.n_elev, spec.n_range_bins, spec.n_az_bins]


def trace_bytes(son, sid, spec, prm, wide=None):
    """Algorithmic bytes of one sensor's ray cast, from the counter mode: the
    distinct nodes (128 bytes 4-wide, 256 bytes 8-wide) and 48-byte triangles
    its rays touch plus a 16-byte record per ray.  The counter mode walks the
    tree of the shape's tuning row; `wide` (True / False) walks the 8-wide or
    4-wide tree instead, by a temporary row."""
    rows = son.tune_get().tolist()
    row = next((r for r in rows if r[:4] == shape_of(spec)), None)
    if wide is not None:
        forced = list(row) if row else shape_of(spec) + [1, 8, 128, 8]
        forced[7] = (forced[7] | WIDE) if wide else (forced[7] & ~WIDE)
        son.tune_set([forced])
        row = forced
    try:
        st = son.trace_stats(sid, spec, prm)
    finally:
        if wide is not None:
            if rows:
                son.tune_set(rows)
            # a temporary row for an untuned shape cannot be removed; it names the
            # tiles that shape would default to
    node = 256 if (row and row[7] & WIDE) else 128
    return st["nodes_touched"] * node + st["tris_touched"] * 48 + spec.n_rays * 16, st


def trace_roofline(son, items, trace_ms, peak, scale=1.0):
    """The ray-cast launch's HBM roofline for a batch: algorithmic bytes (per
    item, the distinct nodes and triangles its rays touch plus a 16-byte record
    per ray, from the counter mode) over the launch's in-graph time.  `items`
    may be a sample of the batch, `scale` the batch size over the sample size."""
    from paper_2503_01074_gb300.sonar import RenderParams
    alg = 0
    for sid, spec in items:
        alg += trace_bytes(son, sid, spec, RenderParams())[0]
    alg *= scale
    gbs = alg / (trace_ms / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "algorithmic_bytes_per_launch": int(alg), "avg_launch_ms": trace_ms,
            "sample": f"{len(items)} of {int(round(len(items) * scale))} items"}


def oracle_subset(mesh, mu, spec, frac, seed, params=None, grad=False, fan=True, tv=None):
    """Seconds per frame of the oracle, estimated from a seeded subset of
    `frac` of the frame's rays (cast by brute force in FP64; the time scaled by
    the frame's rays over the subset's) plus the per-bin pipeline of the full
    image (binning, noise, normalisation, fan when the sensor has one) and,
    with `grad`, the analytic gradient (its per-ray part scaled likewise)."""
    import oracle as O
    params = params or O.Params()
    tv = O.tri_verts(mesh) if tv is None else tv
    n = max(32, int(round(frac * spec.n_rays)))
    ids = np.sort(np.random.default_rng(seed).choice(spec.n_rays, n, replace=False))
    t0 = time.perf_counter()
    r = O.render(mesh, mu, ALPHA, GAIN, spec, params, ray_ids=ids, tv=tv)
    t1 = time.perf_counter()
    nb = spec.n_range_bins * spec.n_az_bins
    P = np.zeros(nb)
    O.lib().oracle_accumulate(n, r["key"], r["score"], nb, P)
    In = O.noise(spec, P.reshape(spec.n_range_bins, spec.n_az_bins), 0, 0, params)
    N, _, _ = O.normalise(spec, In, params.normalise)
    if fan and spec.fan_w > 0:
        O.fan_image(spec, N, spec.fan_w, spec.fan_h)
    t2 = time.perf_counter()
    t_grad = 0.0
    if grad:
        G = np.random.default_rng(seed + 1).normal(size=nb) * 1e-3
        t3 = time.perf_counter()
        O.grad(mesh, mu, ALPHA, GAIN, spec, params, 0, 0, G, In, r)
        t_grad = time.perf_counter() - t3
    per_frame = (t1 - t0) * spec.n_rays / n + (t2 - t1) + t_grad
    return per_frame, {"rays_cast": n, "of_rays": spec.n_rays, "cast_s": t1 - t0, "per_bin_s": t2 - t1,
                       "grad_s": t_grad, "threads": int(r["hits"]["threads"])}


def measure_configs(son, args, peak, oracle_frame):
    """The other workload configurations (not the headline line), each with
    its ray-cast launch's HBM roofline and the oracle's estimate from a ray
    subset: the differentiable fit, the heterogeneous batch against single
    renders, the large scene forward + adjoint with recomputed hits, and the
    dense-ray frame (and, with --configs, the large scene with 1024
    materials)."""
    import torch
    import oracle as O
    from paper_2503_01074_gb300 import scenes as S
    from paper_2503_01074_gb300.autograd import sonar_render
    from paper_2503_01074_gb300.sonar import RenderParams
    stream = torch.cuda.current_stream()
    prm = RenderParams()
    steps = args.steps
    out = {}

    # differentiable: 64 materials, a target rendered with perturbed parameters,
    # MSE loss, 32 sequential fit iterations (forward + adjoint each) through
    # the autograd function on the single-sensor path
    mesh, mu, hfn = S.single_frame_scene(n_mat=64, mu_lo=0.05, mu_hi=0.95)
    sid = son.upload_mesh(mesh)
    spec = S.sensor_single(hfn)
    mu_t = (mu * np.random.default_rng(5).uniform(0.8, 1.2, 64)).astype(np.float32)
    target = son.render(sid, spec, son.theta(0.06, 1.2, mu_t), prm, 1, 1, fan=False)["polar"].clone()

    def fit(n_it):
        th = son.theta(ALPHA, GAIN, mu).requires_grad_(True)
        opt = torch.optim.Adam([th], lr=0.02)
        losses = []
        for _ in range(n_it):
            opt.zero_grad()
            loss = torch.mean((sonar_render(th, son, sid, spec, prm, 1, 1, save_hits=True) - target) ** 2)
            loss.backward()
            opt.step()
            losses.append(loss.detach())
        return [float(x) for x in losses]
    fit(4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = fit(32)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    b1 = son.batch([(sid, spec, 1, 1)])
    theta = son.theta(ALPHA, GAIN, mu)
    for _ in range(3):
        b1.render(theta, prm, hits=True, fan=False)
    tr = []
    for _ in range(steps):
        b1.render(theta, prm, hits=True, fan=False)
        tr.append(b1.timings()["trace"])
    b1.close()
    ent = {"materials": 64, "iterations": 32, "fwd_bwd_fps": 32 / fit_s, "ms_per_iteration": 1e3 * fit_s / 32,
           "loss_first": losses[0], "loss_last": losses[-1],
           "roofline": trace_roofline(son, [(sid, spec)], float(np.mean(tr)), peak)}
    if oracle_frame is not None:
        # the oracle's forward is the headline's whole-frame time (same seabed
        # geometry, so the same brute-force cost), plus its analytic gradient
        r, t_frame, ospec, omesh, omu = oracle_frame
        nb = ospec.n_range_bins * ospec.n_az_bins
        P = np.zeros(nb)
        O.lib().oracle_accumulate(len(r["key"]), r["key"], r["score"], nb, P)
        In = O.noise(ospec, P.reshape(ospec.n_range_bins, ospec.n_az_bins), 0, 0, O.Params())
        G = np.random.default_rng(9).normal(size=nb) * 1e-3
        t0 = time.perf_counter()
        O.grad(omesh, omu, ALPHA, GAIN, ospec, O.Params(), 0, 0, G, In, r)
        t_g = time.perf_counter() - t0
        ent["oracle"] = {"fwd_bwd_fps": 1.0 / (t_frame + t_g), "kind": "oracle",
                         "sample": f"one whole frame cast by brute force ({t_frame:.1f} s, the headline baseline's) "
                                   f"+ the analytic gradient ({t_g:.2f} s)"}
    out["differentiable_fit"] = ent
    son.release(sid)

    # heterogeneous batch: 4 scenes, 128 sensors of three shapes, vs 128 single renders
    scenes, mu, sensors = S.batched_workload()
    sids = [son.upload_mesh(m) for m, _ in scenes]
    items = [(sids[si], spec, 500 + k, k) for k, (si, spec) in enumerate(sensors)]
    theta = son.theta(ALPHA, GAIN, mu)
    b = son.batch(items)
    b.autotune(theta, prm)
    rays = sum(spec.n_rays for _, spec in sensors)
    ms_b = timed(lambda: b.render(theta, prm, hits=True, fan=True), steps, stream)
    outs = [son.render(sid, spec, theta, prm, seed, fr, hits=True, fan=True) for sid, spec, seed, fr in items]

    def singles():
        for (sid, spec, seed, fr), o in zip(items, outs):
            son.render(sid, spec, theta, prm, seed, fr, hits=True, fan=True, outputs=o)
    ms_s = timed(singles, max(2, steps // 2), stream)
    b.render(theta, prm, hits=True, fan=True)
    ph = b.timings()
    ent = {"sensors": len(items), "rays": rays, "batched_fwd_fps": len(items) / ms_b * 1e3,
           "single_fwd_fps": len(items) / ms_s * 1e3, "batched_Mrays_s": rays / ms_b / 1e3,
           "speedup": ms_s / ms_b, "phase_ms": ph,
           "roofline": trace_roofline(son, [(sid, spec) for sid, spec, _, _ in items], ph["trace"], peak)}
    if oracle_frame is not None:
        est, shapes = {}, {}
        for si, spec in sensors:
            key = (spec.n_beams, spec.n_elev, spec.n_range_bins)
            if key not in est:
                est[key], shapes[str(key)] = oracle_subset(scenes[si][0], mu, spec, 0.01, 31)
        per_frame = [est[(spec.n_beams, spec.n_elev, spec.n_range_bins)] for _, spec in sensors]
        ent["oracle"] = {"fwd_fps": len(per_frame) / float(np.sum(per_frame)), "kind": "oracle",
                         "sample": "1% of the rays of one sensor of each shape (beams, elevations, range bins), "
                                   "scaled to its frame, + its per-bin pipeline; weighted by the batch's mix",
                         "shapes": shapes}
    out["heterogeneous_batch"] = ent
    b.close()
    del outs
    for sid in sids:
        son.release(sid)

    # large: 33.6M triangles, 1024 x 256 rays, 4000 bins, 0.1-60 m; 256 poses,
    # forward + adjoint with recomputed hits (and with 1024 materials: --configs)
    for n_mat, name in ((64, "large"), (1024, "large_1024_materials")):
        if n_mat == 1024 and not args.configs:
            continue
        t0 = time.perf_counter()
        mesh, mu, hfn = S.large_scene(n_mat=n_mat)
        gen_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sid = son.upload_mesh(mesh)
        torch.cuda.synchronize()
        build_ms = 1000.0 * (time.perf_counter() - t0)
        base = S.sensor_single(hfn, n_beams=1024, n_elev=256, n_range_bins=4000, r_min=0.1, r_max=60.0,
                               fan_w=0, fan_h=0)
        poses = S.trajectory(base, hfn, 256, radius=60.0, seed=7)
        theta = son.theta(ALPHA, GAIN, mu)
        b = son.batch([(sid, p, 900 + k, k) for k, p in enumerate(poses)])
        b.autotune(theta, prm)
        G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(2)).to(son.device) * 1e-3
        d = torch.empty_like(theta)

        def fwd_adj():
            b.render(theta, prm, hits=False, fan=False)
            b.backward(theta, prm, G, hits=False, out=d)
        ms = timed(fwd_adj, max(2, steps // 2), stream)
        ph = b.timings()
        ent = {"tris": mesh.n_tris, "materials": n_mat, "frames": len(poses), "rays_per_frame": base.n_rays,
               "fwd_adj_recompute_fps": len(poses) / ms * 1e3,
               "Mrays_s": len(poses) * base.n_rays / ms / 1e3, "scene_build_ms": build_ms,
               "scene_generation_s": gen_s, "phase_ms": ph,
               "roofline": trace_roofline(son, [(sid, p) for p in poses[::32]], ph["trace"], peak,
                                          scale=len(poses) / len(poses[::32]))}
        if oracle_frame is not None and n_mat == 64:
            pf, info = oracle_subset(mesh, mu, poses[0], 0.002, 41, grad=True, fan=False)
            ent["oracle"] = {"fwd_adj_fps": 1.0 / pf, "kind": "oracle", "detail": info,
                             "sample": "0.2% of one frame's rays cast by brute force and differentiated, scaled "
                                       "to the frame, + the per-bin pipeline and gradient terms of the full image"}
        out[name] = ent
        b.close()
        son.release(sid)
        del mesh
    # dense rays: 3000 x 460 rays into 350 x 220 bins
    mesh, mu, hfn = S.single_frame_scene()
    sid = son.upload_mesh(mesh)
    spec = S.sensor_single(hfn, n_beams=3000, n_elev=460, n_range_bins=350, n_az_bins=220, fan_w=440, fan_h=248)
    theta = son.theta(ALPHA, GAIN, mu)
    b = son.batch([(sid, spec, 3, 3)])
    b.autotune(theta, prm)
    ms = timed(lambda: b.render(theta, prm, hits=True, fan=True), steps, stream)
    ph = b.timings()
    ent = {"rays_per_frame": spec.n_rays, "bins": 350 * 220, "fwd_fps": 1e3 / ms,
           "Mrays_s": spec.n_rays / ms / 1e3, "phase_ms": ph,
           "roofline": trace_roofline(son, [(sid, spec)], ph["trace"], peak)}
    if oracle_frame is not None:
        pf, info = oracle_subset(mesh, mu, spec, 0.005, 51)
        ent["oracle"] = {"fwd_fps": 1.0 / pf, "kind": "oracle", "detail": info,
                         "sample": "0.5% of the frame's rays cast by brute force, scaled to the frame, + the "
                                   "per-bin pipeline of the full image"}
    out["dense_rays"] = ent
    b.close()
    son.release(sid)
    return out


# the kernel's sources, and the scene build whose tree shape decides what it reads
RAY_CAST_SOURCES = ("paper_2503_01074_gb300/csrc/trace.cu", "paper_2503_01074_gb300/csrc/devmath.cuh",
                    "paper_2503_01074_gb300/csrc/sonar_internal.cuh", "paper_2503_01074_gb300/csrc/bvh_build.cu")


def ray_cast_sources_sha():
    h = hashlib.sha256()
    for rel in RAY_CAST_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(tb: int, occ: int):
    """Per-frame counters of the ray-cast kernel for warp tile `tb` (beams per
    warp) and occupancy variant `occ` from the committed ncu summary, if they
    were taken on the current kernel sources (else None: the counters no
    longer describe the kernel): {"dram": DRAM bytes read + written, "l2": L2
    bytes (lts__t_bytes)}."""
    path = os.path.join(ROOT, "profiles", "k_trace_dram.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    pre = f"tb{tb}_occ{occ}_"
    if kv.get("ray_cast_sources_sha256_16") != ray_cast_sources_sha() or pre + "dram_bytes_per_frame" not in kv:
        return None
    return {"dram": float(kv[pre + "dram_bytes_per_frame"]), "l2": float(kv[pre + "l2_bytes_per_frame"])}


def l2_read_peak(son, dev, stream):
    """Measured L2 read rate (GB/s): the library's probe reads a 32 MiB buffer
    (a quarter of L2) 40 times per launch with L2-cached 16-byte loads on 4
    blocks of 512 per SM; best of 5 launches after 2 warm-ups."""
    import torch
    buf = torch.ones(8 << 20, dtype=torch.float32, device=dev)
    blocks = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    passes = 40
    best = None
    with torch.cuda.stream(stream):
        for r in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            son.probe_l2_read(buf, passes, blocks, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if r >= 2:
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
    del buf
    return {"gbs": (8 << 20) * 4 * passes / (best / 1000.0) / 1e9, "buffer_mib": 32, "passes": passes,
            "blocks": blocks, "how": "sonar_probe_l2_read: 16-byte ld.global.cg loads, best of 5 launches"}


def run_ours(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2503_01074_gb300 import scenes as S
    from paper_2503_01074_gb300.sonar import RenderParams, Sonar

    dev = torch.device("cuda", local)
    B = args.frames
    mesh, mu, base, poses, fids = workload(rank, world, B, args.small)
    son = Sonar(local)
    verts = torch.from_numpy(mesh.verts).to(dev)
    tris = torch.from_numpy(mesh.tris).to(dev)
    mat = torch.from_numpy(mesh.mat).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sid = son.upload(verts, tris, mat)
    torch.cuda.synchronize()
    build_ms = 1000.0 * (time.perf_counter() - t0)
    prm = RenderParams()
    theta = son.theta(ALPHA, GAIN, mu)
    items = [(sid, p, SEED, f) for p, f in zip(poses, fids)]
    if args.tune:
        cols, tb, block, occ = (int(x) for x in args.tune.split(","))
        son.tune_set([[base.n_beams, base.n_elev, base.n_range_bins, base.n_az_bins, cols, tb, block, occ]])
    batch = son.batch(items)
    if not args.tune:
        batch.autotune(theta, prm)
    G = torch.randn(batch.n_polar, generator=torch.Generator().manual_seed(5)).to(dev) * 1e-3
    dtheta = torch.empty_like(theta)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        batch.render(theta, prm, hits=True, fan=True)
        batch.backward(theta, prm, G, hits=True, out=dtheta)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    uuid = str(getattr(torch.cuda.get_device_properties(dev), "uuid", "") or "") or None
    clocks = Clocks(local, uuid) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase = []
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between timed iterations (256 MiB write)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phase.append(batch.timings())       # in-graph events of this step's replays
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    kern = batch.kernels()                 # our kernels per replayed step (graph kernel nodes)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    frames_total = B * args.steps * world
    value = job_value(B, args.steps, world, total_ms)
    rays_per_frame = base.n_rays
    trace_ms = float(np.mean([p["trace"] for p in phase]))
    bin_ms = float(np.mean([p["bin_noise"] for p in phase]))
    info = batch.info()

    extras = {}
    e2e = None
    # algorithmic bytes per frame (the per-kernel figures of the design notes):
    # the ray cast reads the nodes (128 B 4-wide, 256 B 8-wide) and triangles
    # (48 B) its rays touch and writes a 16-byte record per ray; binning reads the records and
    # writes I~; the normalisation + fan reads I~, writes N and the fan image
    # and reads the shared coordinate table (16 B a pixel, once per launch);
    # the adjoint reads I~ and G per bin, the records and a G gather per ray
    alg = 0
    visits = tests = exact = 0
    for p in poses:
        b_, st = trace_bytes(son, sid, p, prm)
        alg += b_
        visits += st["visits"]
        tests += st["tests"]
        exact += st["exact_tests"]
    nbin, npx, nray = base.n_range_bins * base.n_az_bins, base.fan_w * base.fan_h, base.n_rays
    bytes_frame = {"trace": alg / B, "bin_noise": nray * 16 + nbin * 4,
                   "normalise_fan": nbin * 8 + npx * 4 + npx * 16 / B,
                   "adjoint_rows": nbin * 8, "adjoint_gather": nray * 20}
    fwd_bytes = bytes_frame["trace"] + bytes_frame["bin_noise"] + bytes_frame["normalise_fan"]
    adj_bytes = bytes_frame["adjoint_rows"] + bytes_frame["adjoint_gather"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))

    def leg_roofline(bytes_per_frame, ms_per_frame):
        gbs = bytes_per_frame / (ms_per_frame / 1e3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "algorithmic_bytes_per_frame": int(bytes_per_frame), "device_ms_per_frame": ms_per_frame}

    if not args.no_extras:
        # batched forward only (the forward graph), its phases from in-graph events
        e_f = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        fwd_ms, fwd_ph = [], []
        for k in range(args.steps):
            flush.zero_()
            e_f[0].record(stream)
            batch.render(theta, prm, hits=True, fan=True)
            e_f[1].record(stream)
            torch.cuda.synchronize()
            fwd_ms.append(e_f[0].elapsed_time(e_f[1]))
            fwd_ph.append(batch.timings())
        fms = float(np.mean(fwd_ms))
        extras["batched_fwd"] = {
            "fps": B / (fms / 1e3), "device_ms_per_step": fms,
            "phase_ms": {k: float(np.mean([q[k] for q in fwd_ph])) for k in ("trace", "bin_noise", "normalise_fan")},
            "roofline": leg_roofline(fwd_bytes, fms / B),
            "phase_frac": {k: bytes_frame[k] * B / (float(np.mean([q[k] for q in fwd_ph])) / 1e3) / 1e9 / peak
                           for k in ("trace", "bin_noise", "normalise_fan")}}
        extras["batched_fwd_fps"] = extras["batched_fwd"]["fps"]
        # the same forward + adjoint as one graph (sonar_render_batch_step): the
        # adjoint branch runs beside the normalisation and fan
        st_ms = []
        for k in range(args.steps):
            flush.zero_()
            e_f[0].record(stream)
            batch.step(theta, prm, G, out=dtheta)
            e_f[1].record(stream)
            torch.cuda.synchronize()
            st_ms.append(e_f[0].elapsed_time(e_f[1]))
        sms = float(np.mean(st_ms))
        extras["combined_step"] = {"fps": B / (sms / 1e3), "device_ms_per_step": sms,
                                   "roofline": leg_roofline(fwd_bytes + adj_bytes, sms / B),
                                   "graph_kernels": batch.kernels()}
        # the timed step with an unbounded cast (clip_tmax = 0): the same images,
        # fans and gradient, with the rays that reach the seabed beyond r_max
        # followed to their returns
        prm_ub = RenderParams(clip_tmax=0)
        ub_ms, ub_trace = [], []
        for k in range(args.steps + 2):
            flush.zero_()
            e_f[0].record(stream)
            batch.render(theta, prm_ub, hits=True, fan=True)
            batch.backward(theta, prm_ub, G, hits=True, out=dtheta)
            e_f[1].record(stream)
            torch.cuda.synchronize()
            if k >= 2:
                ub_ms.append(e_f[0].elapsed_time(e_f[1]))
                ub_trace.append(batch.timings()["trace"])
        ums = float(np.mean(ub_ms))
        extras["unbounded_cast"] = {"fps": B / (ums / 1e3), "device_ms_per_step": ums,
                                    "trace_ms": float(np.mean(ub_trace))}
        step()
        torch.cuda.synchronize()
        # the plain single-sensor path: one sonar_render (and sonar_render_backward)
        # call per frame, no batching, no graph.  Host loop: the Python loop as a
        # caller runs it.  Device: the same calls queued behind a long sleep
        # kernel, so that the host is ahead and the frames' kernels run back to
        # back (their device time without host launch gaps).
        out = {"polar": torch.empty(base.n_range_bins, base.n_az_bins, device=dev),
               "noised": torch.empty(base.n_range_bins, base.n_az_bins, device=dev),
               "hits": torch.empty(base.n_rays, 4, dtype=torch.int32, device=dev),
               "fan": torch.empty(base.fan_h, base.fan_w, device=dev)}
        g1 = G[: base.n_range_bins * base.n_az_bins].view(base.n_range_bins, base.n_az_bins)
        for p in poses[:4]:
            son.render(sid, p, theta, prm, 0, 0, hits=True, fan=True, outputs=out)
            son.backward(sid, p, theta, prm, 0, 0, g1, out["noised"], out["hits"])
        torch.cuda.synchronize()

        def frames(with_adj):
            for j, p in enumerate(poses):
                son.render(sid, p, theta, prm, SEED, fids[j], hits=True, fan=True, outputs=out)
                if with_adj:
                    son.backward(sid, p, theta, prm, SEED, fids[j], g1, out["noised"], out["hits"])

        # the single-sensor path walks the tree its own launch calls for: the
        # 8-wide one when the frame's ray cast is at most one wave of one-warp
        # blocks (32 per SM), as the library decides
        row = next((r for r in son.tune_get().tolist() if r[:4] == shape_of(base)), None)
        tbw = row[5] if row else 8
        blocks1 = -(-base.n_beams // tbw) * -(-base.n_elev // (32 // tbw))
        wide1 = blocks1 <= 32 * torch.cuda.get_device_properties(dev).multi_processor_count
        tr1 = float(np.mean([trace_bytes(son, sid, p, prm, wide=wide1)[0] for p in poses]))
        fwd_bytes1 = fwd_bytes - bytes_frame["trace"] + tr1
        single = {"tree": "8-wide" if wide1 else "4-wide"}
        for with_adj in (False, True):
            host, devt = [], []
            for k in range(max(2, args.steps // 2)):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                e_f[0].record(stream)
                frames(with_adj)
                e_f[1].record(stream)
                torch.cuda.synchronize()
                host.append(1e3 * (time.perf_counter() - t0))
                flush.zero_()
                torch.cuda._sleep(60_000_000)          # about 30 ms of GPU time, longer than the host loop
                e_f[0].record(stream)
                frames(with_adj)
                e_f[1].record(stream)
                torch.cuda.synchronize()
                devt.append(e_f[0].elapsed_time(e_f[1]))
            tag = "fwd_adj" if with_adj else "fwd"
            hms, dms = float(np.mean(host)) / B, float(np.mean(devt)) / B
            single[tag] = {"fps": 1e3 / hms, "host_ms_per_frame": hms, "device_ms_per_frame": dms,
                           "device_fps": 1e3 / dms,
                           "roofline": leg_roofline(fwd_bytes1 + (adj_bytes if with_adj else 0), dms)}
            extras["single_fwd_adj_fps" if with_adj else "single_fwd_fps"] = single[tag]["fps"]
        single["launches_per_frame"] = {"fwd": 4, "adjoint": 3}
        single["note"] = ("host_ms_per_frame: the Python loop of one sonar_render (+ sonar_render_backward) "
                          "call per frame; device_ms_per_frame: the same calls with the host ahead of the "
                          "GPU (queued behind a sleep kernel), i.e. the frame's kernels and their "
                          "device-side launch gaps alone")
        extras["single"] = single
        # end to end through the public API with host buffers: every step copies
        # its inputs (theta, the upstream gradient image, the pose descriptors)
        # from pinned host memory and reads its outputs (polar and fan images,
        # gradient) back into pinned host memory.  Two batches with their own
        # device buffers alternate, so that one step's copies overlap the
        # neighbouring steps' kernels (copy-in, compute and copy-out streams).
        pin = lambda t: torch.empty(t.shape, dtype=t.dtype, pin_memory=True)   # noqa: E731
        h_theta, h_G = pin(theta), pin(G)
        h_theta.copy_(theta.cpu())
        h_G.copy_(G.cpu())
        batch2 = son.batch(items)
        lanes = [(batch, theta, G, dtheta), (batch2, theta.clone(), G.clone(), torch.empty_like(dtheta))]
        h_out = [(pin(batch.polar), pin(batch.fan), pin(dtheta)) for _ in range(2)]
        s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        for bj, th, Gj, dj in lanes:          # graphs of the second batch are captured here, untimed
            bj.render(th, prm, hits=True, fan=True, stream=s_cmp)
            bj.backward(th, prm, Gj, hits=True, out=dj, stream=s_cmp)
        torch.cuda.synchronize()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        used = [False, False]
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_start.record(s_cmp)
        s_in.wait_event(e_start)
        s_out.wait_event(e_start)
        for k in range(args.steps):
            j = k % 2
            bj, th, Gj, dj = lanes[j]
            if used[j]:
                s_in.wait_event(ev_done[j])          # the lane's previous kernels are done with its inputs
            with torch.cuda.stream(s_in):
                th.copy_(h_theta, non_blocking=True)
                Gj.copy_(h_G, non_blocking=True)
            bj.update(items, stream=s_in)
            ev_in[j].record(s_in)
            s_cmp.wait_event(ev_in[j])
            if used[j]:
                s_cmp.wait_event(ev_out[j])          # ... and its previous outputs are on the host
            with torch.cuda.stream(s_cmp):
                flush.zero_()
            bj.render(th, prm, hits=True, fan=True, stream=s_cmp)
            bj.backward(th, prm, Gj, hits=True, out=dj, stream=s_cmp)
            ev_done[j].record(s_cmp)
            s_out.wait_event(ev_done[j])
            hp, hf, hd = h_out[j]
            with torch.cuda.stream(s_out):
                hp.copy_(bj.polar, non_blocking=True)
                hf.copy_(bj.fan, non_blocking=True)
                hd.copy_(dj, non_blocking=True)
            ev_out[j].record(s_out)
            used[j] = True
        s_cmp.wait_event(ev_out[0])
        s_cmp.wait_event(ev_out[1])
        s_cmp.wait_stream(s_in)
        e_end.record(s_cmp)
        torch.cuda.synchronize()
        e2e_ms = [e_start.elapsed_time(e_end)]
        batch2.close()
        from paper_2503_01074_gb300.sonar import BatchItem
        h2d = theta.numel() * 4 + G.numel() * 4 + B * __import__("ctypes").sizeof(BatchItem)
        d2h = batch.polar.numel() * 4 + batch.fan.numel() * 4 + dtheta.numel() * 4
        e2e_total = max_over_ranks(float(sum(e2e_ms)), dev)
        e2e = {"value": job_value(B, args.steps, world, e2e_total), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "note": "inputs copied from and outputs read back to pinned host memory every step; two "
                       "batches alternate so copies overlap neighbouring steps' kernels; L2 flushed per step"}

    # underwater camera image (Eq. 1): 64 frames of 1920 x 1080, inputs resident
    # in HBM, 12 B of in-air RGB + 4 B of depth read and 12 B written per pixel
    uw = None
    if not args.no_extras:
        H, W, F = 1080, 1920, B
        J1 = torch.tensor(S.camera_rgb(H, W, 9), device=dev)
        d1 = torch.tensor(S.camera_seabed_depth(H, W), device=dev)
        Jg = J1.expand(F, H, W, 3).contiguous()
        dg = (d1 * torch.linspace(0.5, 1.5, F, device=dev).view(F, 1, 1)).contiguous()
        Ig = torch.empty_like(Jg)
        coef = [0.35, 0.12, 0.08, 0.30, 0.15, 0.10, 0.05, 0.25, 0.35]
        for _ in range(3):
            son.uw_image(Jg, dg, coef, out=Ig)
        e_u = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ums = []
        for _ in range(args.steps):
            flush.zero_()
            e_u[0].record(stream)
            son.uw_image(Jg, dg, coef, out=Ig)
            e_u[1].record(stream)
            torch.cuda.synchronize()
            ums.append(e_u[0].elapsed_time(e_u[1]))
        u_ms = float(np.mean(ums))
        px = F * H * W
        gbs = px * 28 / (u_ms / 1e3) / 1e9
        uw = {"frames": F, "pixels_per_frame": H * W, "ms_per_launch": u_ms, "Gpix_s": px / (u_ms / 1e3) / 1e9,
              "frames_s": F / (u_ms / 1e3),
              "roofline": {"bound": "hbm", "achieved": gbs, "unit": "GB/s", "algorithmic_bytes_per_pixel": 28}}
        del Jg, dg, Ig, J1, d1
    # DVL: 4096 vehicles x 256 steps of 20 ms on the same scene (1M poses, 4M
    # beams) per launch, then their measurement schedule
    dvl = None
    if not args.no_extras:
        from paper_2503_01074_gb300.sonar import DvlParams
        hfn_d = S.height_function(100.0, 2.0, 1)
        nv, ns, dt = 4096, 256, 0.02
        dp, dv = S.dvl_trajectories(hfn_d, nv, ns, dt, seed=21)
        dp = torch.tensor(dp.reshape(-1, 12), device=dev)
        dv = torch.tensor(dv.reshape(-1, 3), device=dev)
        prm_d = DvlParams()
        for _ in range(3):
            o = son.dvl(sid, dp, dv, prm_d, seed=5)
            son.dvl_schedule(o["period"].view(nv, ns), dt)
        e_d = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        dms, sms = [], []
        for _ in range(args.steps):
            flush.zero_()
            e_d[0].record(stream)
            o = son.dvl(sid, dp, dv, prm_d, seed=5)
            e_d[1].record(stream)
            son.dvl_schedule(o["period"].view(nv, ns), dt)
            e_d[2].record(stream)
            torch.cuda.synchronize()
            dms.append(e_d[0].elapsed_time(e_d[1]))
            sms.append(e_d[1].elapsed_time(e_d[2]))
        fl = o["flags"]
        dvl = {"vehicles": nv, "steps": ns, "poses": nv * ns, "ms_measure": float(np.mean(dms)),
               "ms_schedule": float(np.mean(sms)), "Mposes_s": nv * ns / float(np.mean(dms)) / 1e3,
               "Mbeams_s": 4 * nv * ns / float(np.mean(dms)) / 1e3,
               "valid_fraction": float(((fl & 16) != 0).float().mean().item())}
        del dp, dv, o
    # the dominant kernel's roofline: one ray-cast launch's algorithmic bytes
    # (summed over the B frames it renders) over its in-graph time
    achieved = alg / (trace_ms / 1000.0) / 1e9
    tune_row = [r for r in son.tune_get().tolist() if r[:4] == [base.n_beams, base.n_elev, base.n_range_bins,
                                                                 base.n_az_bins]]
    tb = traffic_from_profile(tune_row[0][5], tune_row[0][7]) if tune_row else None
    if uw is not None:
        uw["roofline"].update({"peak": peak, "frac": uw["roofline"]["achieved"] / peak})
    l2 = None
    if rank == 0:
        l2p = l2_read_peak(son, dev, stream)
        l2 = {"peak": l2p["gbs"], "unit": "GB/s", "peak_source": l2p, "achieved": None, "frac": None,
              "traffic": None}
        if tb is not None:
            l2["traffic"] = tb["l2"] * B
            l2["achieved"] = l2["traffic"] / (trace_ms / 1000.0) / 1e9
            l2["frac"] = l2["achieved"] / l2["peak"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tb["dram"] * B if tb is not None else None), "l2": l2,
                "warp_tile": (f"{tune_row[0][5]} beams x {32 // tune_row[0][5]} elevations, variant "
                              f"{tune_row[0][7]} ({'8' if tune_row[0][7] & WIDE else '4'}-wide tree, registers "
                              f"{'capped at 64' if tune_row[0][7] & 8 else 'uncapped'})" if tune_row else None),
                "kernel": "k_trace (ray generation + LBVH walk + Moller-Trumbore + bin key)",
                "avg_launch_ms": trace_ms, "algorithmic_bytes_per_launch": int(alg),
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    # the binning kernel streams hit records in and I~ out: its own figure
    bin_bytes = B * (base.n_rays * 16 + base.n_range_bins * base.n_az_bins * 4)
    extras["bin_noise_GBps"] = bin_bytes / (bin_ms / 1000.0) / 1e9
    extras["node4_visits_per_ray"] = visits / (B * base.n_rays)
    extras["tri_tests_per_ray"] = tests / (B * base.n_rays)
    extras["fp64_tests_per_ray"] = exact / (B * base.n_rays)
    # the whole forward + adjoint step against the HBM roofline, and per phase
    ph_mean = {k: float(np.mean([p[k] for p in phase])) for k in phase[0]}
    extras["step_roofline"] = dict(leg_roofline(fwd_bytes + adj_bytes, total_ms / args.steps / B),
                                   phase_frac={k: bytes_frame[k] * B / (ph_mean[k] / 1e3) / 1e9 / peak
                                               for k in ph_mean})

    cpu = oracle_frame = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, r0, t_frame = cpu_baseline(mesh, mu, poses[0])
        oracle_frame = (r0, t_frame, poses[0], mesh, mu)

    tune_rows = son.tune_get().tolist()     # the headline batch's tune (the configurations re-tune)
    configs = None
    if rank == 0 and world == 1 and not args.no_configs:
        batch.close()
        configs = measure_configs(son, args, peak, oracle_frame)
        batch = None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": arm_config(B, rays_per_frame, world, args.small),
                "Mrays_s": value * rays_per_frame / 1e6,
                "scene_build_ms": build_ms,
                "phase_ms": ph_mean,
                "batch": info, "tune": tune_rows,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": (kern["forward"] + kern["adjoint"]) * args.steps}
        line.update({k: (v if isinstance(v, dict) else float(v)) for k, v in extras.items()})
        if uw is not None:
            line["uw_image"] = uw
        if dvl is not None:
            line["dvl"] = dvl
        if configs is not None:
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    if batch is not None:
        batch.close()
    son.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
