#!/usr/bin/env python3
"""Light-field rendering benchmark: DirectL vs the standard paradigm on GB300.

Workload (``--workload 4k``, the default): a 3840x2160 lenticular panel with
45 views (pitch 8.1 subpixels, slant tan 0.18, offset 0, views spanning 40
degrees at distance 4, fov 40 degrees) and a seeded synthetic scene of 1M
Gaussians, SH degree 3, scale/rotation/opacity/SH stored in BF16 (means FP32),
with a 200-pose camera path sweeping the light-field centre's yaw over +-5
degrees.

One step = one DirectL light-field frame through the C ABI: view cameras,
multi-view EWA projection with SH colour, tile keys and the depth sort, and
front-to-back compositing of the required rays straight into the encoded
image.  The standard paradigm (every view rendered at panel resolution with
the tile rasteriser, then interweaved) is timed the same way on the same GPU
and reported under "standard".  Every step works on more than L2's worth of
data (2.2 GB of per-view splat records alone), so no L2 flush is added.
Timed frames run with stage events only (the compositing kernels' plain
variant); the pair counts behind the roofline come from an untimed pass
over the same poses with the counting variant.

Two more sections follow on fresh contexts (skipped under torchrun):
"graph_batched" renders the 8K panel (100 views, 3M Gaussians, BF16) from a
captured CUDA graph of the frame batch after the autotuner has picked the
tile shape, and "serving" runs the continuous-batching server on a mix of
256 Poisson-arriving requests (scenes of 100k-3M Gaussians in FP16, 1080p/45,
4K/45 and 4K/60 displays, 150 GB HBM budget) and reports p50/p99 latency.

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(a bounded sample of rays per step, extrapolated to frames/s).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "light-field frames/s & subpixels/s: DirectL vs 45-view+interweave, same GB300, at oracle tol"
# compositing work per (ray, Gaussian) pair: dx, dy (2), quadratic form (9),
# clamp and threshold compare (2) -> 13 FP32 ops + 1 ex2; a composited pair
# adds T(1-alpha), alpha*T and three colour FMAs (9 more).
FLOP_PER_EVAL = 13
FLOP_PER_BLEND = 9
SMS = 152
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16  # ex2 results an SM produces per clock
# algorithmic bytes of the compositing stage (see the roofline section)
KEY_BYTES = 8
RECORD_BYTES = 32   # conic (6 floats) and packed colour (64 bits): the whole stored record
RAY_COLOUR_BYTES = 12
HBM_FALLBACK_GBS = 6800.0


def compositing_roofline(comp_ms: float, keys: float, n_rays: float, evaluated: float,
                         blended: float, hbm_gbs: float, hbm_source: str,
                         alu_peaks: dict | None = None) -> dict:
    """Roofline of the compositing stage from its algorithmic work.

    Three lower bounds on the stage's time:
      FP32: FLOP_PER_EVAL ops per evaluated (ray, Gaussian) pair plus
            FLOP_PER_BLEND per composited pair, against 152 SMs x 128 lanes
            x 2 (FMA) x 2070 MHz;
      MUFU: one ex2 per evaluated pair, against 152 SMs x 16 x 2070 MHz;
      HBM:  per key its 8-byte sort key and its 32-byte record (the six
            conic floats the test and blend need and the packed colour), per
            ray 12 bytes of colour, against the measured copy bandwidth.
    The roofline is the largest of the three (the binding one); its fraction
    is that bound's time over the stage's time.  alu_peaks (from
    dl_measure_peaks on the same GPU) replaces the derived FP32 and ex2 peaks
    by measured ones: the larger of the scalar and packed FP32 FMA rates."""
    comp_s = comp_ms / 1e3 if comp_ms > 0 else float("inf")
    clk = 2070.0
    flops = FLOP_PER_EVAL * evaluated + FLOP_PER_BLEND * blended
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
    mufu_peak = SMS * MUFU_LANES_PER_SM * clk * 1e6
    alu_source = "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2070 MHz"
    mufu_source = "derived: 152 SMs x 16 ex2 a clock x 2070 MHz"
    if alu_peaks:
        peak_tflops = max(alu_peaks["fp32_tflops"], alu_peaks["fp32x2_tflops"])
        mufu_peak = alu_peaks["ex2_per_s"]
        alu_source = ("measured: FP32 FMA microbenchmark on this GPU (dl_measure_peaks; "
                      f"scalar {alu_peaks['fp32_tflops']:.1f}, packed FP32x2 "
                      f"{alu_peaks['fp32x2_tflops']:.1f} TFLOP/s)")
        mufu_source = "measured: ex2.approx microbenchmark on this GPU (dl_measure_peaks)"
    bytes_alg = keys * (KEY_BYTES + RECORD_BYTES) + n_rays * RAY_COLOUR_BYTES
    bounds_ms = {"hbm": 1e3 * bytes_alg / (hbm_gbs * 1e9),
                 "alu": 1e3 * flops / (peak_tflops * 1e12),
                 "mufu": 1e3 * evaluated / mufu_peak}
    bound = max(bounds_ms, key=bounds_ms.get)
    alu = {"achieved": flops / comp_s / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
           "frac": flops / comp_s / 1e12 / peak_tflops,
           "peak_source": alu_source, "mufu_peak_per_s": mufu_peak, "mufu_source": mufu_source,
           "flop_per_launch": flops,
           "flop_model": f"{FLOP_PER_EVAL} per evaluated (ray, Gaussian) pair + "
                         f"{FLOP_PER_BLEND} per composited pair"}
    if bound == "hbm":
        head = {"bound": "hbm", "achieved": bytes_alg / comp_s / 1e9, "peak": hbm_gbs,
                "unit": "GB/s", "frac": bytes_alg / comp_s / 1e9 / hbm_gbs,
                "peak_source": hbm_source}
    else:  # FP32 or MUFU arithmetic binds: reported against the FP32 peak
        head = {"bound": "alu", "achieved": alu["achieved"], "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": bounds_ms[bound] / comp_ms if comp_ms > 0 else 0.0,
                "peak_source": alu["peak_source"] + f" ({bound} binds)"}
    return {**head, "bytes_per_launch": bytes_alg, "ms_per_launch": comp_ms,
            "byte_model": f"{KEY_BYTES} B key + {RECORD_BYTES} B record per key, "
                          f"{RAY_COLOUR_BYTES} B per ray",
            "bounds_ms": bounds_ms, "alu": alu}


def stage_roofline(name: str, ms: float, bytes_alg: float, model: str, hbm_gbs: float,
                   hbm_source: str) -> dict:
    """HBM roofline of a bandwidth-bound stage: algorithmic bytes over the
    stage's CUDA-event time against the measured copy bandwidth."""
    s = ms / 1e3 if ms > 0 else float("inf")
    return {"kernel": name, "bound": "hbm", "achieved": bytes_alg / s / 1e9, "peak": hbm_gbs,
            "unit": "GB/s", "frac": bytes_alg / s / 1e9 / hbm_gbs, "peak_source": hbm_source,
            "bytes_per_launch": bytes_alg, "ms_per_launch": ms, "byte_model": model}


def attribute_bytes(spec: W.SceneSpec) -> int:
    """Bytes of one stored Gaussian: FP32 mean, then log-scale (3), rotation
    (4), opacity (1) and SH (3 (d+1)^2) in the storage type."""
    elem = 4 if spec.dtype == "f32" else 2
    return 12 + elem * (3 + 4 + 1 + 3 * (spec.sh_degree + 1) ** 2)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and its ISA."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                name = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu model")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{name or 'unknown'} ({platform.machine()})"


def measured_hbm_gbs():
    """The copy bandwidth measured on the GB300s (driver-written
    peaks file), else the earlier single measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        if v > 0:
            return v, "measured: STREAM-style copy on this pool's GB300s (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return HBM_FALLBACK_GBS, "fallback: 6.8 TB/s, one earlier copy measurement on a GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="4k", choices=sorted(W.WORKLOADS))
    ap.add_argument("--no-standard", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the continuous-batching serving mix")
    ap.add_argument("--no-raycast", action="store_true",
                    help="skip the ray-order 3DGS timing")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the 8K/100-view captured-graph batch section")
    ap.add_argument("--two-pass-emission", action="store_true",
                    help="DirectL keys through tile metadata and an emission kernel instead of "
                         "from the projection kernel")
    return ap.parse_args()


def workload_desc(wl: W.Workload) -> str:
    d, s = wl.display, wl.scene
    return (f"{wl.name}: {d.width}x{d.height} panel, {d.num_views} views, pitch {d.pitch_lx}, "
            f"slant {d.tan_slant:.4g}, P_w {d.p_w}; {s.n} Gaussians SH{s.sh_degree} "
            f"{s.layout}, {s.dtype} storage")


# --------------------------------------------------------------- ranks ----
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        import torch
        if not torch.cuda.is_available():
            backend = "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int, device=None) -> float:
    """Maximum of a float over ranks (the slowest rank sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int, device=None) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# -------------------------------------------------------------- clocks ----
class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(self.REASONS, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_id_for(device_index: int) -> str:
    import torch
    try:
        u = torch.cuda.get_device_properties(device_index).uuid
        return "GPU-" + str(u)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[device_index] if vis else str(device_index)


# --------------------------------------------------------- CPU oracle -----
def oracle_frame_estimate(wl: W.Workload, per_view: int, seed: int, n_rays_frame: int,
                          scene=None, tables=None) -> dict:
    """Time the FP64 oracle on two ray samples of a DirectL frame and
    extrapolate a whole frame: T = N_v * T_project + N_rays * T_ray.

    Sample A holds one ray per view, sample B ``per_view`` rays per view, all
    drawn from the oracle's own view map and repurposing table."""
    import oracle
    d = wl.display
    if tables is None:
        V = oracle.view_map(d)
        tables = (V, oracle.repurpose(d, V))
    V, src = tables
    if scene is None:
        scene = oracle.Scene(W.make_scene(wl.scene) if wl.scene.dtype == "f32" else
                             W.quantise_storage(W.make_scene(wl.scene), wl.scene.dtype))
    rng = np.random.default_rng(seed)
    sub = rng.integers(0, 3 * d.width * d.height, size=400 * d.num_views)
    rays = oracle.subpixel_rays(d, sub, V, src)
    picks_a, picks_b = [], []
    for v in range(d.num_views):
        idx = np.where(rays[:, 0] == v)[0]
        if idx.size == 0:
            continue
        picks_a.append(idx[:1])
        picks_b.append(idx[:per_view])
    ra = rays[np.concatenate(picks_a)]
    rb = rays[np.concatenate(picks_b)]
    L0 = W.light_field_centre(wl.camera_distance, 1.0)
    t0 = time.perf_counter()
    oracle.render_rays(scene, d, L0, ra)
    ta = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.render_rays(scene, d, L0, rb)
    tb = time.perf_counter() - t0
    nv = len(picks_a)
    t_ray = max((tb - ta) / max(rb.shape[0] - ra.shape[0], 1), 1e-9)
    t_proj = max((ta - ra.shape[0] * t_ray) / nv, 0.0)
    frame_s = d.num_views * t_proj + n_rays_frame * t_ray
    return {"frame_s": frame_s, "t_project_view_s": t_proj, "t_ray_s": t_ray,
            "sample_s": ta + tb, "rays_sampled": int(ra.shape[0] + rb.shape[0]),
            "threads": oracle.max_threads()}


def run_reference(args):
    """FP64 oracle arm: each step times a bounded ray sample and extrapolates."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    wl = W.WORKLOADS[args.workload]
    d = wl.display
    V = oracle.view_map(d)
    src = oracle.repurpose(d, V)
    _, rays = oracle.ray_table(d, V, src)
    n_rays = int(rays.shape[0])
    sc = W.make_scene(wl.scene)
    scene = oracle.Scene(W.quantise_storage(sc, wl.scene.dtype))
    frame_times, walls, last = [], [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        est = oracle_frame_estimate(wl, 4, 100 + i, n_rays, scene, (V, src))
        wall = time.perf_counter() - t0
        if i >= args.warmup:
            frame_times.append(est["frame_s"])
            walls.append(wall)
        last = est
    frame_ms = 1e3 * statistics.mean(frame_times)
    fps = 1e3 / frame_ms
    cores = int(last["threads"])
    # a step is one bounded ray sample (its wall time is ms_per_step); the
    # value is the frame rate extrapolated from the samples
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(walls), "extrapolated_ms_per_frame": frame_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": workload_desc(wl), "global_batch": 1, "parallelism": "none"},
            "subpixels_per_s": fps * 3 * d.width * d.height,
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": ("per step: one ray per view, then 4 rays per view "
                                        f"({last['rays_sampled']} rays, all 45 views projected "
                                        "twice); frame time extrapolated as N_v*T_project + "
                                        f"N_rays*T_ray with N_rays={n_rays}")},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- GPU arm ----
def timed_loop(fn, steps, world, device):
    import torch
    barrier(world)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    for i in range(steps):
        fn(i)
    end.record()
    torch.cuda.synchronize()
    barrier(world)
    return start.elapsed_time(end)


def per_frame(totals: dict, n: int) -> dict:
    keys = ("ms_project", "ms_scan", "ms_sync", "ms_emit", "ms_sort", "ms_ranges", "ms_composite",
            "ms_interweave", "ms_total")
    out = {k[3:]: totals[k] / max(n, 1) for k in keys}
    out["keys"] = totals["n_keys"] / max(n, 1)
    out["visible"] = totals["n_visible"] / max(n, 1)
    out["pairs_evaluated"] = totals["pairs_evaluated"] / max(n, 1)
    out["pairs_blended"] = totals["pairs_blended"] / max(n, 1)
    out["reemitted_frames"] = int(totals.get("reemitted", 0))  # keys emitted a second time
    out["dropped_frames"] = int(totals.get("status", 0))
    return out


def load_traffic(kernel: str, workload: str, source_file: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(f"{kernel}@{workload}")
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    h = hashlib.sha256(open(source_file, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    return rec.get("dram_bytes_per_launch")


def run_graph_batched(device: int, steps: int, two_pass: bool = False) -> dict:
    """8K panel, 100 views, 3M Gaussians (BF16): tile shape picked by the
    autotuner, then one frame per step from a captured CUDA graph of the
    frame batch (no host synchronisation inside a frame)."""
    import torch

    from paper_2407_14053_gb300 import Renderer
    wl = W.WORKLOADS["8k"]
    r = Renderer(device)
    if two_pass:
        r.set_key_emission("two_pass")
    try:
        t0 = time.perf_counter()
        scene = W.make_scene(wl.scene)
        sid = r.load_gaussians(scene, wl.scene.dtype)
        del scene
        did = r.set_display(wl.display)
        setup_s = time.perf_counter() - t0
        poses = W.camera_path(200, wl.camera_distance, 10.0)
        cands = [(16, 16), (32, 16), (32, 32), (64, 32)]
        best, ms = r.autotune_tile(sid, did, poses[0], cands, reps=3)
        b = r.batch([(sid, did, best, poses[0])], margin=1.25)
        out = torch.empty((wl.display.height, wl.display.width, 3), dtype=torch.float32,
                          device=f"cuda:{device}")
        st = torch.cuda.Stream()
        b.assign(0, sid, did, out, tile=best)
        with torch.cuda.stream(st):
            b.capture()
            for i in range(3):
                b.set_pose(0, poses[i])
                b.launch()
            b.wait()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(steps):
                b.set_pose(0, poses[(7 * i) % 200])
                b.launch()
            e1.record()
            status = b.wait(raise_on_capacity=False)
        st.synchronize()
        graph_ms = e0.elapsed_time(e1) / steps
        # the same frames through dl_render_frame (host sync per frame)
        r.set_tile("directl", *best)
        torch.cuda.synchronize()
        e0.record()
        for i in range(steps):
            r.render(sid, did, poses[(7 * i) % 200], "directl", out)
        e1.record()
        torch.cuda.synchronize()
        direct_ms = e0.elapsed_time(e1) / steps
        n_rays, beta = r.display_info(did)
        bytes_, long_cap = b.info()
        b.close()
        return {"workload": workload_desc(wl), "tile_autotuned": list(best),
                "autotune_ms": {f"{c[0]}x{c[1]}": m for c, m in zip(cands, ms)},
                "frames_per_s": 1e3 / graph_ms, "ms_per_frame": graph_ms, "steps": steps,
                "subpixels_per_s": 1e3 / graph_ms * 3 * wl.display.width * wl.display.height,
                "render_frame_ms": direct_ms, "status": status, "batch_bytes": bytes_,
                "beta": beta, "n_rays": int(n_rays), "setup_s": setup_s,
                "note": "one slot, captured graph replayed with a new pose per step"}
    finally:
        r.close()
        torch.cuda.empty_cache()


def _time_batch(r, specs, steps: int, device: int):
    """Loads each (scene spec, display) of `specs`, then times one frame of
    each per step: the frames rendered together by one launch sequence (one
    persistent launch per compositing class over all their tile lists)
    replayed from a captured CUDA graph, against the same frames through one
    dl_render_frame call each."""
    import torch
    S, D, outs = [], [], []
    for spec, disp in specs:
        S.append(r.load_gaussians(W.make_scene(spec), spec.dtype))
        D.append(r.set_display(disp))
        outs.append(torch.empty((disp.height, disp.width, 3), dtype=torch.float32,
                                device=f"cuda:{device}"))
    n = len(specs)
    poses = W.camera_path(200, 4.0, 10.0)
    b = r.batch([(S[k], D[k], None, poses[0]) for k in range(n)], margin=1.25)
    st = torch.cuda.Stream()
    for k in range(n):
        b.assign(k, S[k], D[k], outs[k])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        b.capture()
        for i in range(3):
            for k in range(n):
                b.set_pose(k, poses[(i + 40 * k) % 200])
            b.launch()
        b.wait()
        e0.record()
        for i in range(steps):
            for k in range(n):
                b.set_pose(k, poses[(7 * i + 40 * k) % 200])
            b.launch()
        e1.record()
        status = b.wait(raise_on_capacity=False)
    st.synchronize()
    graph_ms = e0.elapsed_time(e1) / steps
    torch.cuda.synchronize()
    for i in range(2):
        for k in range(n):
            r.render(S[k], D[k], poses[(i + 40 * k) % 200], "directl", outs[k])
    torch.cuda.synchronize()
    e0.record()
    for i in range(steps):
        for k in range(n):
            r.render(S[k], D[k], poses[(7 * i + 40 * k) % 200], "directl", outs[k])
    e1.record()
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1) / steps
    bytes_, _ = b.info()
    b.close()
    return {"ms_per_launch": graph_ms, "frames_per_s": n * 1e3 / graph_ms,
            "render_frame_ms_for_all": single_ms, "speedup_over_render_frame": single_ms / graph_ms,
            "steps": steps, "status": status, "batch_bytes": bytes_}


def run_multislot(device: int, steps: int) -> dict:
    """Uneven frames in one batch: a 4K/45-view frame of 1M Gaussians (BF16),
    a 1080p/45-view frame of 200k (FP32) and a 4K/60-view frame of 300k
    (FP16); and sixteen small frames (240x135 and 480x270 panels, 45 views,
    four scenes of 5k-40k Gaussians), where one launch per class in place of
    sixteen frames' launches is what batching saves."""
    import torch

    from paper_2407_14053_gb300 import Renderer
    p4k, p1080 = W.WORKLOADS["4k"].display, W.WORKLOADS["1080p"].display
    large = [(W.WORKLOADS["4k"].scene, p4k),
             (W.WORKLOADS["1080p"].scene, p1080),
             (W.SceneSpec(300_000, 3, "clustered", "f16", seed=5), p4k.replace(num_views=60))]
    tiny = W.WORKLOADS["tiny"].display
    small_disp = [tiny, tiny.replace(width=480, height=270)]
    small = [(W.SceneSpec(n, 3, "clustered", "f16", seed=60 + k), small_disp[k % 2])
             for k, n in enumerate([5_000, 10_000, 20_000, 40_000] * 4)]
    out = {}
    for name, specs in (("large", large), ("small", small)):
        r = Renderer(device)
        try:
            out[name] = _time_batch(r, specs, steps, device)
        finally:
            r.close()
            torch.cuda.empty_cache()
    res = out["large"]
    res.update({"frames": ["4k/45 views, 1M Gaussians bf16", "1080p/45 views, 200k f32",
                           "4k/60 views, 300k f16"],
                "render_frame_ms_for_the_three": res.pop("render_frame_ms_for_all"),
                "note": "three uneven frames per launch, captured graph replayed with new poses"})
    sm = out["small"]
    sm.update({"frames": "16: 240x135 and 480x270 panels, 45 views, scenes of 5k, 10k, 20k, 40k "
                         "Gaussians (SH3, f16)",
               "note": "sixteen small frames per launch, captured graph replayed with new poses"})
    res["small_frames"] = sm
    return res


def run_serving(device: int, n_requests: int = 256, n_scenes: int = 8, util: float = 0.7,
                seed: int = 0) -> dict:
    """Serving mix: Poisson arrivals, scenes of 100k-3M Gaussians
    (log-uniform, SH 3, FP16 storage), displays 1080p/45, 4K/45, 4K/60, head
    yaw U[-5, 5] degrees, 150 GB HBM budget.  The arrival rate is `util`
    times the service rate measured on a burst of the same mix."""
    import torch

    from paper_2407_14053_gb300 import Renderer
    from paper_2407_14053_gb300.serving import Request, Server, poisson_arrivals
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    sizes = np.exp(rng.uniform(np.log(1e5), np.log(3e6), size=n_scenes)).astype(int)
    sizes[0] = 3_000_000  # the slot-sizing scene: the largest of the mix
    scenes = {f"s{i}": (W.make_scene(W.SceneSpec(int(n), 3, "clustered", "f16", seed=50 + i)), "f16")
              for i, n in enumerate(sizes)}
    p1080, p4k = W.WORKLOADS["1080p"].display, W.WORKLOADS["4k"].display
    displays = {"1080p45": p1080, "4k45": p4k, "4k60": p4k.replace(num_views=60)}
    gen_s = time.perf_counter() - t0
    r = Renderer(device)
    try:
        L0 = W.light_field_centre(4.0, 0.0)
        plans = [("s0", "4k60"), ("s0", "4k60"), ("s0", "1080p45"), ("s0", "1080p45")]
        keep = set(range(1000, 1000 + n_requests, 32))  # a seeded sample re-rendered alone below
        srv = Server(r, scenes, displays, plans, L0, lanes=2, hbm_budget=150e9, margin=1.3,
                     keep_outputs=keep)

        def mix(n, arrivals, base):
            keys, dkeys = sorted(scenes), sorted(displays)
            return [Request(base + i, keys[rng.integers(len(keys))], dkeys[rng.integers(3)],
                            W.light_field_centre(4.0, float(rng.uniform(-5, 5))), float(a))
                    for i, a in enumerate(arrivals)]

        # the first burst loads scenes and displays and builds their tables
        # (its rate varies with which of them it meets first); the service
        # rate is taken from a second burst of the same mix, all resident
        cold = srv.run(mix(32, np.zeros(32), 0))
        burst = srv.run(mix(32, np.zeros(32), 100))
        rate = util * burst["frames_per_s"]
        reqs = mix(n_requests, poisson_arrivals(n_requests, rate, seed + 1), 1000)
        summary = srv.run(reqs)
        # served frames against the same frames rendered alone
        same = compared = 0
        for q in reqs:
            ks, kd = ("scene", q.scene), ("display", q.display)
            if q.rid not in keep or q.out is None or ks not in srv.cache.items or \
                    kd not in srv.cache.items:
                continue  # (a scene evicted since cannot be re-rendered here)
            alone = torch.empty_like(q.out)
            r.render(srv.cache.handle(ks), srv.cache.handle(kd), q.L0, "directl", alone)
            torch.cuda.synchronize()
            compared += 1
            same += int(torch.equal(alone, q.out))
        summary["alone_vs_mix"] = {"compared": compared, "bit_equal": same}
        summary.update({"arrival_rate_per_s": rate, "burst_frames_per_s": burst["frames_per_s"],
                        "cold_burst_frames_per_s": cold["frames_per_s"],
                        "target_utilisation": util, "hbm_budget_gb": 150.0,
                        "hbm_reserved_gb": srv.cache.reserved / 1e9,
                        "hbm_used_gb": srv.cache.used / 1e9, "scene_loads": srv.cache.loads,
                        "evictions": srv.cache.evictions, "scene_sizes": [int(x) for x in sizes],
                        "lanes": 2, "slots_per_lane": len(plans), "scene_gen_s": gen_s,
                        "mix": "scenes log-uniform 100k-3M (SH3, FP16), displays 1080p/45, "
                               "4K/45, 4K/60 uniform, yaw U[-5,5] deg, Poisson arrivals"})
        srv.close()
        return summary
    finally:
        r.close()
        torch.cuda.empty_cache()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    from paper_2407_14053_gb300 import Renderer

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2407_14053_gb300 import _binding as B
    alu_peaks = B.dl_measure_peaks(local)  # FP32 and ex2 rates for the roofline
    wl = W.WORKLOADS[args.workload]
    d = wl.display
    scene = W.make_scene(wl.scene)
    r = Renderer(local)
    if args.two_pass_emission:
        r.set_key_emission("two_pass")
    sid = r.load_gaussians(scene, wl.scene.dtype)
    t0 = time.perf_counter()
    did = r.set_display(d)
    offline_s = time.perf_counter() - t0
    n_rays, beta = r.display_info(did)
    poses = W.camera_path(200, wl.camera_distance, 10.0)
    out = torch.empty((d.height, d.width, 3), dtype=torch.float32, device=dev)
    subpix = 3 * d.width * d.height

    # ---- DirectL frames ----
    for i in range(args.warmup):
        r.render(sid, did, poses[i % 200], "directl", out)
    r.enable_stage_timing(True, count_pairs=False)  # stage events only
    torch.cuda.synchronize()
    r.stage_totals()
    sampler = ClockSampler(gpu_id_for(local)).start() if rank == 0 else None
    ms = timed_loop(lambda i: r.render(sid, did, poses[i % 200], "directl", out), args.steps, world,
                    dev)
    clocks = sampler.stop() if sampler else None
    tot, nf = r.stage_totals()
    dl_stages = per_frame(tot, nf)
    launches = int(tot["n_launches"])
    # pair counts of the same poses (counting kernels, untimed)
    r.enable_stage_timing(True, count_pairs=True)
    for i in range(args.steps):
        r.render(sid, did, poses[i % 200], "directl", out)
    tot_c, nf_c = r.stage_totals()
    cnt = per_frame(tot_c, nf_c)
    dl_stages["pairs_evaluated"], dl_stages["pairs_blended"] = cnt["pairs_evaluated"], cnt["pairs_blended"]
    r.enable_stage_timing(True, count_pairs=False)
    ms_max = reduce_max(ms, world, dev)
    frames_total = reduce_sum(args.steps, world, dev)
    fps = frames_total / (ms_max / 1e3)

    # ---- standard paradigm ----
    std = None
    if not args.no_standard:
        k_std = max(3, args.steps // 2)
        for i in range(2):
            r.render(sid, did, poses[i % 200], "standard", out)
        torch.cuda.synchronize()
        r.stage_totals()
        ms_s = timed_loop(lambda i: r.render(sid, did, poses[(7 * i) % 200], "standard", out), k_std,
                          world, dev)
        tot_s, nf_s = r.stage_totals()
        ms_s = reduce_max(ms_s, world, dev)
        fps_s = reduce_sum(k_std, world, dev) / (ms_s / 1e3)
        std_stages = per_frame(tot_s, nf_s)
        # pair counts of two of the same poses (counting kernels, untimed)
        r.enable_stage_timing(True, count_pairs=True)
        for i in range(2):
            r.render(sid, did, poses[(7 * i) % 200], "standard", out)
        cnt_s = per_frame(*r.stage_totals())
        std_stages["pairs_evaluated"] = cnt_s["pairs_evaluated"]
        std_stages["pairs_blended"] = cnt_s["pairs_blended"]
        r.enable_stage_timing(True, count_pairs=False)
        std = {"frames_per_s": fps_s, "subpixels_per_s": fps_s * subpix, "ms_per_frame": ms_s / k_std,
               "steps": k_std, "stages_ms": std_stages,
               "speedup_directl_over_standard": fps / fps_s}
        # the paper's LR / MR configurations of the standard paradigm (views
        # rendered smaller, upsampled while interweaving); 4K panel sizes
        # from its display table, other panels scaled by the same factors
        lowres = {}
        for name, frac in (("lr", 800 / 3840), ("mr", 1920 / 3840)):
            vw, vh = max(1, round(d.width * frac)), max(1, round(d.height * frac))
            r.set_standard_view_size(vw, vh)
            for i in range(2):
                r.render(sid, did, poses[i % 200], "standard", out)
            ms_l = timed_loop(lambda i: r.render(sid, did, poses[(7 * i) % 200], "standard", out),
                              k_std, world, dev)
            ms_l = reduce_max(ms_l, world, dev)
            fps_l = reduce_sum(k_std, world, dev) / (ms_l / 1e3)
            lowres[name] = {"view": [vw, vh], "frames_per_s": fps_l, "ms_per_frame": ms_l / k_std,
                            "speedup_directl_over": fps / fps_l}
        r.set_standard_view_size(0, 0)
        std["lowres"] = lowres
        # the paper's "HR w SR": views at panel resolution, each subpixel read
        # at its repurposed source pixel (DirectL's image, computed the
        # standard way)
        for i in range(2):
            r.render(sid, did, poses[i % 200], "standard_sr", out)
        ms_sr = timed_loop(lambda i: r.render(sid, did, poses[(7 * i) % 200], "standard_sr", out),
                           k_std, world, dev)
        ms_sr = reduce_max(ms_sr, world, dev)
        fps_sr = reduce_sum(k_std, world, dev) / (ms_sr / 1e3)
        std["hr_with_repurposing"] = {"frames_per_s": fps_sr, "ms_per_frame": ms_sr / k_std,
                                      "speedup_directl_over": fps / fps_sr}
    r.enable_stage_timing(False)

    # ---- the paper's ray-order 3DGS (Alg. 3) on the same rays ----
    raycast = None
    if not args.no_raycast:
        r.render(sid, did, poses[0], "raycast", out)  # builds the scene's tree
        k_rc = 3
        ms_rc = timed_loop(lambda i: r.render(sid, did, poses[(11 * i) % 200], "raycast", out), k_rc,
                           world, dev)
        ms_rc = reduce_max(ms_rc, world, dev)
        fps_rc = reduce_sum(k_rc, world, dev) / (ms_rc / 1e3)
        raycast = {"frames_per_s": fps_rc, "ms_per_frame": ms_rc / k_rc, "heap_capacity": 128,
                   "steps": k_rc, "speedup_directl_over": fps / fps_rc,
                   "note": "one thread per ray (rays grouped by view and tile), 8-wide SAH tree "
                           "over the Morton-ordered scene"}

    # ---- end to end through the C ABI with host (pinned) frames ----
    # value: frames delivered to host memory by dl_render_frame_async_host,
    # each frame's copy (on a second stream) overlapping the next frame;
    # sync_frames_per_s: dl_render_frame with a host frame, each call
    # returning once its frame is in host memory.  Both timed regions end
    # after the last frame has reached the host.
    e2e = None
    if not args.no_e2e:
        hosts = [torch.empty((d.height, d.width, 3), dtype=torch.float32).pin_memory()
                 for _ in range(2)]
        copy_stream = torch.cuda.Stream()

        def wall_of(step):
            for i in range(2):
                step(i)
            copy_stream.synchronize()
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(args.steps):
                step(i)
            copy_stream.synchronize()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            barrier(world)
            return reduce_max(wall, world, dev)

        wall_sync = wall_of(lambda i: r.render_to_host(sid, did, poses[i % 200], hosts[0], "directl"))
        wall = wall_of(lambda i: r.render_to_host_async(sid, did, poses[i % 200], hosts[i % 2],
                                                        copy_stream, "directl"))
        cam_bytes = 15 * 4 * 128 * math.ceil(d.num_views / 128)
        frames = reduce_sum(args.steps, world, dev)
        e2e = {"value": frames / wall, "unit": "frames/s",
               "h2d_bytes_per_step": cam_bytes, "d2h_bytes_per_step": 12 * d.width * d.height,
               "sync_frames_per_s": frames / wall_sync,
               "api": "dl_render_frame_async_host (copy of frame i on a second stream overlaps "
                      "frame i+1); sync_frames_per_s: dl_render_frame into host memory"}

    # ---- roofline of the compositing stage ----
    # The stage is the persistent warp-per-tile kernel's two classes (lists
    # of <= 512 and <= 1024 keys; longer lists would add the block class),
    # timed with CUDA events on the launching stream around the launches.
    src_file = os.path.join(ROOT, "paper_2407_14053_gb300", "csrc", "composite.cu")
    kname = "composite_rays_warp_kernel"
    hbm_gbs, hbm_source = measured_hbm_gbs()
    roofline = {"kernel": kname + " (512- and 1024-key classes: the compositing stage)",
                **compositing_roofline(dl_stages["composite"], dl_stages["keys"], n_rays,
                                       dl_stages["pairs_evaluated"], dl_stages["pairs_blended"],
                                       hbm_gbs, hbm_source, alu_peaks),
                "traffic": load_traffic(kname, args.workload, src_file)}

    # ---- rooflines of the other stages (HBM-bound; per frame) ----
    ne = d.num_views * wl.scene.n
    # the library's default emits the keys from the projection for scenes of
    # 131,072 Gaussians or more
    if args.two_pass_emission or wl.scene.n < 131072:
        stages_roof = {
            "project": stage_roofline(
                "project_kernel (with the camera upload and counter resets before it)",
                dl_stages["project"],
                wl.scene.n * attribute_bytes(wl.scene) + 16 * ne +
                RECORD_BYTES * dl_stages["visible"],
                f"{attribute_bytes(wl.scene)} B of attributes read once per Gaussian, 16 B tile "
                f"metadata written per (view, Gaussian), {RECORD_BYTES} B record written per "
                "visible (view, Gaussian)", hbm_gbs, hbm_source),
            "emit": stage_roofline(
                "emit_binned_kernel", dl_stages["emit"], 16 * ne + 8 * dl_stages["keys"],
                "16 B tile metadata read per (view, Gaussian), 8 B key written per key",
                hbm_gbs, hbm_source),
        }
    else:
        stages_roof = {
            "project": stage_roofline(
                "project_direct_kernel (projection emitting the tile keys; with the camera "
                "upload and the cursor copy before it)",
                dl_stages["project"],
                wl.scene.n * attribute_bytes(wl.scene) + RECORD_BYTES * dl_stages["visible"] +
                KEY_BYTES * dl_stages["keys"],
                f"{attribute_bytes(wl.scene)} B of attributes read once per Gaussian, "
                f"{RECORD_BYTES} B record written per visible (view, Gaussian), {KEY_BYTES} B "
                "key written per key", hbm_gbs, hbm_source),
        }
    if std is not None:
        ss = std["stages_ms"]
        pix = d.num_views * d.width * d.height
        stages_roof["standard_composite"] = {
            "kernel": "composite_full_binned_kernel (every pixel of every view into M_m)",
            **compositing_roofline(ss["composite"], ss["keys"], pix, ss["pairs_evaluated"],
                                   ss["pairs_blended"], hbm_gbs, hbm_source, alu_peaks)}
        stages_roof["standard_interweave"] = stage_roofline(
            "interweave_kernel", ss["interweave"], subpix * (2 + 4 + 4),
            "2 B view index read, 4 B gathered from M_m and 4 B written per subpixel",
            hbm_gbs, hbm_source)

    # ---- CPU oracle baseline (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est = oracle_frame_estimate(wl, 4, 7, int(n_rays))
        cpu = {"value": 1.0 / est["frame_s"], "unit": "frames/s", "cores": int(est["threads"]),
               "kind": "oracle", "cpu": cpu_model(),
               "sample": (f"one ray per view then 4 rays per view ({est['rays_sampled']} rays; "
                          f"every view's {wl.scene.n} Gaussians projected in FP64), frame time "
                          f"extrapolated as N_v*T_project + N_rays*T_ray, N_rays={n_rays}; "
                          f"{est['sample_s']:.1f} s of CPU time")}

    r.free_scene(sid)
    r.free_display(did)
    r.close()
    del out
    torch.cuda.empty_cache()

    graph = None
    if not args.no_graph and world == 1:
        graph = run_graph_batched(local, max(3, args.steps // 4), args.two_pass_emission)
        graph["uneven_multislot"] = run_multislot(local, max(3, args.steps // 2))
    serving = None
    if not args.no_serving and world == 1:
        serving = run_serving(local)

    if rank == 0:
        line = {
            "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scene and camera path)",
            "config": {"workload": workload_desc(wl), "global_batch": 1,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "no flush: each frame streams > 2 GB (inputs larger than L2)",
                       "storage": wl.scene.dtype, "beta": beta, "n_rays": int(n_rays)},
            "subpixels_per_s": fps * subpix,
            "standard_frames_per_s": std["frames_per_s"] if std else None,
            "speedup_vs_standard": fps / std["frames_per_s"] if std else None,
            "stages_ms": dl_stages,
            "offline_tables_s": offline_s,
            "standard": std,
            "raycast": raycast,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": e2e,
            "roofline": roofline,
            "roofline_stages": stages_roof,
            "alu_peaks_measured": alu_peaks,
            "cpu_baseline": cpu,
            "graph_batched": graph,
            "serving": serving,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
