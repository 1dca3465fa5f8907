#!/usr/bin/env python
"""Benchmark of the per-pixel Whitted ray tracer (arXiv 2305.07450) on B300.

One step = one frame of the workload rendered by rt_render (all steps of the hot
path: staging, primary rays, closest hits, shading, shadow rays, reflection
bounces, framebuffer write) from a scene already resident in HBM.  Prints ONE
JSON line.  Default workload: 3840x2160 RGBA8, 256 spheres + plane, 3 point + 1
square area light (16 Philox samples), depth 8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own frames (independent replicas, no
collective on the data path): value = frames of all ranks / max-over-ranks time.
--impl reference times the FP64 oracle (the CPU baseline) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_07450_b300 import scenes as S  # noqa: E402

METRIC = "frames/s & Mrays/s at 720p/1080p/4K vs FP32 roofline; fwd+adjoint frames/s"
L2_FLUSH_BYTES = 256 << 20

# Algorithmic FP32 work per counted operation (minimal formulas, FMA = 2 flops;
# square roots, reciprocals and exp2/log2 are MUFU work and not counted).
FLOPS = {
    "closest_sphere_tests": 17,   # oc (3), b' = oc.d (5), c' = oc.oc - r^2 (7), disc (2)
    "closest_plane_tests": 12,    # general plane n.x + d = 0: d.n (5), o.n + d (6), t = num * rcp (1)
    "shadow_sphere_tests": 17,
    "shadow_plane_tests": 12,
    "primary_rays": 20,           # NDC (4), u R + v U + b F (12), normalise (4)
    "hits": 50,                   # point, normal, face-forward, offset, reflection, accumulate
    "light_evals": 16,            # L - p, |L - p|^2, normalise, n.l for every light at a hit
    "lit_lights": 21,             # Phong r, v.r, x^32, A and S updates
    "light_samples": 18,          # sample point and its unit direction
}


def flops_of(c: dict) -> float:
    return sum(FLOPS[k] * c[k] for k in FLOPS)


def rays_of(c: dict) -> float:
    return c["primary_rays"] + c["reflection_rays"] + c["shadow_rays"]


def workload(name: str) -> S.Workload:
    return S.WORKLOADS[name]()


# ----------------------------------------------------------------- CPU oracle
def oracle_sample(w: S.Workload, budget_s: float, threads: int | None = None):
    """Time the oracle (as it stands) on a lattice sample of the frame sized to
    roughly budget_s seconds; returns frames/s, Mrays/s, counters per pixel."""
    import oracle
    W, H = w.params.width, w.params.height
    stride = max(1, int(math.sqrt(W * H / 2048)))
    for _ in range(4):
        px = S.pixel_lattice(W, H, stride)
        t0 = time.perf_counter()
        r = oracle.trace(w.scene, w.camera, w.params, px, counters=True, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * budget_s or stride == 1:
            break
        stride = max(1, int(stride / math.sqrt(min(budget_s / max(dt, 1e-3), 400.0))))
    c = dict(r["counters"])
    per_px = {k: v / len(px) for k, v in c.items()}
    per_px["light_evals"] = per_px["hits"] * w.scene.n_lights
    frac = len(px) / float(W * H)
    return {
        "frames_per_s": frac / dt,
        "seconds": dt,
        "pixels": int(len(px)),
        "stride": stride,
        "threads": int(r["threads"]),
        "per_pixel": per_px,
        "mrays_per_s": rays_of(c) / dt / 1e6,
    }


def host_cpu_name() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- traffic record
# the sources the forward kernel is compiled from (its translation unit and the
# headers it includes); the batch and adjoint kernels' headers do not change it
FWD_SOURCES = ("rt_api.cu", "rt_device.cuh", "rt_trace.cuh", "rt_stage.cuh", "rt_bvh.cuh", "rt_errword.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_07450_b300", "csrc")
    for f in FWD_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name: str, kernel: str = "rt_fwd_kernel"):
    """DRAM bytes per frame of the forward kernel(s) from the committed ncu summary
    ("rt_fwd_kernel": the one-pass launch; "rt_render_ws": the sum over the first
    pass and the D queue passes of one frame), only if it was taken on the current
    kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for ln in open(path):
        f = ln.split()
        if len(f) >= 4 and not ln.startswith("#") and f[0] == kernel and f[1] == want \
                and f[2] == workload_name:
            return float(f[3])
    return None


# Executed FP32 work and hardware load of the forward kernels of one frame, from an ncu
# capture of the same sources (profiles/executed.txt); FP32 flops = fadd + fmul + 2 ffma
# + 2 fadd2 + 2 fmul2 + 4 ffma2 thread instructions (a packed f32x2 instruction does two
# operations per thread).
EXEC_FIELDS = ("fp32_flop", "fma_pipe_pct", "issue_active_pct", "no_instruction_per_issue", "lanes_per_inst",
               "dram_read_bytes", "dram_write_bytes", "ncu_ms")


def recorded_executed(workload_name: str, kernel: str):
    path = os.path.join(ROOT, "profiles", "executed.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for ln in open(path):
        f = ln.split("#", 1)[0].split()
        if len(f) == 3 + len(EXEC_FIELDS) and f[0] == kernel and f[1] == want \
                and f[2] == workload_name:
            return dict(zip(EXEC_FIELDS, map(float, f[3:])))
    return None


def ingest_ncu(csv_paths, kernel: str, workload_name: str) -> str:
    """One line of profiles/executed.txt from ncu --csv logs of one frame's launches
    (the metrics of EXEC_METRICS): sums over the launches, pipe and issue shares
    weighted by launch duration."""
    import csv
    rows = {}
    for p in csv_paths:
        with open(p) as f:
            lines = [ln for ln in f if ln.startswith('"')]
        for r in csv.DictReader(lines):
            key = (p, r["ID"])
            v = float(r["Metric Value"].replace(",", "") or 0)
            v *= UNIT_SCALE.get(r.get("Metric Unit", "").strip(), 1.0)
            rows.setdefault(key, {})[r["Metric Name"]] = v
    tot = dict.fromkeys(EXEC_FIELDS, 0.0)
    wsum = 0.0
    for m in rows.values():
        ms = m.get("gpu__time_duration.sum", 0.0) / 1e6
        th = lambda op: m.get(f"sm__sass_thread_inst_executed_op_{op}_pred_on.sum", 0.0)  # noqa: E731
        tot["fp32_flop"] += th("fadd") + th("fmul") + 2 * th("ffma") + 2 * th("fadd2") + 2 * th("fmul2") \
            + 4 * th("ffma2")
        tot["fma_pipe_pct"] += ms * m.get("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active", 0.0)
        tot["issue_active_pct"] += ms * m.get("smsp__issue_active.avg.pct_of_peak_sustained_active", 0.0)
        tot["no_instruction_per_issue"] += ms * m.get(
            "smsp__average_warps_issue_stalled_no_instruction_per_issue_active.ratio", 0.0)
        tot["lanes_per_inst"] += m.get("smsp__thread_inst_executed.sum", 0.0)
        tot["dram_read_bytes"] += m.get("dram__bytes_read.sum", 0.0)
        tot["dram_write_bytes"] += m.get("dram__bytes_write.sum", 0.0)
        tot["ncu_ms"] += ms
        wsum += m.get("smsp__inst_executed.sum", 0.0)
    for k in ("fma_pipe_pct", "issue_active_pct", "no_instruction_per_issue"):
        tot[k] /= max(tot["ncu_ms"], 1e-12)
    tot["lanes_per_inst"] /= max(wsum, 1.0)
    vals = " ".join(f"{tot[k]:.6g}" for k in EXEC_FIELDS)
    return f"{kernel} {kernel_source_hash()} {workload_name} {vals}  # {len(rows)} launches"


# ncu units to base units (bytes, nanoseconds); captures use --print-units base
UNIT_SCALE = {"Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "usecond": 1e3, "msecond": 1e6, "second": 1e9}

EXEC_METRICS = ",".join([
    "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
    *[f"sm__sass_thread_inst_executed_op_{op}_pred_on.sum" for op in ("fadd", "fmul", "ffma", "fadd2", "fmul2", "ffma2")],
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "smsp__average_warps_issue_stalled_no_instruction_per_issue_active.ratio",
    "smsp__thread_inst_executed.sum", "smsp__inst_executed.sum"])


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6400.0, "of fallback (6.4 TB/s)"


def workload_config(w: S.Workload, world: int) -> dict:
    """The `config` object of both arms' JSON lines: what the workload is."""
    return {"workload": w.name, "width": w.params.width, "height": w.params.height, "spheres": w.scene.n_spheres,
            "lights": w.scene.n_lights, "max_depth": w.params.max_depth,
            "shadow_samples": w.params.shadow_samples, "out": "rgba8" if w.params.out_format == 0 else "f32",
            "l2": f"flushed between timed frames ({L2_FLUSH_BYTES >> 20} MB write)",
            "parallelism": f"replicas x{world}"}


# ----------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2305_07450_b300 import rt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    w = workload(args.workload)
    W, H = w.params.width, w.params.height

    # CPU baseline first (host threads only; no process is forked after CUDA init)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, args.cpu_budget)

    ds = rt.DeviceScene(w.scene)
    out, pitch = rt.alloc_output(w.params, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    from paper_2305_07450_b300 import autotune
    launch = autotune.tune_render(ds, w.scene, w.camera, w.params, stream=stream)  # untimed; cached
    # rt_render_ws when the tuner chose the queued passes: its workspace is resident
    wsbuf = rt.alloc_workspace(ds, w.params, device=dev) if launch.get("queued") else None

    def step():
        rt.render(ds, w.camera, w.params, out=out, pitch=pitch, launch=launch, stream=stream, workspace=wsbuf)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    n0 = rt.launch_count()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        for a, b in evs:
            flush.zero_()                       # L2 flush between timed frames
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    launches = rt.launch_count() - n0
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = sum(ms) / len(ms)
    total_s = sum(ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    frames = world * args.steps
    fps = frames / total_s
    assert rt.device_errors() == 0

    # end to end through the public API with host buffers: every frame uploads the scene
    # records from host memory (pinned staging inside rt_scene_update), renders, and
    # reads the framebuffer back to pinned host memory.  Serial: one frame at a time.
    host_out = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        ds.update(w.scene, stream=stream)
        step()
        host_out.copy_(out, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e_serial_fps = 1e3 / (sum(e2e_ms) / len(e2e_ms)) * world
    # Pipelined (the headline e2e): two framebuffers; frame i's read-back runs on a copy
    # stream while frame i + 1 uploads and renders; one window over all the frames'
    # uploads, renders and read-backs.
    out2, _ = rt.alloc_output(w.params, device=dev)
    outs = (out, out2)
    hosts = (host_out, torch.empty(out.shape, dtype=out.dtype, pin_memory=True))
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def pipelined(n):
        for i in range(n):
            j = i & 1
            ds.update(w.scene, stream=stream)
            stream.wait_event(copied[j])  # this framebuffer's previous read-back is done
            rt.render(ds, w.camera, w.params, out=outs[j], pitch=pitch, launch=launch, stream=stream,
                      workspace=wsbuf)
            rendered[j].record(stream)
            copy_stream.wait_event(rendered[j])
            with torch.cuda.stream(copy_stream):
                hosts[j].copy_(outs[j], non_blocking=True)
            copied[j].record(copy_stream)
        return copied[(n - 1) & 1]

    pipelined(args.warmup)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    end = pipelined(args.steps)
    end.synchronize()
    e2e_fps = args.steps / (t0.elapsed_time(end) / 1e3) * world

    rec = None
    if rank == 0:
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        clocks = clk.summary()
        rec = {
            "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded scene (PCG64), no dataset",
            "config": dict(workload_config(w, world), launch=dict(launch, chosen_by="autotune")),
            "clocks": clocks,
            "gpu_launches": int(launches),
        }
        per_px = cpu["per_pixel"] if cpu else None
        if per_px:
            flops_frame = flops_of(per_px) * W * H
            rays_frame = rays_of(per_px) * W * H
            achieved = flops_frame / (ms_step / 1e3) / 1e12
            peak_max = sm_count * 128 * 2 * 2032e6 / 1e12
            rec["mrays_per_s"] = rays_frame * fps / 1e6
            kset = "rt_render_ws" if wsbuf is not None else "rt_fwd_kernel"
            rec["roofline"] = {
                "bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s",
                "frac": achieved / peak_max,
                "frac_basis": "algorithmic (the brute-force method's FP32 work per frame / frame time / peak)",
                "algorithmic_frac": achieved / peak_max,
                "traffic": recorded_traffic(w.name, kset),
                "kernel": ("rt_fwd_p0_kernel + rt_fwd_queue_kernel x D (rt_render_ws: one frame = 1 + D launches, "
                           "timed together)" if wsbuf is not None else "rt_fwd_kernel"),
                "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 x 2032 MHz (max SM clock)",
                "frac_at_measured_clock": (achieved / (sm_count * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
                                           if clocks.get("sm_mhz") else None),
                "algorithmic_gflop_per_frame": flops_frame / 1e9,
                "work_basis": f"oracle counters on a {cpu['pixels']}-pixel lattice (stride {cpu['stride']}) x W*H",
                "note": ("algorithmic work = the brute-force method's sphere tests (17 flop each, up to the first "
                         "blocker) as the oracle counts them; the kernels prove most of them unnecessary (line "
                         "filter, cone tests; bit-identical verdicts) and skip them, so frac can exceed 1; "
                         "executed_frac is the FP32 work the kernels do execute (ncu instruction counts of the "
                         "same sources) per frame time, against the same peak"),
            }
            ex = recorded_executed(w.name, kset)
            fb_bytes = out.numel() * out.element_size()
            hbm = measured_hbm_gbs()
            rec["roofline"].update({
                "executed_frac": (ex["fp32_flop"] / (ms_step / 1e3) / 1e12 / peak_max) if ex else None,
                "executed_tflops": (ex["fp32_flop"] / (ms_step / 1e3) / 1e12) if ex else None,
                "executed_gflop_per_frame": ex["fp32_flop"] / 1e9 if ex else None,
                "fma_pipe_busy_pct": ex["fma_pipe_pct"] if ex else None,
                "issue_active_pct": ex["issue_active_pct"] if ex else None,
                "no_instruction_stalls_per_issue": ex["no_instruction_per_issue"] if ex else None,
                "warp_exec_eff": ex["lanes_per_inst"] / 32.0 if ex else None,
                "framebuffer_write_gbs": fb_bytes / (ms_step / 1e3) / 1e9,
                "framebuffer_write_frac_of_hbm": fb_bytes / (ms_step / 1e3) / 1e9 / hbm[0],
                "hbm_peak_gbs": hbm[0], "hbm_peak_basis": hbm[1],
                "executed_basis": ("ncu instruction counts of one frame's launches on the current kernel sources "
                                   "(profiles/executed.txt; FP32 flops = fadd + fmul + 2 ffma + 2 fadd2 + 2 fmul2 + "
                                   "4 ffma2 thread instructions), per CUDA-event frame time"
                                   if ex else "no ncu record for the current kernel sources"),
            })
        if cpu:
            rec["cpu_baseline"] = {"value": cpu["frames_per_s"], "unit": "frames/s", "cores": cpu["threads"],
                                   "kind": "oracle",
                                   "sample": f"{cpu['pixels']} pixels (lattice stride {cpu['stride']}) of the frame, "
                                             f"{cpu['seconds']:.1f} s, scaled to frames/s",
                                   "cpu": host_cpu_name(), "mrays_per_s": cpu["mrays_per_s"]}
        rec["e2e"] = {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": int(ds.nbytes),
                      "d2h_bytes_per_step": int(out.numel() * out.element_size()),
                      "mode": "pipelined: frame i's read-back overlaps frame i+1's upload and render (two "
                              "framebuffers, a copy stream); every frame's upload and read-back inside the window",
                      "serial_value": e2e_serial_fps}
    ds.close()
    if rank == 0 and not args.no_extras:
        rec["also"] = extras(args, dev, stream)
    if world > 1:
        dist.destroy_process_group()
    return rec


def _time_device(fn, stream, reps, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def extras(args, dev, stream):
    """Secondary measurements (not the headline value): the forward render at
    1280x720 and 1920x1080 (64 spheres, 2 lights, depth 4), and the 64-scene
    batch as one graph-captured persistent launch against 64 per-frame launches."""
    import torch
    from paper_2305_07450_b300 import autotune, rt
    out = {}
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm_count * 128 * 2 * 2032e6 / 1e12
    for name in ("720p", "1080p"):
        w = workload(name)
        ds = rt.DeviceScene(w.scene)
        o, pitch = rt.alloc_output(w.params, device=dev)
        launch = autotune.tune_render(ds, w.scene, w.camera, w.params, stream=stream)
        wsb = rt.alloc_workspace(ds, w.params, device=dev) if launch.get("queued") else None
        ms = _time_device(lambda: rt.render(ds, w.camera, w.params, out=o, pitch=pitch, launch=launch,
                                            stream=stream, workspace=wsb), stream, 20)
        rec = {"workload": w.name, "frames_per_s": 1e3 / ms, "ms_per_frame": ms, "launch": launch}
        # executed FP32 work of the same kernels (ncu record of the current sources)
        ex = recorded_executed(w.name, "rt_render_ws" if launch.get("queued") else "rt_fwd_kernel")
        if ex:
            rec.update({"executed_tflops": ex["fp32_flop"] / (ms / 1e3) / 1e12,
                        "executed_frac": ex["fp32_flop"] / (ms / 1e3) / 1e12 / peak,
                        "executed_gflop_per_frame": ex["fp32_flop"] / 1e9,
                        "fma_pipe_busy_pct": ex["fma_pipe_pct"], "issue_active_pct": ex["issue_active_pct"],
                        "warp_exec_eff": ex["lanes_per_inst"] / 32.0})
        if not args.no_cpu_baseline:
            # algorithmic work from the oracle's counters on a bounded lattice sample
            cs = oracle_sample(w, min(3.0, args.cpu_budget))
            px = w.params.width * w.params.height
            tf = flops_of(cs["per_pixel"]) * px / (ms / 1e3) / 1e12
            rec.update({"mrays_per_s": rays_of(cs["per_pixel"]) * px / (ms / 1e3) / 1e6, "alg_tflops": tf,
                        "frac_of_fp32_peak": tf / peak, "peak_tflops": peak,
                        "work_sample": f"{cs['pixels']} pixels (lattice stride {cs['stride']})"})
        out[name] = rec
        ds.close()
    ws = S.batch_scenes()
    dss = [rt.DeviceScene(w.scene) for w in ws]
    blaunch = autotune.tune_batch(dss, [w.scene for w in ws], [w.camera for w in ws], [w.params for w in ws],
                                  stream=stream)
    b = rt.Batch(dss, [w.camera for w in ws], [w.params for w in ws], launch=blaunch, stream=stream)
    ms_graph = _time_device(lambda: b.launch(stream), stream, 5)
    flaunch = [autotune.tune_render(d, w.scene, w.camera, w.params, stream=stream, reps=1) for w, d in zip(ws, dss)]
    fws = [rt.alloc_workspace(d, w.params) if fl.get("queued") else None for w, d, fl in zip(ws, dss, flaunch)]

    def seq():
        for w, d, o, pt, fl, wb in zip(ws, dss, b.outs, b.pitches, flaunch, fws):
            rt.render(d, w.camera, w.params, out=o, pitch=pt, launch=fl, stream=stream, workspace=wb)
    ms_seq = _time_device(seq, stream, 3)
    px = sum(w.params.width * w.params.height for w in ws)
    out["batch64"] = {"workload": "64 seeded scenes, 8-512 spheres, 1-4 lights, depth 1-6, 256^2..1080p, F32",
                      "pixels": px, "ms_graph_launch": ms_graph, "ms_64_rt_render": ms_seq,
                      "launch_batch": blaunch, "launch_per_frame": "autotuned per frame",
                      "frames_per_s_batched": 64e3 / ms_graph, "frames_per_s_per_frame_launches": 64e3 / ms_seq,
                      "speedup": ms_seq / ms_graph}
    b.close()
    for d in dss:
        d.close()
    out["bvh"] = bvh_extra(dev, stream)
    out["animated"] = animated_extra(dev, stream)
    out["fwd_adjoint"] = fwd_adjoint(dev, stream)
    out["paper_scene"] = paper_scene(dev, stream)
    return out


def animated_extra(dev, stream):
    """The animated loop (Sections 3.8-3.9, the paper's interactive setting: hard
    shadows, bounce limit 1, five spheres, a light, the plane, a sky panorama):
    every frame a Verlet step on the device, the scene update from device records,
    the render and the pixels read back to pinned host memory, the host waiting for
    each frame as a display loop does.  End-to-end frames/s by host clock over 120
    frames; the device time of one frame (physics + update + render) by events."""
    import torch
    from paper_2305_07450_b300 import animate
    res = {"note": "paper's 234/152/45 frames/s (RTX 2060, GUI, its own scene and sky) are context, not a target"}
    for W, H in ((1280, 720), (1920, 1080), (3840, 2160)):
        w, prev = S.animated_scene(W, H)
        an = animate.Animation(w, prev, stream=stream)
        for _ in range(5):
            an.step()
        torch.cuda.synchronize()
        n = 120
        t0 = time.perf_counter()
        for _ in range(n):
            an.step(readback=True)
            stream.synchronize()
        e2e = n / (time.perf_counter() - t0)
        ms_dev = _time_device(lambda: an.step(readback=False), stream, 60)
        res[f"{W}x{H}"] = {"workload": w.name, "frames_per_s_end_to_end": e2e, "ms_device_frame": ms_dev,
                           "d2h_bytes_per_frame": int(an.out.numel() * an.out.element_size()),
                           "launches_per_frame": 3}
        an.close()
    return res


def bvh_extra(dev, stream):
    """The sphere hierarchy (the paper's future work; not the headline, which is
    the paper's brute-force method): frames/s through it against brute force on
    the 4K workload, the 1080p area-light scene and a 4096-sphere scene, with the
    outputs compared bit for bit on the device."""
    import torch
    from paper_2305_07450_b300 import autotune, rt
    big = S.random_scene(41, 4096, 2, 12.0, area_lights=1)
    huge = S.random_scene(43, 8192, 2, 16.0, area_lights=1)
    cases = [workload("4k"), workload("4k_scene_1080p"),
             S.Workload("1920x1080_4096sph_2pt+area16_d4_rgba8", big, S.default_camera(12.0),
                        S._params(big, width=1920, height=1080, max_depth=4, shadow_samples=16, seed=41)),
             # beyond the brute force's cone pre-pass (tables of at most 4096 spheres)
             S.Workload("1280x720_8192sph_2pt+area16_d4_rgba8", huge, S.default_camera(16.0),
                        S._params(huge, width=1280, height=720, max_depth=4, shadow_samples=16, seed=43))]
    res = {}
    for w in cases:
        ds = rt.DeviceScene(w.scene)
        info = ds.build_bvh(stream=stream)
        o1, pitch = rt.alloc_output(w.params, device=dev)
        o2, _ = rt.alloc_output(w.params, device=dev)
        bf = autotune.tune_render(ds, w.scene, w.camera, w.params, stream=stream)
        wbf = rt.alloc_workspace(ds, w.params) if bf.get("queued") else None
        ms_bf = _time_device(lambda: rt.render(ds, w.camera, w.params, out=o1, pitch=pitch, launch=bf, stream=stream,
                                               workspace=wbf), stream, 5)
        best = None
        for cand in ({"block_x": 16, "block_y": 8}, {"block_x": 8, "block_y": 8}, {"block_x": 32, "block_y": 4},
                     {"block_x": 8, "block_y": 16}, {"block_x": 16, "block_y": 16}):
            cfg = dict(cand, accel=1, staging=1)
            ms = _time_device(lambda: rt.render(ds, w.camera, w.params, out=o2, pitch=pitch, launch=cfg,
                                                stream=stream), stream, 5)
            if best is None or ms < best[0]:
                best = (ms, cfg)
        torch.cuda.synchronize()
        same = bool(torch.equal(o1, o2))
        res[w.name] = {"spheres": w.scene.n_spheres, "hierarchy": info, "ms_brute_force": ms_bf,
                       "ms_bvh": best[0], "launch_bvh": best[1], "frames_per_s_brute_force": 1e3 / ms_bf,
                       "frames_per_s_bvh": 1e3 / best[0], "speedup": ms_bf / best[0], "bit_identical": same}
        ds.close()
    assert rt.device_errors() == 0
    return res


PAPER_FPS_RTX2060 = {"1280x720": 234, "1920x1080": 152, "3840x2160": 45}


def paper_scene(dev, stream):
    """The paper's benchmark-scene structure (one spherical light, one plane, five
    spheres; seeded, no sky): its real-time settings (hard shadows = 1 sample,
    bounce limit 1) and its render-only settings (200 sunflower samples, bounce
    limit 3) at 720p / 1080p / 4K, and the sweeps of its Section 4.3 (shadow
    samples at bounce 1; bounce limit at 200 samples), frames/s on this GPU."""
    from paper_2305_07450_b300 import rt

    def fps(w):
        ds = rt.DeviceScene(w.scene)
        o, pitch = rt.alloc_output(w.params, device=dev)
        ms = _time_device(lambda: rt.render(ds, w.camera, w.params, out=o, pitch=pitch, stream=stream), stream, 10)
        ds.close()
        return 1e3 / ms
    res = {"note": "paper's figures (RTX 2060, GUI, its own scene with HDR sky) are context, not a target",
           "paper_reported_fps_hard_b1": PAPER_FPS_RTX2060}
    for tag, samples, depth in (("hard_b1", 1, 1), ("soft200_b3", 200, 3)):
        res[tag] = {f"{W}x{H}": fps(S.paper_scene(W, H, samples, depth))
                    for W, H in ((1280, 720), (1920, 1080), (3840, 2160))}
    res["samples_sweep_1280x720_b1"] = {n: fps(S.paper_scene(1280, 720, n, 1)) for n in (1, 10, 50, 100, 200, 300, 500)}
    res["bounce_sweep_1280x720_s200"] = {d: fps(S.paper_scene(1280, 720, 200, d)) for d in range(0, 9)}
    return res


def fwd_adjoint(dev, stream):
    """512x512 differentiable workload: forward with hit record + adjoint
    (replay) per frame, against the plain forward; then the 200-step Adam
    inverse-rendering loop from the unperturbed parameters to a perturbed target."""
    import torch
    from paper_2305_07450_b300 import inverse, rt
    w = workload("diff512")
    p = w.params
    ds = rt.DeviceScene(w.scene)
    out, pitch = rt.alloc_output(p, device=dev)
    hr = torch.empty(rt.hitrec_bytes(ds, p) // 4 + 1, dtype=torch.float32, device=dev)
    dl = torch.randn((p.height, p.width, 4), dtype=torch.float32, device=dev,
                     generator=torch.Generator(dev).manual_seed(0))
    grad = torch.empty(rt.grad_count(ds), dtype=torch.float32, device=dev)
    wsb = torch.empty(1 << 20, dtype=torch.float32, device=dev)
    ms_fwd = _time_device(lambda: rt.render(ds, w.camera, p, out=out, pitch=pitch, stream=stream), stream, 20)

    def fwd_bwd():
        rt.render(ds, w.camera, p, out=out, pitch=pitch, hitrec=hr, stream=stream)
        rt.render_backward(ds, w.camera, p, dl, hitrec=hr, grad=grad, workspace=wsb, stream=stream)
    ms_fb = _time_device(fwd_bwd, stream, 20)
    ms_bwd_recompute = _time_device(
        lambda: rt.render_backward(ds, w.camera, p, dl, hitrec=None, grad=grad, workspace=wsb, stream=stream),
        stream, 10)
    ds.close()
    truth = S.perturbed_target(w)
    tgt = inverse.target_image(truth, w)
    # untimed: the first optimizer step of a process imports PyTorch modules lazily
    # (seconds on a cold box), which is not the loop's cost; with the truth, so that the
    # error measures at the end are warm as well
    inverse.inverse_render(w, tgt, steps=2, lr=0.05, truth=truth)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = inverse.inverse_render(w, tgt, steps=200, lr=0.05, truth=truth)
    torch.cuda.synchronize()
    h = res["history"]
    return {"workload": w.name, "ms_forward": ms_fwd, "ms_forward_hitrec_plus_adjoint": ms_fb,
            "ms_adjoint_recompute": ms_bwd_recompute, "frames_per_s_forward": 1e3 / ms_fwd,
            "frames_per_s_fwd_adjoint": 1e3 / ms_fb, "adjoint_over_forward": ms_fb / ms_fwd,
            "inverse_200_adam": {"lr": 0.05, "seconds": time.perf_counter() - t0, "loss_first": h[0],
                                 "loss_last": h[-1], "loss_drop": h[0] / h[-1],
                                 "material_rmse_before_after": res["material_rmse"],
                                 "light_rmse_before_after": res["light_rmse"]}}


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    w = workload(args.workload)
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        info = oracle_sample(w, args.ref_budget)
        if i >= args.warmup:
            vals.append(info["frames_per_s"])
    fps = statistics.mean(vals)
    return {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / fps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic: seeded scene (PCG64), no dataset",
        "config": workload_config(w, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": info["threads"], "kind": "oracle",
                         "sample": f"{info['pixels']} pixels (lattice stride {info['stride']}) per step, "
                                   f"scaled to frames/s", "cpu": host_cpu_name()},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def profile_render(args):
    """Only the render of the workload, warmup + steps frames, with the library's
    default launch (16x8 pixels, TMA staging): rt_render, or with --queued rt_render_ws
    (1 + D launches per frame): the program ncu captures for the forward kernels."""
    import torch
    from paper_2305_07450_b300 import rt
    w = workload(args.workload)
    ds = rt.DeviceScene(w.scene)
    out, pitch = rt.alloc_output(w.params)
    launch = {"accel": 1} if args.accel else None
    if args.accel:
        ds.build_bvh()
    if args.tuned:
        from paper_2305_07450_b300 import autotune
        launch = autotune.tune_render(ds, w.scene, w.camera, w.params)
    wsbuf = rt.alloc_workspace(ds, w.params) if (args.queued or (launch or {}).get("queued")) else None
    for _ in range(args.warmup + args.steps):
        rt.render(ds, w.camera, w.params, out=out, pitch=pitch, launch=launch, workspace=wsbuf)
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    print(json.dumps({"profile_render": w.name, "accel": bool(args.accel), "queued": wsbuf is not None,
                      "launch": launch,
                      "frames": args.warmup + args.steps}))


def profile_batch(args):
    import torch
    from paper_2305_07450_b300 import rt
    ws = S.batch_scenes()
    dss = [rt.DeviceScene(w.scene) for w in ws]
    b = rt.Batch(dss, [w.camera for w in ws], [w.params for w in ws])
    for _ in range(args.warmup + args.steps):
        b.launch()
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    print(json.dumps({"profile_batch": True, "launches": args.warmup + args.steps}))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(S.WORKLOADS), default="4k")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=8.0, help="seconds of oracle work per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 720p/1080p/batch measurements")
    ap.add_argument("--profile-render", action="store_true",
                    help="only render the workload (warmup + steps launches, default launch), for ncu")
    ap.add_argument("--accel", action="store_true", help="with --profile-render: through the sphere hierarchy")
    ap.add_argument("--queued", action="store_true", help="with --profile-render: rt_render_ws (queued passes)")
    ap.add_argument("--tuned", action="store_true",
                    help="with --profile-render: the autotuned launch the bench times (queued if it chose so)")
    ap.add_argument("--ingest-ncu", nargs="+", metavar="CSV",
                    help="print the profiles/executed.txt line of ncu --csv logs (EXEC_METRICS) of one frame")
    ap.add_argument("--kernel-set", default="rt_render_ws", help="with --ingest-ncu: the record's kernel column")
    ap.add_argument("--profile-batch", action="store_true",
                    help="only launch the 64-scene batch graph --warmup + --steps times (a profiling target)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.ingest_ncu:
        print(ingest_ncu(args.ingest_ncu, args.kernel_set, workload(args.workload).name))
        return None
    if args.profile_batch:
        return profile_batch(args)
    if args.profile_render:
        return profile_render(args)
    rec = run_reference(args) if args.impl == "reference" else run_ours(args)
    if rec is not None:
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
