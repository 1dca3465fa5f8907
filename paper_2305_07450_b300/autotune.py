"""Autotuner of the render kernels' launch shape (CTA pixel tile, staging mode,
one pass (rt_render) or queued passes (rt_render_ws)).

A launch configuration is measured, not guessed: every candidate CTA shape is
timed with CUDA events on the caller's stream (median of a few launches after a
warm-up) and the fastest is kept.  Results are cached per key
(GPU name, sphere-count bucket, lights, bounce limit, samples, resolution, output
format, shading model) in a JSON file: first the table shipped with the package
(``tuned.json``, measured on B300), then the user cache
(``$RT_AUTOTUNE_CACHE``, default ``~/.cache/paper_2305_07450_b300/autotune.json``).
Every candidate produces bit-identical images (the per-pixel computation does not
depend on the tile shape), so tuning never changes results.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import threading

import torch

from . import rt, scenes

PKG = os.path.dirname(os.path.abspath(__file__))
SHIPPED = os.path.join(PKG, "tuned.json")

# CTA pixel tiles (block_x, block_y): warps are 8x4 pixel patches
FWD_CANDIDATES = [(8, 4), (8, 8), (16, 4), (16, 8), (8, 16), (32, 4), (16, 16), (32, 8), (8, 32)]
BATCH_CANDIDATES = [(8, 4), (8, 8), (16, 4), (16, 8), (8, 16), (32, 4)]

_lock = threading.Lock()
_mem: dict[str, dict] = {}


def user_cache_path() -> str:
    return os.environ.get("RT_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2305_07450_b300", "autotune.json"))


def _bucket(n: int) -> int:
    b = 1
    while b < max(n, 1):
        b <<= 1
    return b


def gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"


def key_for(scene: scenes.Scene, params: scenes.Params, kind: str = "fwd") -> str:
    sampled = int(any(float(l[4]) > 0 or float(l[5]) > 0 for l in scene.lights))
    return "|".join(str(v) for v in (kind, gpu_name(), _bucket(scene.n_spheres), scene.n_lights, sampled,
                                     params.max_depth, params.shadow_samples if sampled else 1,
                                     params.width, params.height, params.out_format, params.shading_model))


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(key: str):
    with _lock:
        if key in _mem:
            return _mem[key]
        for path in (SHIPPED, user_cache_path()):
            table = _load(path)
            if key in table:
                _mem[key] = table[key]
                return table[key]
    return None


def _store(key: str, entry: dict):
    with _lock:
        _mem[key] = entry
        path = user_cache_path()
        table = _load(path)
        table[key] = entry
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass  # an unwritable cache only costs re-tuning


def _time(fn, stream, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def tune_render(dscene: rt.DeviceScene, scene: scenes.Scene, camera, params: scenes.Params, *, reps: int = 3,
                candidates=FWD_CANDIDATES, stream=None, force: bool = False, queued: bool = True) -> dict:
    """Best launch for one frame (measured, then cached): CTA tile and staging
    mode, through rt_render or (queued=True) also rt_render_ws -- the returned
    launch then holds "queued": 1, and the caller passes a workspace
    (rt.alloc_workspace) or lets rt.render allocate one."""
    key = key_for(scene, params, "fwd")
    hit = None if force else lookup(key)
    if hit is not None:
        return hit["launch"]
    stream = stream or torch.cuda.current_stream()
    out, pitch = rt.alloc_output(params)
    ws = rt.alloc_workspace(dscene, params) if queued else None
    results = {}
    for bx, by in candidates:
        # staging 1 / 2 through rt_render; 1 / 2 through rt_render_ws (queued, q = 1)
        for staging, q in ((1, 0), (2, 0)) + (((1, 1), (2, 1)) if queued else ()):
            launch = {"block_x": bx, "block_y": by, "staging": staging}
            results[(bx, by, staging, q)] = _time(
                lambda: rt.render(dscene, camera, params, out=out, pitch=pitch, launch=launch, stream=stream,
                                  workspace=ws if q else None),
                stream, reps)
    (bx, by, staging, q), ms = min(results.items(), key=lambda kv: kv[1])
    best = {"block_x": bx, "block_y": by, "staging": staging}
    if q:
        best["queued"] = 1
    entry = {"launch": best, "ms": ms,
             "candidates": {f"{a}x{b}/s{c}{'/q' if d else ''}": round(v, 4) for (a, b, c, d), v in results.items()}}
    _store(key, entry)
    return entry["launch"]


def tune_batch(dscenes, scene_list, cameras, params_list, *, reps: int = 3, candidates=BATCH_CANDIDATES,
               stream=None, force: bool = False) -> dict:
    """Best launch for a batch (the key covers every frame of the batch)."""
    sub = sorted(key_for(s, p, "b") for s, p in zip(scene_list, params_list))
    key = "batch|" + gpu_name() + "|" + hashlib.sha1("\n".join(sub).encode()).hexdigest()[:16]
    hit = None if force else lookup(key)
    if hit is not None:
        return hit["launch"]
    stream = stream or torch.cuda.current_stream()
    outs, pitches = rt.alloc_batch_outputs(params_list)
    results = {}
    for bx, by in candidates:
        launch = {"block_x": bx, "block_y": by}
        b = rt.Batch(dscenes, cameras, params_list, outs=outs, pitches=pitches, launch=launch, stream=stream)
        results[(bx, by)] = _time(lambda: b.launch(stream), stream, reps)
        b.close()
    (bx, by), ms = min(results.items(), key=lambda kv: kv[1])
    entry = {"launch": {"block_x": bx, "block_y": by}, "ms": ms,
             "candidates": {f"{a}x{b}": round(v, 4) for (a, b), v in results.items()}}
    _store(key, entry)
    return entry["launch"]


def write_table(path: str, reps: int = 7) -> dict:
    """Tune the standard workloads (forward at every workload, the 64-scene batch,
    the animated loop's frames) with `reps` timed launches per candidate and write
    the entries to `path`: the table shipped as tuned.json."""
    global _mem
    table = {}
    stream = torch.cuda.current_stream()
    names = ["256", "720p", "1080p", "4k", "4k_scene_1080p", "diff512"]
    works = [scenes.WORKLOADS[n]() for n in names]
    works += [scenes.paper_scene(W, H, s, d) for W, H in ((1280, 720), (1920, 1080), (3840, 2160))
              for s, d in ((1, 1), (200, 3))]
    works += [scenes.animated_scene(W, H)[0] for W, H in ((1280, 720), (1920, 1080), (3840, 2160))]
    for w in works:
        ds = rt.DeviceScene(w.scene)
        tune_render(ds, w.scene, w.camera, w.params, reps=reps, stream=stream, force=True)
        key = key_for(w.scene, w.params, "fwd")
        table[key] = dict(_mem[key], workload=w.name)
        ds.close()
    ws = scenes.batch_scenes()
    dss = [rt.DeviceScene(w.scene) for w in ws]
    tune_batch(dss, [w.scene for w in ws], [w.camera for w in ws], [w.params for w in ws], reps=reps,
               stream=stream, force=True)
    for k, v in _mem.items():
        if k.startswith("batch|"):
            table[k] = dict(v, workload="64-scene batch")
    for d in dss:
        d.close()
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="write the shipped launch table (run on the target GPU)")
    ap.add_argument("--out", default=SHIPPED)
    ap.add_argument("--reps", type=int, default=7)
    a = ap.parse_args()
    t = write_table(a.out, a.reps)
    print(json.dumps({k: v["launch"] for k, v in t.items()}, indent=1))
