"""Splitting render work over several GPUs (one process per GPU).

Two ways to spread frames, neither with an exchange during rendering:
  * one frame over R ranks: contiguous row bands, each rank renders its band with
    rt_render_region (bit-identical to the full frame), then the bands are
    gathered (torch.distributed all_gather);
  * many frames over R ranks: longest-processing-time-first assignment of frames
    by estimated cost, each rank renders (or batches) its own frames.
The bench itself runs replicas (every rank renders its own frames).
"""
from __future__ import annotations

import heapq

import torch

from . import scenes


def row_bands(height: int, world: int) -> list[tuple[int, int]]:
    """Contiguous bands [y0, y1) covering 0..height, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(height, world)
    out, y = [], 0
    for r in range(world):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def frame_cost(scene: scenes.Scene, params: scenes.Params) -> float:
    """Relative cost of a frame: pixels x (bounces + 1) x (spheres + plane) x rays per hit."""
    sampled = sum(1 for l in scene.lights if float(l[4]) > 0 or float(l[5]) > 0)
    rays = 1 + scene.n_lights + sampled * (params.shadow_samples - 1)
    return float(params.width * params.height) * (1 + params.max_depth) * (scene.n_spheres + 2) * rays


def lpt(costs: list[float], world: int) -> list[list[int]]:
    """Assign item indices to `world` ranks, longest first, each to the least-loaded
    rank (ties: lowest rank).  Returns the item lists in assignment order."""
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return out


def render_band(dscene, camera, params: scenes.Params, y0: int, y1: int, *, launch=None, stream=None):
    """This rank's rows [y0, y1) of the frame (rt_render_region), as the same
    tensor layout rt.render returns for a full frame."""
    from . import rt
    return rt.render_region(dscene, camera, params, 0, y0, params.width, y1 - y0, launch=launch, stream=stream)


def gather_bands(local: torch.Tensor, bands: list[tuple[int, int]], group=None) -> torch.Tensor:
    """All-gather row bands (padded to the tallest band) and stitch the frame."""
    import torch.distributed as dist
    world = len(bands)
    hmax = max(b - a for a, b in bands)
    pad = torch.zeros((hmax,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: b - a] for r, (a, b) in enumerate(bands)], 0)
