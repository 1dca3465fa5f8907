"""The animated loop (the paper's interactive renderer, Sections 3.8-3.9): every
frame, the physics step moves the bodies on the device (rt_verlet_step), the new
positions are streamed into the scene table (rt_scene_update from device records),
the frame is rendered (rt_render) and, end to end, the pixels are read back to
host memory (the paper's streamOut).  No step leaves the GPU except the read-back.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rt, scenes


class Animation:
    """Bodies of `workload` (with previous centres `prev` [N, 3]) moving under Verlet
    physics, rendered every frame."""

    def __init__(self, workload: scenes.Workload, prev: np.ndarray, *, dt: float = 1.0 / 60.0,
                 gravity: float = 9.81, restitution: float = 0.7, substeps: int = 1, launch=None, stream=None,
                 device="cuda"):
        self.w = workload
        self.dt, self.gravity, self.restitution, self.substeps = dt, gravity, restitution, substeps
        self.launch = launch
        self.stream = stream
        sc = workload.scene
        self.ds = rt.DeviceScene(sc, stream=stream)
        self.spheres = torch.from_numpy(np.ascontiguousarray(sc.spheres, np.float32)).to(device)
        self.prev = torch.from_numpy(np.ascontiguousarray(prev, np.float32).reshape(-1, 3)).to(device)
        self.plane_rec = None if sc.plane is None else np.ascontiguousarray(sc.plane, np.float32)
        self.plane_t = None if sc.plane is None else torch.from_numpy(self.plane_rec).to(device)
        self.lights_t = torch.from_numpy(np.ascontiguousarray(sc.lights, np.float32)).to(device)
        self.out, self.pitch = rt.alloc_output(workload.params, device=device)
        self.ws = (rt.alloc_workspace(self.ds, workload.params, device=device)
                   if launch is not None and dict(launch).get("queued") else None)
        self.host = torch.empty(self.out.shape, dtype=self.out.dtype, pin_memory=True)
        self.frames = 0

    def step(self, readback: bool = True) -> torch.Tensor:
        """One frame: physics, scene update, render (and the pixels to pinned host
        memory when readback).  Returns the device framebuffer (or the host copy)."""
        rt.verlet_step(self.spheres, self.prev, self.plane_rec, dt=self.dt, gravity=self.gravity,
                       restitution=self.restitution, steps=self.substeps, stream=self.stream)
        self.ds.update(spheres=self.spheres, plane=self.plane_t, lights=self.lights_t, stream=self.stream)
        rt.render(self.ds, self.w.camera, self.w.params, out=self.out, pitch=self.pitch, launch=self.launch,
                  stream=self.stream, workspace=self.ws)
        self.frames += 1
        if readback:
            self.host.copy_(self.out, non_blocking=True)
            return self.host
        return self.out

    def positions(self) -> np.ndarray:
        torch.cuda.synchronize()
        return self.spheres[:, :3].cpu().numpy().copy()

    def close(self):
        self.ds.close()
