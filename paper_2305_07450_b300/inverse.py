"""Inverse rendering on top of the hand-written adjoint (not in the paper).

Recovers material and light parameters of a scene from a target image by Adam on
the L2 image loss: albedo, specular coefficient and reflectivity of every sphere
and of the plane, light positions and intensities.  Geometry (sphere centres and
radii) is held at its initial value unless `optimize_centres` is set.  Every
render and gradient runs in the library's kernels; the loop (InverseLoop) keeps
parameters, Adam state and loss history on the device and replays one captured
CUDA graph per step.  RenderFn (rt.py) is the autograd route to the same
adjoint for use inside other PyTorch code (SceneParams / render_image).
Checkpoints ({parameters, Adam state, step, loss history}) are saved with
torch.save every `checkpoint_every` steps and resumed from when present.
"""
from __future__ import annotations

import os

import numpy as np
import torch

from . import rt, scenes


class SceneParams(torch.nn.Module):
    def __init__(self, scene: scenes.Scene, optimize_centres: bool = False, device="cuda"):
        super().__init__()
        sph = torch.tensor(scene.spheres, dtype=torch.float32, device=device)
        self.register_buffer("centre0", sph[:, 0:3].clone())
        self.register_buffer("radius", sph[:, 3:4].clone())
        self.register_buffer("spec_exp", sph[:, 8:9].clone())
        self.centre = torch.nn.Parameter(sph[:, 0:3].clone(), requires_grad=optimize_centres)
        self.albedo = torch.nn.Parameter(sph[:, 4:7].clone())
        self.ks = torch.nn.Parameter(sph[:, 7:8].clone())
        self.refl = torch.nn.Parameter(sph[:, 9:10].clone())
        pl = torch.tensor(scene.plane, dtype=torch.float32, device=device)
        self.register_buffer("plane_fixed", pl.clone())
        self.plane_albedo = torch.nn.Parameter(pl[4:7].clone())
        self.plane_ks = torch.nn.Parameter(pl[7:8].clone())
        self.plane_refl = torch.nn.Parameter(pl[9:10].clone())
        lig = torch.tensor(scene.lights, dtype=torch.float32, device=device)
        self.register_buffer("light_fixed", lig.clone())
        self.light_pos = torch.nn.Parameter(lig[:, 0:3].clone())
        self.light_I = torch.nn.Parameter(lig[:, 3:4].clone())

    def records(self):
        sph = torch.cat([self.centre, self.radius, self.albedo, self.ks, self.spec_exp, self.refl], 1)
        pl = torch.cat([self.plane_fixed[0:4], self.plane_albedo, self.plane_ks, self.plane_fixed[8:9],
                        self.plane_refl])
        lig = torch.cat([self.light_pos, self.light_I, self.light_fixed[:, 4:]], 1)
        return sph.contiguous(), pl.contiguous(), lig.contiguous()

    @torch.no_grad()
    def clamp_(self):
        self.albedo.clamp_(0.0, 1.0)
        self.ks.clamp_(0.0, 1.0)
        self.refl.clamp_(0.0, 0.5)
        self.plane_albedo.clamp_(0.0, 1.0)
        self.plane_ks.clamp_(0.0, 1.0)
        self.plane_refl.clamp_(0.0, 0.5)
        self.light_I.clamp_(0.05, 2.0)

    def material_vector(self) -> torch.Tensor:
        return torch.cat([self.albedo.flatten(), self.ks.flatten(), self.refl.flatten(), self.plane_albedo,
                          self.plane_ks, self.plane_refl]).detach()

    def light_vector(self) -> torch.Tensor:
        return torch.cat([self.light_pos.flatten(), self.light_I.flatten()]).detach()


def render_image(params: SceneParams, dscene, camera, rp: scenes.Params) -> torch.Tensor:
    sph, pl, lig = params.records()
    return rt.RenderFn.apply(sph, pl, lig, dscene, camera, rp)


class FlatParams:
    """The trainable parameters as one flat device vector theta, in the order
    [albedo N x 3 | k_s N | reflectivity N | plane albedo 3 | plane k_s | plane
    reflectivity | light positions L x 3 | light intensities L | (centres N x 3)],
    with the index maps that scatter theta into the scene records [spheres N x 10 |
    plane 10 | lights L x 8] and gather its gradient from the adjoint's packed
    gradient, and the clamp bounds of each entry."""

    def __init__(self, scene: scenes.Scene, optimize_centres: bool = False, device="cuda"):
        N, L = scene.n_spheres, scene.n_lights
        has_plane = scene.plane is not None
        self.N, self.L, self.has_plane = N, L, has_plane
        sph = np.asarray(scene.spheres, np.float32).reshape(N, 10)
        pl = np.asarray(scene.plane if has_plane else np.zeros(10), np.float32)
        lig = np.asarray(scene.lights, np.float32).reshape(L, 8)
        rec = np.concatenate([sph.ravel(), pl, lig.ravel()])
        i, p0, l0 = np.arange(N)[:, None], 10 * N, 10 * N + 10
        pos, lo, hi = [], [], []

        def add(idx, a, b):
            idx = np.asarray(idx, np.int64).ravel()
            pos.append(idx)
            lo.append(np.full(idx.size, a, np.float32))
            hi.append(np.full(idx.size, b, np.float32))
        add(10 * i + np.arange(4, 7), 0.0, 1.0)
        add(10 * i[:, 0] + 7, 0.0, 1.0)
        add(10 * i[:, 0] + 9, 0.0, 0.5)
        n_mat = 5 * N
        if has_plane:
            add(p0 + np.arange(4, 7), 0.0, 1.0)
            add([p0 + 7], 0.0, 1.0)
            add([p0 + 9], 0.0, 0.5)
            n_mat += 5
        add(l0 + 8 * np.arange(L)[:, None] + np.arange(3), -np.inf, np.inf)
        add(l0 + 8 * np.arange(L) + 3, 0.05, 2.0)
        if optimize_centres:
            add(10 * i + np.arange(3), -np.inf, np.inf)
        pos = np.concatenate(pos)
        self.n_mat, self.n_light = n_mat, 4 * L
        self.pos = torch.from_numpy(pos).to(device)
        self.lo = torch.from_numpy(np.concatenate(lo)).to(device)
        self.hi = torch.from_numpy(np.concatenate(hi)).to(device)
        self.records = torch.from_numpy(rec).to(device)        # fixed entries stay as given
        self.theta0 = self.records[self.pos].clone()
        # packed gradient index of each theta entry (rt.unpack_grad's map, restricted)
        self.grad_index = rt._unpack_index(N, L, device)[self.pos].clone()

    def views(self):
        """(spheres [N, 10], plane [10] or None, lights [L, 8]) views of the records."""
        N, L, r = self.N, self.L, self.records
        return (r[: 10 * N].view(N, 10), r[10 * N: 10 * N + 10] if self.has_plane else None,
                r[10 * N + 10:].view(L, 8))

    def material(self, theta: torch.Tensor) -> torch.Tensor:
        return theta[: self.n_mat]

    def lights(self, theta: torch.Tensor) -> torch.Tensor:
        return theta[self.n_mat: self.n_mat + self.n_light]


class InverseLoop:
    """The inverse-rendering step held on the device: parameters, Adam moments,
    step counter, loss history, packed gradient and every intermediate are device
    tensors, and one step is a fixed sequence of kernels -- scatter theta into the
    records, pack the scene (rt_scene_update from device records), forward render
    with hit record, loss and its image gradient, adjoint (rt_render_backward),
    gather of theta's gradient, Adam (Kingma and Ba, bias-corrected, beta = (0.9,
    0.999), eps = 1e-8), clamp to the valid ranges, loss into the history -- that
    is captured once into a CUDA graph and replayed, with no host synchronisation
    between steps.  graph=False runs the same sequence eagerly."""

    B1, B2, EPS = 0.9, 0.999, 1e-8

    def __init__(self, init: scenes.Workload, target: torch.Tensor, steps: int, lr: float,
                 optimize_centres: bool = False, graph: bool = True):
        rp = init.params
        assert rp.out_format == scenes.OUT_F32
        self.rp, self.camera, self.lr = rp, init.camera, float(lr)
        self.fp = FlatParams(init.scene, optimize_centres)
        self.ds = rt.DeviceScene(init.scene)
        dev = self.fp.records.device
        self.theta = self.fp.theta0.clone()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.t = torch.zeros((), dtype=torch.float32, device=dev)
        self.k = torch.zeros(1, dtype=torch.int64, device=dev)
        self.hist = torch.zeros(max(int(steps), 1), dtype=torch.float32, device=dev)
        self.tgt = target.contiguous()
        assert self.tgt.shape == (rp.height, rp.width, 4) and bool((self.tgt[..., 3] == 1.0).all())
        self.npx = float(rp.height * rp.width)
        self.img, self.pitch = rt.alloc_output(rp, device=dev)
        self.hr = torch.empty(rt.hitrec_bytes(self.ds, rp) // 4 + 1, dtype=torch.float32, device=dev)
        self.diff = torch.empty_like(self.img)
        self.dl = torch.empty_like(self.img)
        self.grad = torch.empty(rt.grad_count(self.ds), dtype=torch.float32, device=dev)
        self.ws = torch.empty(rt.backward_workspace_bytes(self.ds, rp) // 4 + 4, dtype=torch.float32, device=dev)
        self.graph = None
        if graph:
            self._capture()

    def _step(self):
        fp = self.fp
        fp.records.index_copy_(0, fp.pos, self.theta)
        sph, pl, lig = fp.views()
        self.ds.update(spheres=sph, plane=pl, lights=lig)
        rt.render(self.ds, self.camera, self.rp, out=self.img, pitch=self.pitch, hitrec=self.hr)
        # loss = sum over RGB of (img - target)^2 / pixels; alpha is 1 on both sides
        torch.sub(self.img, self.tgt, out=self.diff)
        loss = self.diff.square().sum() / self.npx
        torch.mul(self.diff, 2.0 / self.npx, out=self.dl)
        rt.render_backward(self.ds, self.camera, self.rp, self.dl, hitrec=self.hr, grad=self.grad,
                           workspace=self.ws)
        g = self.grad.index_select(0, fp.grad_index)
        self.t.add_(1.0)
        self.m.mul_(self.B1).add_(g, alpha=1.0 - self.B1)
        self.v.mul_(self.B2).addcmul_(g, g, value=1.0 - self.B2)
        bc1 = 1.0 - torch.pow(self.B1, self.t)
        bc2 = 1.0 - torch.pow(self.B2, self.t)
        upd = (self.m / bc1) / ((self.v / bc2).sqrt_().add_(self.EPS))
        self.theta.sub_(upd, alpha=self.lr)
        torch.clamp(self.theta, min=self.fp.lo, max=self.fp.hi, out=self.theta)
        self.hist.index_copy_(0, self.k, loss.view(1))
        self.k.add_(1)

    def _capture(self):
        state = self.state()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):     # warm-up: library and torch set-up outside the capture
                self._step()
        torch.cuda.current_stream().wait_stream(side)
        self.load_state(state)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._step()
        torch.cuda.synchronize()

    def run(self, n: int):
        for _ in range(n):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._step()

    def state(self) -> dict:
        return {"theta": self.theta.clone(), "m": self.m.clone(), "v": self.v.clone(), "t": self.t.clone(),
                "k": self.k.clone(), "hist": self.hist.clone()}

    def load_state(self, st: dict):
        for name in ("theta", "m", "v", "t", "k"):
            getattr(self, name).copy_(st[name])
        n = min(self.hist.numel(), st["hist"].numel())
        self.hist.zero_()
        self.hist[:n].copy_(st["hist"][:n])

    def close(self):
        self.graph = None
        self.ds.close()


def inverse_render(init: scenes.Workload, target: torch.Tensor, steps: int = 200, lr: float = 0.05,
                   optimize_centres: bool = False, checkpoint: str | None = None, checkpoint_every: int = 50,
                   truth: scenes.Scene | None = None, log=None, graph: bool = True) -> dict:
    """Adam on mean squared RGB error against `target` ([H, W, 4] float32 cuda),
    through InverseLoop (one CUDA graph replay per step).  The loss history stays
    on the device and is read once at the end; with `log`, every 20 steps.
    Checkpoints {theta, Adam moments, step, loss history} are saved every
    `checkpoint_every` steps and resumed from when present."""
    rp = init.params if init.params.out_format == scenes.OUT_F32 else \
        scenes.Params(**{**init.params.__dict__, "out_format": scenes.OUT_F32})
    w = scenes.Workload(init.name, init.scene, init.camera, rp)
    loop = InverseLoop(w, target, steps, lr, optimize_centres, graph=graph)
    start = 0
    if checkpoint and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location="cuda")
        loop.load_state(st)
        start = int(st["k"].item())
    step = start
    while step < steps:
        n = steps - step
        if checkpoint:
            n = min(n, checkpoint_every - step % checkpoint_every)
        if log:
            n = min(n, 20 - step % 20)
        loop.run(n)
        step += n
        if log:
            log(f"step {step - 1:4d} loss {float(loop.hist[step - 1]):.6e}")
        if checkpoint and step % checkpoint_every == 0:
            torch.save({k: v.cpu() for k, v in loop.state().items()}, checkpoint)
    torch.cuda.synchronize()
    history = loop.hist[:steps].tolist()
    out = {"history": history, "theta": loop.theta.clone(), "flat": loop.fp}
    if truth is not None:
        ft = FlatParams(truth, optimize_centres)
        rm = lambda a, b: float(torch.sqrt(torch.mean((a - b) ** 2)))  # noqa: E731
        fp = loop.fp
        out["material_rmse"] = (rm(fp.material(fp.theta0), fp.material(ft.theta0)),
                                rm(fp.material(loop.theta), fp.material(ft.theta0)))
        out["light_rmse"] = (rm(fp.lights(fp.theta0), fp.lights(ft.theta0)),
                             rm(fp.lights(loop.theta), fp.lights(ft.theta0)))
    loop.close()
    return out


def target_image(truth: scenes.Scene, w: scenes.Workload) -> torch.Tensor:
    ds = rt.DeviceScene(truth)
    rp = scenes.Params(**{**w.params.__dict__, "out_format": scenes.OUT_F32})
    img = rt.render(ds, w.camera, rp).clone()
    torch.cuda.synchronize()
    ds.close()
    return img


def loss_drop(history) -> float:
    return float(history[0] / max(history[-1], 1e-30)) if history else float("nan")


__all__ = ["SceneParams", "FlatParams", "InverseLoop", "inverse_render", "target_image", "render_image",
           "loss_drop", "np"]
