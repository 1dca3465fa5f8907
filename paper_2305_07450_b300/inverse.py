"""Inverse rendering on top of the hand-written adjoint (not in the paper).

Recovers material and light parameters of a scene from a target image by Adam on
the L2 image loss: albedo, specular coefficient and reflectivity of every sphere
and of the plane, light positions and intensities.  Geometry (sphere centres and
radii) is held at its initial value unless `optimize_centres` is set.  Every
render and gradient runs in the library's kernels (RenderFn); the Python loop
only assembles parameter tensors, calls Adam and clamps to the valid ranges.
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


def inverse_render(init: scenes.Workload, target: torch.Tensor, steps: int = 200, lr: float = 0.05,
                   optimize_centres: bool = False, checkpoint: str | None = None, checkpoint_every: int = 50,
                   truth: scenes.Scene | None = None, log=None) -> dict:
    """Adam on mean squared RGB error against `target` ([H, W, 4] float32 cuda)."""
    rp = init.params
    ds = rt.DeviceScene(init.scene)
    P = SceneParams(init.scene, optimize_centres)
    trainable = [p for p in P.parameters() if p.requires_grad]
    # one fused kernel for every parameter instead of a sequence of foreach ops
    opt = torch.optim.Adam(trainable, lr=lr, fused=all(p.is_cuda for p in trainable))
    start, history = 0, []
    if checkpoint and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location="cuda")
        P.load_state_dict(st["params"])
        opt.load_state_dict(st["opt"])
        start, history = st["step"], st["history"]
    tgt = target[..., :3].contiguous()
    npx = float(tgt.shape[0] * tgt.shape[1])
    for step in range(start, steps):
        opt.zero_grad(set_to_none=True)
        img = render_image(P, ds, init.camera, rp)
        loss = ((img[..., :3] - tgt) ** 2).sum() / npx
        loss.backward()
        opt.step()
        P.clamp_()
        history.append(float(loss.detach()))
        if log and (step % 20 == 0 or step == steps - 1):
            log(f"step {step:4d} loss {history[-1]:.6e}")
        if checkpoint and (step + 1) % checkpoint_every == 0:
            torch.save({"params": P.state_dict(), "opt": opt.state_dict(), "step": step + 1, "history": history},
                       checkpoint)
    out = {"history": history, "params": P}
    if truth is not None:
        Pt = SceneParams(truth, device="cuda")
        P0 = SceneParams(init.scene, device="cuda")
        rm = lambda a, b: float(torch.sqrt(torch.mean((a - b) ** 2)))  # noqa: E731
        out["material_rmse"] = (rm(P0.material_vector(), Pt.material_vector()),
                                rm(P.material_vector(), Pt.material_vector()))
        out["light_rmse"] = (rm(P0.light_vector(), Pt.light_vector()), rm(P.light_vector(), Pt.light_vector()))
    ds.close()
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


__all__ = ["SceneParams", "inverse_render", "target_image", "render_image", "loss_drop", "np"]
