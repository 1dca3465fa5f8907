"""ctypes binding of ``librt.so`` (include/rt.h): argument marshalling only.

Every step of the render runs in the library's CUDA kernels; PyTorch only
allocates device memory and provides the stream.  There is no CPU fallback: if
the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import scenes
from .build import LIB

RT_OK = 0
STATUS = {0: "RT_OK", 1: "RT_ERR_INVALID_ARG", 2: "RT_ERR_CUDA", 3: "RT_ERR_OOM",
          4: "RT_ERR_UNSUPPORTED", 5: "RT_ERR_TIMEOUT", 6: "RT_ERR_EXCEEDS_SCRATCH"}


class RtError(RuntimeError):
    def __init__(self, where: str, status: int):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres", C.c_void_p), ("has_plane", C.c_int32),
                ("plane", C.c_void_p), ("n_lights", C.c_int32), ("lights", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("yaw_deg", C.c_float), ("pitch_deg", C.c_float),
                ("fov_deg", C.c_float)]


class RenderParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("max_depth", C.c_int32),
                ("shadow_samples", C.c_int32), ("shading_model", C.c_int32),
                ("out_format", C.c_int32), ("ambient", C.c_float), ("eps", C.c_float),
                ("refl_coupled", C.c_int32), ("max_reflectivity", C.c_float), ("seed", C.c_uint64)]


class LaunchConfig(C.Structure):
    _fields_ = [("block_x", C.c_int32), ("block_y", C.c_int32), ("staging", C.c_int32),
                ("min_blocks_per_sm", C.c_int32), ("accel", C.c_int32)]


class BvhInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("depth", C.c_int32), ("max_leaf", C.c_int32), ("r_scene", C.c_float)]

    def as_dict(self) -> dict:
        return {"n_nodes": int(self.n_nodes), "depth": int(self.depth), "max_leaf": int(self.max_leaf),
                "r_scene": float(self.r_scene)}


_lib = None


def lib():
    """Load librt.so (built in-tree by paper_2305_07450_b300.build; the
    environment variable RT_LIBRARY may name another build of the same ABI)."""
    global _lib
    if _lib is None:
        path = os.environ.get("RT_LIBRARY", LIB)
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with `python -m paper_2305_07450_b300.build` "
                              "(or __graft_entry__.build()); there is no fallback path")
        L = C.CDLL(path)
        vp, i32, sz = C.c_void_p, C.c_int32, C.c_size_t
        L.rt_status_string.restype = C.c_char_p
        L.rt_status_string.argtypes = [C.c_int]
        L.rt_scene_upload.argtypes = [C.POINTER(SceneDesc), vp, C.POINTER(vp)]
        L.rt_scene_update.argtypes = [vp, C.POINTER(SceneDesc), i32, vp]
        L.rt_scene_free.argtypes = [vp]
        L.rt_render.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), vp, sz, vp,
                                C.POINTER(LaunchConfig), vp]
        L.rt_render_region.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), i32, i32, i32, i32, vp, sz,
                                       C.POINTER(LaunchConfig), vp]
        L.rt_render_region.restype = C.c_int
        L.rt_hitrec_bytes.argtypes = [vp, C.POINTER(RenderParams)]
        L.rt_hitrec_bytes.restype = sz
        L.rt_device_errors.argtypes = [vp, C.POINTER(C.c_uint32)]
        L.rt_launch_count.restype = C.c_uint64
        L.rt_scene_bytes.argtypes = [vp]
        L.rt_scene_bytes.restype = sz
        PP = C.POINTER(vp)
        L.rt_render_ws.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), vp, sz, vp,
                                   C.POINTER(LaunchConfig), vp, sz, vp]
        L.rt_render_ws.restype = C.c_int
        L.rt_render_workspace_bytes.argtypes = [vp, C.POINTER(RenderParams)]
        L.rt_render_workspace_bytes.restype = sz
        L.rt_batch_workspace_bytes.argtypes = [i32, PP, C.POINTER(RenderParams), C.POINTER(LaunchConfig)]
        L.rt_batch_workspace_bytes.restype = sz
        L.rt_render_batch.argtypes = [i32, PP, C.POINTER(Camera), C.POINTER(RenderParams), PP,
                                      C.POINTER(sz), vp, sz, C.POINTER(LaunchConfig), vp]
        L.rt_batch_create.argtypes = [i32, PP, C.POINTER(Camera), C.POINTER(RenderParams), PP,
                                      C.POINTER(sz), C.POINTER(LaunchConfig), vp, C.POINTER(vp)]
        L.rt_batch_launch.argtypes = [vp, vp]
        L.rt_selftest_wait_timeout.argtypes = [C.c_uint32, vp]
        L.rt_selftest_wait_timeout.restype = C.c_int
        L.rt_grad_count.argtypes = [vp]
        L.rt_grad_count.restype = sz
        L.rt_backward_workspace_bytes.argtypes = [vp, C.POINTER(RenderParams), C.POINTER(LaunchConfig)]
        L.rt_backward_workspace_bytes.restype = sz
        L.rt_render_backward.argtypes = [vp, C.POINTER(Camera), C.POINTER(RenderParams), vp, sz, vp, vp, vp, sz,
                                         C.POINTER(LaunchConfig), vp]
        L.rt_render_backward.restype = C.c_int
        L.rt_render_batch_noalloc.argtypes = [i32, PP, C.POINTER(Camera), C.POINTER(RenderParams), PP,
                                              C.POINTER(sz), C.POINTER(LaunchConfig), vp]
        L.rt_render_batch_noalloc.restype = C.c_int
        L.rt_batch_free.argtypes = [vp]
        L.rt_scene_build_bvh.argtypes = [vp, vp, C.POINTER(BvhInfo)]
        L.rt_scene_build_bvh.restype = C.c_int
        L.rt_bvh_build_host.argtypes = [C.POINTER(SceneDesc), vp, i32, vp, C.POINTER(BvhInfo)]
        L.rt_bvh_build_host.restype = C.c_int
        L.rt_scene_set_sky.argtypes = [vp, vp, i32, i32, vp]
        L.rt_scene_set_sky.restype = C.c_int
        L.rt_verlet_step.argtypes = [vp, vp, i32, vp, C.c_float, C.c_float, C.c_float, i32, vp]
        L.rt_verlet_step.restype = C.c_int
        for name in ("rt_scene_upload", "rt_scene_update", "rt_scene_free", "rt_render",
                     "rt_device_errors", "rt_render_batch", "rt_batch_create", "rt_batch_launch",
                     "rt_batch_free"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def check(where: str, st: int):
    if st != RT_OK:
        raise RtError(where, st)


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def camera_struct(cam) -> Camera:
    c = np.asarray(cam, np.float32).reshape(6)
    s = Camera()
    s.pos[0], s.pos[1], s.pos[2] = float(c[0]), float(c[1]), float(c[2])
    s.yaw_deg, s.pitch_deg, s.fov_deg = float(c[3]), float(c[4]), float(c[5])
    return s


def params_struct(p: scenes.Params) -> RenderParams:
    s = RenderParams()
    s.width, s.height, s.max_depth = int(p.width), int(p.height), int(p.max_depth)
    s.shadow_samples, s.shading_model, s.out_format = int(p.shadow_samples), int(p.shading_model), int(p.out_format)
    s.ambient, s.eps = float(p.ambient), float(p.eps)
    s.refl_coupled, s.max_reflectivity = int(p.refl_coupled), float(p.max_reflectivity)
    s.seed = int(p.seed) & 0xFFFFFFFFFFFFFFFF
    return s


def launch_struct(launch) -> LaunchConfig | None:
    if launch is None:
        return None
    s = LaunchConfig()
    fields = {f[0] for f in LaunchConfig._fields_}
    for k, v in dict(launch).items():
        if k in fields:  # "queued" (the autotuner's choice of rt_render_ws) is not a field
            setattr(s, k, int(v))
    return s


class DeviceScene:
    """A scene resident on the device (rt_scene_upload); freed on close()/del."""

    def __init__(self, scene: scenes.Scene, stream=None):
        self._h = C.c_void_p()
        self.n_spheres = scene.n_spheres
        self.n_lights = scene.n_lights
        self.has_plane = scene.plane is not None
        self._keep = self._desc(scene)
        check("rt_scene_upload", lib().rt_scene_upload(C.byref(self._keep[0]), _stream(stream), C.byref(self._h)))
        if getattr(scene, "sky", None) is not None:
            self.set_sky(scene.sky, stream=stream)

    def set_sky(self, texels, stream=None):
        """rt_scene_set_sky: an [H, W, 4] FP32 panorama (host), or None for black misses."""
        if texels is None:
            check("rt_scene_set_sky", lib().rt_scene_set_sky(self._h, None, 0, 0, _stream(stream)))
            return
        t = np.ascontiguousarray(texels, dtype=np.float32)
        assert t.ndim == 3 and t.shape[2] == 4
        check("rt_scene_set_sky", lib().rt_scene_set_sky(self._h, t.ctypes.data, int(t.shape[1]), int(t.shape[0]),
                                                         _stream(stream)))

    @staticmethod
    def _desc(scene: scenes.Scene):
        sph = np.ascontiguousarray(scene.spheres, np.float32).reshape(-1, 10)
        pl = None if scene.plane is None else np.ascontiguousarray(scene.plane, np.float32)
        lig = np.ascontiguousarray(scene.lights, np.float32).reshape(-1, 8)
        d = SceneDesc()
        d.n_spheres = sph.shape[0]
        d.spheres = sph.ctypes.data if sph.size else None
        d.has_plane = 1 if pl is not None else 0
        d.plane = pl.ctypes.data if pl is not None else None
        d.n_lights = lig.shape[0]
        d.lights = lig.ctypes.data if lig.size else None
        return d, sph, pl, lig

    def update(self, scene: scenes.Scene | None = None, *, spheres: torch.Tensor | None = None,
               plane: torch.Tensor | None = None, lights: torch.Tensor | None = None, stream=None):
        """Overwrite the scene: from host records (scene) or device tensors."""
        if scene is not None:
            keep = self._desc(scene)
            check("rt_scene_update", lib().rt_scene_update(self._h, C.byref(keep[0]), 0, _stream(stream)))
            return
        d = SceneDesc()
        d.n_spheres = self.n_spheres
        d.spheres = spheres.data_ptr() if spheres is not None else None
        d.has_plane = 1 if self.has_plane else 0
        d.plane = plane.data_ptr() if plane is not None else None
        d.n_lights = self.n_lights
        d.lights = lights.data_ptr() if lights is not None else None
        for t in (spheres, plane, lights):
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        check("rt_scene_update", lib().rt_scene_update(self._h, C.byref(d), 1, _stream(stream)))

    def build_bvh(self, stream=None) -> dict:
        """rt_scene_build_bvh: (re)build the sphere hierarchy that launch
        {"accel": 1} renders through; returns its figures."""
        info = BvhInfo()
        check("rt_scene_build_bvh", lib().rt_scene_build_bvh(self._h, _stream(stream), C.byref(info)))
        return info.as_dict()

    @property
    def nbytes(self) -> int:
        """Bytes of the device scene table (one host-to-device upload)."""
        return int(lib().rt_scene_bytes(self._h))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().rt_scene_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def verlet_step(spheres: torch.Tensor, prev: torch.Tensor, plane=None, *, dt: float = 1.0 / 60.0,
                gravity: float = 9.81, restitution: float = 0.7, steps: int = 1, stream=None):
    """rt_verlet_step: advance the device sphere records [N, 10] (centres in place)
    and previous centres [N, 3] by `steps` Verlet steps; plane = record (nx, ny, nz,
    d, ...) or None."""
    for t in (spheres, prev):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    n = int(spheres.shape[0])
    assert spheres.numel() == 10 * n and prev.numel() == 3 * n
    pl = None if plane is None else np.ascontiguousarray(np.asarray(plane, np.float32)[:4])
    check("rt_verlet_step", lib().rt_verlet_step(spheres.data_ptr(), prev.data_ptr(), n,
                                                 pl.ctypes.data if pl is not None else None, float(dt), float(gravity),
                                                 float(restitution), int(steps), _stream(stream)))


NODE_DTYPE = np.dtype([("a_lo", "<f4", 3), ("a_hi", "<f4", 3), ("b_lo", "<f4", 3), ("b_hi", "<f4", 3),
                       ("ref", "<i4", 2), ("zero", "<i4", 2)])


def bvh_build_host(scene: scenes.Scene):
    """rt_bvh_build_host: the hierarchy the device would use, built on the host only
    (no GPU needed).  Returns (nodes as a NODE_DTYPE array, prim_idx, info dict)."""
    d, *keep = DeviceScene._desc(scene)
    info = BvhInfo()
    check("rt_bvh_build_host", lib().rt_bvh_build_host(C.byref(d), None, 0, None, C.byref(info)))
    nodes = np.zeros(max(int(info.n_nodes), 1), NODE_DTYPE)
    prim = np.zeros(max(scene.n_spheres, 1), np.int32)
    check("rt_bvh_build_host", lib().rt_bvh_build_host(C.byref(d), nodes.ctypes.data, int(info.n_nodes),
                                                       prim.ctypes.data, C.byref(info)))
    return nodes[: int(info.n_nodes)], prim[: scene.n_spheres], info.as_dict()


def alloc_output(params: scenes.Params, device="cuda") -> tuple[torch.Tensor, int]:
    """Framebuffer tensor and its row pitch in bytes (a multiple of 16)."""
    W, H = int(params.width), int(params.height)
    if params.out_format == scenes.OUT_F32:
        return torch.empty((H, W, 4), dtype=torch.float32, device=device), W * 16
    words = (W + 3) // 4 * 4
    buf = torch.empty((H, words), dtype=torch.int32, device=device)
    return buf, words * 4


def hitrec_bytes(dscene: DeviceScene, params: scenes.Params) -> int:
    return int(lib().rt_hitrec_bytes(dscene.handle, C.byref(params_struct(params))))


def render_workspace_bytes(dscene: DeviceScene, params: scenes.Params) -> int:
    """rt_render_workspace_bytes: the workspace rt_render_ws suggests for a frame."""
    return int(lib().rt_render_workspace_bytes(dscene.handle, C.byref(params_struct(params))))


def alloc_workspace(dscene: DeviceScene, params: scenes.Params, nbytes: int | None = None,
                    device="cuda") -> torch.Tensor:
    """A 256-byte aligned device buffer for rt_render_ws (torch allocations are)."""
    n = render_workspace_bytes(dscene, params) if nbytes is None else int(nbytes)
    ws = torch.empty(max(n, 256), dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def render(dscene: DeviceScene, camera, params: scenes.Params, *, out: torch.Tensor | None = None,
           pitch: int | None = None, hitrec: torch.Tensor | None = None, launch=None,
           stream=None, workspace: torch.Tensor | None = None) -> torch.Tensor:
    """rt_render, or rt_render_ws when a workspace (alloc_workspace) is given -- the
    same pixels, rendered in passes over compacted paths.  A launch with
    "queued": 1 (the autotuner's choice) and no workspace gets one allocated here.
    Returns the framebuffer: float32 [H, W, 4] (F32) or int32 [H, W] holding
    0xAABBGGRR (RGBA8)."""
    if workspace is None and launch is not None and dict(launch).get("queued"):
        workspace = alloc_workspace(dscene, params)
    if out is None:
        out, pitch = alloc_output(params)
    elif pitch is None:
        pitch = out.stride(0) * out.element_size()
    cam, prm, cfg = camera_struct(camera), params_struct(params), launch_struct(launch)
    hr = None
    if hitrec is not None:
        assert hitrec.is_cuda and hitrec.numel() * hitrec.element_size() >= hitrec_bytes(dscene, params)
        hr = hitrec.data_ptr()
    cfgp = C.byref(cfg) if cfg is not None else None
    if workspace is not None:
        assert workspace.is_cuda and workspace.is_contiguous()
        nb = workspace.numel() * workspace.element_size()
        check("rt_render_ws", lib().rt_render_ws(dscene.handle, C.byref(cam), C.byref(prm), out.data_ptr(), pitch,
                                                 hr, cfgp, workspace.data_ptr(), nb, _stream(stream)))
    else:
        check("rt_render", lib().rt_render(dscene.handle, C.byref(cam), C.byref(prm), out.data_ptr(), pitch, hr,
                                           cfgp, _stream(stream)))
    if params.out_format != scenes.OUT_F32:
        return out[:, : params.width]
    return out


def render_region(dscene: DeviceScene, camera, params: scenes.Params, x0: int, y0: int, width: int, height: int,
                  *, out: torch.Tensor | None = None, pitch: int | None = None, launch=None,
                  stream=None) -> torch.Tensor:
    """rt_render_region: rows y0..y0+height and columns x0..x0+width of the frame
    described by params (x0 a multiple of 8), bit-identical to those pixels of the
    full frame."""
    sub = scenes.Params(**{**params.__dict__, "width": width, "height": height})
    if out is None:
        out, pitch = alloc_output(sub)
    elif pitch is None:
        pitch = out.stride(0) * out.element_size()
    cam, prm, cfg = camera_struct(camera), params_struct(params), launch_struct(launch)
    check("rt_render_region", lib().rt_render_region(dscene.handle, C.byref(cam), C.byref(prm), int(x0), int(y0),
                                                     int(width), int(height), out.data_ptr(), pitch,
                                                     C.byref(cfg) if cfg is not None else None, _stream(stream)))
    if params.out_format != scenes.OUT_F32:
        return out[:, :width]
    return out


def device_errors(stream=None) -> int:
    bits = C.c_uint32(0)
    st = lib().rt_device_errors(_stream(stream), C.byref(bits))
    if st not in (RT_OK, 5):
        raise RtError("rt_device_errors", st)
    return int(bits.value)


def launch_count() -> int:
    return int(lib().rt_launch_count())


def rgba8_to_float(img: torch.Tensor) -> torch.Tensor:
    """Unpack 0xAABBGGRR words into uint8 channels [..., 4]."""
    v = img.contiguous().view(torch.uint8).reshape(*img.shape, 4)
    return v


# ------------------------------------------------------------------ batches
def _batch_arrays(dscenes, cameras, params_list, outs, pitches):
    n = len(dscenes)
    sc = (C.c_void_p * n)(*[d.handle.value for d in dscenes])
    cams = (Camera * n)(*[camera_struct(c) for c in cameras])
    prm = (RenderParams * n)(*[params_struct(p) for p in params_list])
    op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    pt = (C.c_size_t * n)(*[int(p) for p in pitches])
    return n, sc, cams, prm, op, pt


def alloc_batch_outputs(params_list, device="cuda"):
    outs, pitches = [], []
    for p in params_list:
        o, pt = alloc_output(p, device)
        outs.append(o)
        pitches.append(pt)
    return outs, pitches


def batch_workspace_bytes(dscenes, params_list, launch=None) -> int:
    n = len(dscenes)
    sc = (C.c_void_p * n)(*[d.handle.value for d in dscenes])
    prm = (RenderParams * n)(*[params_struct(p) for p in params_list])
    cfg = launch_struct(launch)
    return int(lib().rt_batch_workspace_bytes(n, sc, prm, C.byref(cfg) if cfg is not None else None))


def render_batch(dscenes, cameras, params_list, *, outs=None, pitches=None, workspace=None, launch=None,
                 stream=None):
    """rt_render_batch: one persistent-kernel launch over every frame, with a
    caller-owned device workspace (allocated here as a torch tensor if None)."""
    if outs is None:
        outs, pitches = alloc_batch_outputs(params_list)
    ws_bytes = batch_workspace_bytes(dscenes, params_list, launch)
    if workspace is None:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    n, sc, cams, prm, op, pt = _batch_arrays(dscenes, cameras, params_list, outs, pitches)
    cfg = launch_struct(launch)
    check("rt_render_batch", lib().rt_render_batch(n, sc, cams, prm, op, pt, workspace.data_ptr(),
                                                   workspace.numel() * workspace.element_size(),
                                                   C.byref(cfg) if cfg is not None else None, _stream(stream)))
    return [o[:, : p.width] if p.out_format != scenes.OUT_F32 else o for o, p in zip(outs, params_list)], workspace


class Batch:
    """rt_batch_create / rt_batch_launch: the batch planned once and replayed as a
    CUDA graph {reset work counter, persistent kernel}."""

    def __init__(self, dscenes, cameras, params_list, *, outs=None, pitches=None, launch=None, stream=None):
        if outs is None:
            outs, pitches = alloc_batch_outputs(params_list)
        self.outs, self.pitches, self.params = outs, pitches, params_list
        self._scenes = list(dscenes)  # keep the scenes alive
        n, sc, cams, prm, op, pt = _batch_arrays(dscenes, cameras, params_list, outs, pitches)
        cfg = launch_struct(launch)
        self._h = C.c_void_p()
        check("rt_batch_create", lib().rt_batch_create(n, sc, cams, prm, op, pt,
                                                       C.byref(cfg) if cfg is not None else None,
                                                       _stream(stream), C.byref(self._h)))

    def launch(self, stream=None):
        check("rt_batch_launch", lib().rt_batch_launch(self._h, _stream(stream)))

    def outputs(self):
        return [o[:, : p.width] if p.out_format != scenes.OUT_F32 else o for o, p in zip(self.outs, self.params)]

    def close(self):
        if self._h:
            lib().rt_batch_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ adjoint
def grad_count(dscene: DeviceScene) -> int:
    return int(lib().rt_grad_count(dscene.handle))


def backward_workspace_bytes(dscene: DeviceScene, params: scenes.Params, launch=None) -> int:
    """rt_backward_workspace_bytes: the workspace rt_render_backward needs."""
    cfg = launch_struct(launch)
    return int(lib().rt_backward_workspace_bytes(dscene.handle, C.byref(params_struct(params)),
                                                 C.byref(cfg) if cfg is not None else None))


def render_backward(dscene: DeviceScene, camera, params: scenes.Params, dl_dimg: torch.Tensor, *,
                    hitrec: torch.Tensor | None = None, grad: torch.Tensor | None = None,
                    workspace: torch.Tensor | None = None, launch=None, stream=None) -> torch.Tensor:
    """rt_render_backward: packed gradient (rt_grad_count floats) of
    sum(dl_dimg * image) with respect to the scene parameters."""
    assert dl_dimg.is_cuda and dl_dimg.dtype == torch.float32 and dl_dimg.shape[-1] == 4
    dl = dl_dimg.contiguous()
    cam, prm, cfg = camera_struct(camera), params_struct(params), launch_struct(launch)
    cfgp = C.byref(cfg) if cfg is not None else None
    if grad is None:
        grad = torch.empty(grad_count(dscene), dtype=torch.float32, device="cuda")
    need = int(lib().rt_backward_workspace_bytes(dscene.handle, C.byref(prm), cfgp))
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(max(need, 16) // 4 + 4, dtype=torch.float32, device="cuda")
    check("rt_render_backward", lib().rt_render_backward(
        dscene.handle, C.byref(cam), C.byref(prm), dl.data_ptr(), dl.stride(0) * 4,
        hitrec.data_ptr() if hitrec is not None else None, grad.data_ptr(), workspace.data_ptr(),
        workspace.numel() * workspace.element_size(), cfgp, _stream(stream)))
    return grad


_UNPACK_INDEX: dict = {}


def _unpack_index(n_spheres: int, n_lights: int, device, coupled: bool = False) -> torch.Tensor:
    """Gather map from the packed gradient (plus one appended zero, index G) to
    the concatenated records [spheres N x 10 | plane 10 | lights L x 8].  The
    packed reflectivity entry goes to the reflectivity field (column 9), or with
    the coupled reflection ratio to the specular exponent field (column 8)."""
    key = (n_spheres, n_lights, str(device), bool(coupled))
    idx = _UNPACK_INDEX.get(key)
    if idx is None:
        N, L = n_spheres, n_lights
        z = 8 * (N + 1) + 4 * L
        sph = np.full((N, 10), z, np.int64)
        base = 8 * np.arange(N, dtype=np.int64)[:, None]
        sph[:, 0:3] = base + np.array([5, 6, 7])
        sph[:, 4:8] = base + np.array([0, 1, 2, 3])
        rcol = 8 if coupled else 9
        sph[:, rcol] = base[:, 0] + 4
        pl = np.full(10, z, np.int64)
        pl[4:8] = 8 * N + np.arange(4)
        pl[rcol] = 8 * N + 4
        lig = np.full((L, 8), z, np.int64)
        lig[:, 0:4] = 8 * (N + 1) + 4 * np.arange(L, dtype=np.int64)[:, None] + np.arange(4)
        idx = torch.from_numpy(np.concatenate([sph.ravel(), pl, lig.ravel()])).to(device)
        _UNPACK_INDEX[key] = idx
    return idx


def unpack_grad(grad: torch.Tensor, n_spheres: int, n_lights: int, coupled: bool = False):
    """Packed gradient -> (spheres [N, 10], plane [10], lights [L, 8]) laid out
    like the scene records (zeros where a field is not differentiated): one
    gather through a cached index map (coupled: the render used the coupled
    reflection ratio, so the reflectivity entry belongs to the exponent field)."""
    N, L = n_spheres, n_lights
    G = 8 * (N + 1) + 4 * L
    flat = torch.cat([grad[:G], grad.new_zeros(1)])[_unpack_index(N, L, grad.device, coupled)]
    return flat[: 10 * N].view(N, 10), flat[10 * N: 10 * N + 10], flat[10 * N + 10:].view(L, 8)


class RenderFn(torch.autograd.Function):
    """Differentiable render.  forward(spheres [N,10], plane [10], lights [L,8],
    dscene, camera, params) -> image [H, W, 4] (F32, linear); backward through
    the hand-written adjoint, replaying the hit record of the forward render.
    The scene records are device tensors; the device scene is overwritten with
    them (device-to-device) before each render and again before the adjoint."""

    @staticmethod
    def forward(ctx, spheres, plane, lights, dscene, camera, params):
        p = params if params.out_format == scenes.OUT_F32 else dataclasses_replace(params)
        sph, pl, lig = spheres.detach().contiguous(), plane.detach().contiguous(), lights.detach().contiguous()
        dscene.update(spheres=sph, plane=pl if dscene.has_plane else None, lights=lig)
        hr = torch.empty(hitrec_bytes(dscene, p) // 4 + 1, dtype=torch.float32, device="cuda")
        img = render(dscene, camera, p, hitrec=hr)
        ctx.save_for_backward(sph, pl, lig, hr)
        ctx.dscene, ctx.camera, ctx.params = dscene, camera, p
        return img

    @staticmethod
    def backward(ctx, grad_img):
        sph, pl, lig, hr = ctx.saved_tensors
        ds = ctx.dscene
        ds.update(spheres=sph, plane=pl if ds.has_plane else None, lights=lig)
        g = render_backward(ds, ctx.camera, ctx.params, grad_img.float(), hitrec=hr)
        gs, gp, gl = unpack_grad(g, ds.n_spheres, ds.n_lights, coupled=bool(ctx.params.refl_coupled))
        return gs, gp, gl, None, None, None


def dataclasses_replace(params: scenes.Params) -> scenes.Params:
    import dataclasses
    return dataclasses.replace(params, out_format=scenes.OUT_F32)
