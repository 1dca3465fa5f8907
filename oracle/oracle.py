"""ctypes wrapper of the FP64 C oracle (``rt_oracle.c``).

Test infrastructure only.  It marshals the seeded FP32 scene records into the
oracle's own input block and splits pixel lists over host threads (each C call
renders a contiguous run of pixels; ctypes releases the GIL during the call).
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

COUNTERS = ("primary_rays", "reflection_rays", "shadow_rays", "closest_sphere_tests",
            "closest_plane_tests", "shadow_sphere_tests", "shadow_plane_tests",
            "hits", "lit_lights", "light_samples", "philox_calls", "reserved")


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile the oracle with gcc -O2 (no fast-math: IEEE FP64 throughout)."""
    out = out or LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
               "-fvisibility=hidden", "-fno-fast-math", "-ffp-contract=off",
               *extra_flags, "-o", out, SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return out


class OrcIn(C.Structure):
    _fields_ = [
        ("n_spheres", C.c_int), ("spheres", C.POINTER(C.c_float)),
        ("has_plane", C.c_int), ("plane", C.POINTER(C.c_float)),
        ("n_lights", C.c_int), ("lights", C.POINTER(C.c_float)),
        ("camera", C.POINTER(C.c_float)),
        ("width", C.c_int), ("height", C.c_int), ("max_depth", C.c_int),
        ("shadow_samples", C.c_int), ("shading_model", C.c_int), ("pad_", C.c_int),
        ("ambient", C.c_double), ("eps", C.c_double), ("scene_scale", C.c_double),
        ("seed", C.c_uint64), ("refl_coupled", C.c_int), ("pad2_", C.c_int),
        ("max_reflectivity", C.c_double),
        ("sky", C.POINTER(C.c_float)), ("sky_w", C.c_int), ("sky_h", C.c_int),
    ]


_lib = None


def lib(path: str | None = None):
    global _lib
    if path is not None:
        return _bind(C.CDLL(path))
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(L):
    dp = C.POINTER(C.c_double)
    L.orc_trace.argtypes = [C.POINTER(OrcIn), C.c_int, C.c_int, C.POINTER(C.c_int32),
                            C.c_double, C.c_double, dp, dp, dp]
    L.orc_trace.restype = C.c_int
    L.orc_to_rgba8.argtypes = [C.c_int, dp, C.POINTER(C.c_uint32)]
    L.orc_ndc.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp]
    L.orc_camera_distance.argtypes = [C.c_double]
    L.orc_camera_distance.restype = C.c_double
    L.orc_primary_ray.argtypes = [C.POINTER(OrcIn), C.c_double, C.c_double, C.c_double,
                                  C.c_double, dp]
    L.orc_primary_ray.restype = C.c_int
    L.orc_sphere_root.argtypes = [dp, dp, dp, C.c_double, dp]
    L.orc_sphere_root.restype = C.c_int
    L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
    L.orc_closest.argtypes = [C.POINTER(OrcIn), dp, dp, C.c_int, dp, dp]
    L.orc_closest.restype = C.c_int
    L.orc_occluded.argtypes = [C.POINTER(OrcIn), dp, dp, C.c_double, C.c_int, dp]
    L.orc_occluded.restype = C.c_int
    L.orc_trace_path.argtypes = [C.POINTER(OrcIn), C.c_int, C.c_int, dp]
    L.orc_trace_path.restype = C.c_int
    L.orc_light_samples.argtypes = [C.POINTER(OrcIn), C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
    L.orc_light_samples.restype = C.c_int
    L.orc_sky.argtypes = [C.POINTER(C.c_float), C.c_int, C.c_int, dp, dp]
    L.orc_sky.restype = C.c_int
    L.orc_verlet.argtypes = [C.c_int, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_int]
    L.orc_verlet.restype = C.c_int
    return L


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _In:
    """Keeps the FP32 arrays alive while the C struct points into them."""

    def __init__(self, scene, camera, params):
        self.sph = np.ascontiguousarray(scene.spheres, dtype=np.float32).reshape(-1, 10)
        self.pl = (np.ascontiguousarray(scene.plane, dtype=np.float32) if scene.plane is not None
                   else np.zeros(10, np.float32))
        self.lig = np.ascontiguousarray(scene.lights, dtype=np.float32).reshape(-1, 8)
        self.cam = np.ascontiguousarray(camera, dtype=np.float32).reshape(6)
        s = OrcIn()
        s.n_spheres = self.sph.shape[0]
        s.spheres = _fp(self.sph)
        s.has_plane = 1 if scene.plane is not None else 0
        s.plane = _fp(self.pl)
        s.n_lights = self.lig.shape[0]
        s.lights = _fp(self.lig)
        s.camera = _fp(self.cam)
        s.width, s.height = int(params.width), int(params.height)
        s.max_depth = int(params.max_depth)
        s.shadow_samples = int(params.shadow_samples)
        s.shading_model = int(params.shading_model)
        s.ambient = float(params.ambient)
        s.eps = float(params.eps)
        s.scene_scale = float(scene.scene_scale)
        s.seed = int(params.seed) & 0xFFFFFFFFFFFFFFFF
        s.refl_coupled = int(getattr(params, "refl_coupled", 0))
        s.max_reflectivity = float(getattr(params, "max_reflectivity", 0.0))
        sky = getattr(scene, "sky", None)
        if sky is not None:
            self.sky = np.ascontiguousarray(sky, dtype=np.float32)
            s.sky = _fp(self.sky)
            s.sky_h, s.sky_w = int(self.sky.shape[0]), int(self.sky.shape[1])
        self.s = s


def all_pixels(width: int, height: int) -> np.ndarray:
    ys, xs = np.meshgrid(np.arange(height, dtype=np.int32), np.arange(width, dtype=np.int32),
                         indexing="ij")
    return np.ascontiguousarray(np.stack([xs.ravel(), ys.ravel()], 1))


def trace(scene, camera, params, pixels: np.ndarray | None = None, *, mode: str = "forward",
          ndc_offset: tuple[float, float] = (0.0, 0.0), margin: bool = False,
          counters: bool = False, threads: int | None = None, chunk: int = 256):
    """Trace pixels with the FP64 oracle.

    pixels: int32 [n, 2] (x, y); None = the whole frame (row-major).
    Returns dict: rgb float64 [n, 3]; margin float64 [n] (if asked);
    counters dict (if asked); threads used.
    """
    L = lib()
    inp = _In(scene, camera, params)
    px = all_pixels(params.width, params.height) if pixels is None else \
        np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    n = px.shape[0]
    rgb = np.zeros((n, 3), np.float64)
    mg = np.zeros(n, np.float64) if margin else None
    threads = threads or os.cpu_count() or 1
    m = 1 if mode == "recursive" else 0
    starts = list(range(0, n, chunk))
    cnts = np.zeros((len(starts), 12), np.float64)

    def run(ci):
        a = starts[ci]
        b = min(n, a + chunk)
        sub_px = px[a:b]
        sub_rgb = rgb[a:b]
        st = L.orc_trace(C.byref(inp.s), m, b - a, sub_px.ctypes.data_as(C.POINTER(C.c_int32)),
                         float(ndc_offset[0]), float(ndc_offset[1]), _dp(sub_rgb),
                         _dp(mg[a:b]) if mg is not None else None,
                         _dp(cnts[ci]) if counters else None)
        if st != 0:
            raise ValueError(f"oracle rejected the input (status {st})")

    if threads == 1 or len(starts) == 1:
        for ci in range(len(starts)):
            run(ci)
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, range(len(starts))))
    out = {"rgb": rgb, "threads": threads}
    if margin:
        out["margin"] = mg
    if counters:
        tot = cnts.sum(0)
        out["counters"] = {k: int(v) for k, v in zip(COUNTERS, tot)}
    return out


def render(scene, camera, params, **kw) -> np.ndarray:
    """Whole frame, float64 [H, W, 3]."""
    r = trace(scene, camera, params, None, **kw)
    return r["rgb"].reshape(params.height, params.width, 3)


def to_rgba8(rgb: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(rgb, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(a.shape[0], np.uint32)
    lib().orc_to_rgba8(a.shape[0], _dp(a), out.ctypes.data_as(C.POINTER(C.c_uint32)))
    return out.reshape(rgb.shape[:-1])


def ndc(W: int, H: int, x: float, y: float) -> tuple[float, float]:
    uv = np.zeros(2, np.float64)
    lib().orc_ndc(W, H, float(x), float(y), _dp(uv))
    return float(uv[0]), float(uv[1])


def camera_distance(fov_deg: float) -> float:
    return float(lib().orc_camera_distance(float(fov_deg)))


def primary_ray(scene, camera, params, x: float, y: float, du: float = 0.0, dv: float = 0.0):
    inp = _In(scene, camera, params)
    od = np.zeros(6, np.float64)
    st = lib().orc_primary_ray(C.byref(inp.s), float(x), float(y), du, dv, _dp(od))
    if st:
        raise ValueError("bad input")
    return od[:3].copy(), od[3:].copy()


def sphere_root(o, d, c, r):
    o, d, c = (np.ascontiguousarray(v, np.float64) for v in (o, d, c))
    t = np.zeros(1, np.float64)
    hit = lib().orc_sphere_root(_dp(o), _dp(d), _dp(c), float(r), _dp(t))
    return (float(t[0]) if hit else None)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    u = C.POINTER(C.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(u), k.ctypes.data_as(u), o.ctypes.data_as(u))
    return o


def closest(scene, camera, params, o, d, *, origin: int = -1, margin: bool = False):
    """(id, t) of the closest hit of one ray; id = -1 on a miss.  origin: the
    primitive the ray leaves (-1: none).  margin=True: (id, t, the ray's margin)."""
    inp = _In(scene, camera, params)
    o, d = (np.ascontiguousarray(v, np.float64) for v in (o, d))
    t = np.zeros(1, np.float64)
    m = np.zeros(1, np.float64)
    i = lib().orc_closest(C.byref(inp.s), _dp(o), _dp(d), int(origin), _dp(t), _dp(m) if margin else None)
    if i < -1:
        raise ValueError("bad input")
    res = (i, (float(t[0]) if i >= 0 else None))
    return res + (float(m[0]),) if margin else res


def occluded(scene, camera, params, o, d, dist, *, origin: int = -1, margin: bool = False):
    """Whether the shadow segment o + t d, 0 < t < dist, is blocked; margin=True:
    (blocked, the segment's margin)."""
    inp = _In(scene, camera, params)
    o, d = (np.ascontiguousarray(v, np.float64) for v in (o, d))
    m = np.zeros(1, np.float64)
    r = lib().orc_occluded(C.byref(inp.s), _dp(o), _dp(d), float(dist), int(origin), _dp(m) if margin else None)
    if r < 0:
        raise ValueError("bad input")
    return (bool(r), float(m[0])) if margin else bool(r)


def trace_path(scene, camera, params, x: int, y: int) -> np.ndarray:
    """The ray path of pixel (x, y): [n, 14] rows (id, t, origin 3, direction 3,
    hit point 3, normal 3) per bounce, the last row a miss (id -1) if the path
    leaves the scene before the bounce limit."""
    inp = _In(scene, camera, params)
    out = np.zeros((int(params.max_depth) + 1, 14), np.float64)
    n = lib().orc_trace_path(C.byref(inp.s), int(x), int(y), _dp(out))
    if n < 0:
        raise ValueError("bad input")
    return out[:n].copy()


def light_samples(scene, camera, params, l, x, y, k, p=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Sample points [n, 3] of sampled light l for pixel (x, y), bounce k, point p."""
    inp = _In(scene, camera, params)
    pp = np.ascontiguousarray(p, np.float64)
    out = np.zeros((4096, 3), np.float64)
    n = lib().orc_light_samples(C.byref(inp.s), int(l), int(x), int(y), int(k), _dp(pp), _dp(out))
    if n < 0:
        raise ValueError("bad input")
    return out[:n].copy()


def sky(tex, d) -> np.ndarray:
    """Sky colour (RGB) of direction d for an [H, W, 4] FP32 panorama."""
    t = np.ascontiguousarray(tex, dtype=np.float32)
    dd = np.ascontiguousarray(d, np.float64)
    out = np.zeros(3, np.float64)
    if lib().orc_sky(_fp(t), int(t.shape[1]), int(t.shape[0]), _dp(dd), _dp(out)):
        raise ValueError("bad input")
    return out


def verlet(pos, prev, radius, plane, dt: float, g: float, e: float, steps: int):
    """Position-Verlet physics with ground contact: returns (pos, prev) [n, 3] after
    `steps` steps (FP64); plane = (nx, ny, nz, d) or None."""
    p = np.array(pos, np.float64, copy=True).reshape(-1, 3)
    q = np.array(prev, np.float64, copy=True).reshape(-1, 3)
    r = np.ascontiguousarray(radius, np.float64).reshape(-1)
    pl = None if plane is None else np.ascontiguousarray(np.asarray(plane, np.float64)[:4])
    if lib().orc_verlet(p.shape[0], _dp(p), _dp(q), _dp(r), _dp(pl) if pl is not None else None,
                        float(dt), float(g), float(e), int(steps)):
        raise ValueError("bad input")
    return p, q


class using_library:
    """Context manager: route every call of this module to another build of the
    oracle (the mutation tests load deliberately broken copies this way)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.prev = _lib
        _lib = _bind(C.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev
        return False
