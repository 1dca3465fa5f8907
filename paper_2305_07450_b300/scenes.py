"""Seeded synthetic inputs for the per-pixel ray tracer (arXiv 2305.07450, Section 3).

This module only draws numbers: it holds none of the renderer's arithmetic.  It is
the one module that both the FP64 oracle (``oracle/``) and the CUDA path read, so
that both render exactly the same FP32 scene.

Record layouts (all float32, the paper's body SoA of Section 3.9 widened by the
material fields the shading of Section 3.5 needs):

* sphere  ``[10]``: cx, cy, cz, radius, albedo r, g, b, k_s, spec_exp, reflectivity
* plane   ``[10]``: nx, ny, nz, d (points x with n.x + d = 0), albedo r, g, b,
  k_s, spec_exp, reflectivity
* light   ``[8]`` : x, y, z, intensity, area_side (0 = point light, > 0 = square
  area light of that side, horizontal, facing down), sphere_radius (> 0 = spherical
  light sampled on the great circle facing the point, Section 3.6.1), 0, 0
* camera  ``[6]`` : x, y, z, yaw_deg, pitch_deg, fov_deg (the paper's camera array,
  Section 3.1 / Section 3.9)

The paper's own benchmark scene (one light, one plane, five spheres and an HDR sky,
Section 4.1) is given only in words, so seeded scenes of the same structure stand
in for it.  Draw order is fixed: one ``(N, 8)`` block of U[0,1) for the spheres
(columns cx, cy, cz, r, albedo r, g, b, reflectivity), then one ``(L, 4)`` block for
the lights (x, y, z, intensity).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPHERE_FIELDS = 10
PLANE_FIELDS = 10
LIGHT_FIELDS = 8

PHONG = 0
BLINN_PHONG = 1
OUT_RGBA8 = 0
OUT_F32 = 1

# Material constants that the paper leaves open (ambient strength, Section 3.5.1;
# specular coefficient and exponent, Section 3.5.1 'Specular lighting').
AMBIENT = 0.1
K_S = 0.5
SPEC_EXP = 32.0
PLANE_ALBEDO = 0.75
PLANE_REFL = 0.25
EPS_SCALE = 1e-4


@dataclasses.dataclass
class Scene:
    spheres: np.ndarray            # float32 [N, 10]
    plane: np.ndarray | None       # float32 [10] or None
    lights: np.ndarray             # float32 [L, 8]
    scale: float = 1.0             # the box scale s of the generator
    sky: np.ndarray | None = None  # float32 [H, W, 4] equirectangular panorama (None: black)

    @property
    def scene_scale(self) -> float:
        """Half-extent of the sphere box in x (5 s): the length unit of margins."""
        return 5.0 * self.scale

    @property
    def n_spheres(self) -> int:
        return int(self.spheres.shape[0])

    @property
    def n_lights(self) -> int:
        return int(self.lights.shape[0])


@dataclasses.dataclass
class Params:
    width: int
    height: int
    max_depth: int = 1
    shadow_samples: int = 1        # samples per sampled (area / spherical) light
    shading_model: int = PHONG
    out_format: int = OUT_F32
    ambient: float = AMBIENT
    eps: float = EPS_SCALE * 5.0   # absolute self-intersection offset
    seed: int = 0
    refl_coupled: int = 0          # 1: reflection ratio = spec_exp / max_reflectivity (Section 3.7)
    max_reflectivity: float = 0.0


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    camera: np.ndarray             # float32 [6]
    params: Params


def f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def default_camera(scale: float) -> np.ndarray:
    """Camera above and behind the sphere box, looking down 12 degrees, 60 deg FOV."""
    return f32([0.0, 3.0 * scale, -13.0 * scale, 0.0, -12.0, 60.0])


def default_plane() -> np.ndarray:
    return f32([0.0, 1.0, 0.0, 0.0, PLANE_ALBEDO, PLANE_ALBEDO, PLANE_ALBEDO,
                K_S, SPEC_EXP, PLANE_REFL])


def random_scene(seed: int, n_spheres: int, n_lights: int, scale: float,
                 area_lights: int = 0, area_side: float | None = None,
                 plane: bool = True) -> Scene:
    """Spheres with centres U([-5,5]x[0.3,3]x[-5,5])*s, radii U[0.3,1], albedo
    U[0,1]^3, reflectivity U[0,0.5]; lights with x,z U[-5s,5s], y U[5s,8s],
    intensity U[0.5,1].  The last ``area_lights`` lights become square area lights
    of side ``area_side`` (default s)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n_spheres, 8))
    sph = np.zeros((n_spheres, SPHERE_FIELDS), dtype=np.float64)
    sph[:, 0] = (-5.0 + 10.0 * u[:, 0]) * scale
    sph[:, 1] = (0.3 + 2.7 * u[:, 1]) * scale
    sph[:, 2] = (-5.0 + 10.0 * u[:, 2]) * scale
    sph[:, 3] = 0.3 + 0.7 * u[:, 3]
    sph[:, 4:7] = u[:, 4:7]
    sph[:, 7] = K_S
    sph[:, 8] = SPEC_EXP
    sph[:, 9] = 0.5 * u[:, 7]
    ul = rng.random((n_lights, 4))
    lig = np.zeros((n_lights, LIGHT_FIELDS), dtype=np.float64)
    lig[:, 0] = (-5.0 + 10.0 * ul[:, 0]) * scale
    lig[:, 1] = (5.0 + 3.0 * ul[:, 1]) * scale
    lig[:, 2] = (-5.0 + 10.0 * ul[:, 2]) * scale
    lig[:, 3] = 0.5 + 0.5 * ul[:, 3]
    if area_lights:
        lig[n_lights - area_lights:, 4] = scale if area_side is None else area_side
    return Scene(spheres=f32(sph), plane=default_plane() if plane else None,
                 lights=f32(lig), scale=float(scale))


def _params(scene: Scene, **kw) -> Params:
    p = Params(**kw)
    p.eps = float(np.float32(EPS_SCALE * scene.scene_scale))
    return p


# --- the five workloads: names say what they are --------------------------------

def whitted_256() -> Workload:
    """256x256 FP32, 16 spheres + plane, 1 point light, Phong, hard shadows, depth 1."""
    sc = random_scene(1, 16, 1, 1.0)
    return Workload("256x256_16sph_1pt_d1_f32", sc, default_camera(1.0),
                    _params(sc, width=256, height=256, max_depth=1, out_format=OUT_F32, seed=1))


def whitted_720p() -> Workload:
    """1280x720 RGBA8, 64 spheres (box x2) + plane, 2 point lights, depth 4."""
    sc = random_scene(2, 64, 2, 2.0)
    return Workload("1280x720_64sph_2pt_d4_rgba8", sc, default_camera(2.0),
                    _params(sc, width=1280, height=720, max_depth=4, out_format=OUT_RGBA8, seed=2))


def whitted_1080p() -> Workload:
    """1920x1080 RGBA8 variant of the 720p scene (same seed and scene)."""
    w = whitted_720p()
    w.name = "1920x1080_64sph_2pt_d4_rgba8"
    w.params.width, w.params.height = 1920, 1080
    return w


def area_4k() -> Workload:
    """3840x2160 RGBA8, 256 spheres + plane, 3 point lights + 1 square area light
    (16 stratified Philox shadow samples), depth 8."""
    sc = random_scene(3, 256, 4, 4.0, area_lights=1)
    return Workload("3840x2160_256sph_3pt1area16_d8_rgba8", sc, default_camera(4.0),
                    _params(sc, width=3840, height=2160, max_depth=8, shadow_samples=16,
                            out_format=OUT_RGBA8, seed=3))


def area_scene_1080p() -> Workload:
    """The 4K workload's scene, lights and depth at 1920x1080 (a quarter of the
    pixels): the profiling case of the forward kernel."""
    w = area_4k()
    w.name = "1920x1080_256sph_3pt1area16_d8_rgba8"
    w.params.width, w.params.height = 1920, 1080
    return w


def paper_scene(width: int = 1280, height: int = 720, samples: int = 1, depth: int = 1,
                light_radius: float = 0.5) -> Workload:
    """The structure of the paper's benchmark scene (Section 4.1: one light, one
    plane, five spheres; its coordinates and HDR sky are not given): seeded, s = 1,
    one spherical light sampled with `samples` sunflower points (Section 3.6.1; 1
    sample = the light's centre, a hard shadow), reflection bounce limit `depth`,
    Blinn-Phong shading (the paper's final model, Section 3.5.2).  The paper's
    real-time figures use samples 1 / depth 1, its render-only speed-up samples
    200 / depth 3 (Section 4)."""
    sc = random_scene(2305, 5, 1, 1.0)
    sc.lights[:, 5] = light_radius
    name = f"paper_{width}x{height}_5sph_1sphlight_s{samples}_d{depth}_rgba8"
    return Workload(name, sc, default_camera(1.0),
                    _params(sc, width=width, height=height, max_depth=depth, shadow_samples=samples,
                            shading_model=BLINN_PHONG, out_format=OUT_RGBA8, seed=2305))


BATCH_RESOLUTIONS = ((256, 256), (640, 480), (1280, 720), (1920, 1080))


def batch_scenes(n: int = 64, seed0: int = 100) -> list[Workload]:
    """``n`` scenes, seeds seed0..seed0+n-1: sphere count round(exp(U[ln 8, ln 512])),
    1..4 point lights, depth 1..6, resolution uniform over BATCH_RESOLUTIONS, F32 out,
    box scale sqrt(N/16) (the sphere density of the 256x256 scene)."""
    out = []
    for i in range(n):
        seed = seed0 + i
        rng = np.random.Generator(np.random.PCG64(10_000 + seed))
        nsph = int(round(math.exp(rng.uniform(math.log(8.0), math.log(512.0)))))
        nl = int(rng.integers(1, 5))
        depth = int(rng.integers(1, 7))
        w, h = BATCH_RESOLUTIONS[int(rng.integers(0, len(BATCH_RESOLUTIONS)))]
        s = math.sqrt(nsph / 16.0)
        sc = random_scene(seed, nsph, nl, s)
        out.append(Workload(f"batch{i:02d}_{w}x{h}_{nsph}sph_{nl}pt_d{depth}", sc,
                            default_camera(s),
                            _params(sc, width=w, height=h, max_depth=depth,
                                    out_format=OUT_F32, seed=seed)))
    return out


def diff_512() -> Workload:
    """512x512 FP32, 32 spheres + plane, 2 point lights, depth 2 (differentiable)."""
    s = math.sqrt(2.0)
    sc = random_scene(5, 32, 2, s)
    return Workload("512x512_32sph_2pt_d2_f32", sc, default_camera(s),
                    _params(sc, width=512, height=512, max_depth=2, out_format=OUT_F32, seed=5))


def sky_texture(seed: int = 7, width: int = 512, height: int = 256) -> np.ndarray:
    """A seeded synthetic HDR panorama standing in for the paper's sky image (Section
    3.8; the image itself is not available): float32 [height, width, 4], rows from
    the top (latitude +90 deg) down, columns over longitude.  A zenith-to-horizon
    blue gradient, a darker ground below the horizon, low-frequency cloud bands
    (random harmonics in longitude and latitude) and one soft sun of HDR intensity 4
    (about 3.6 deg wide) at a random azimuth and elevation 20-60 deg; alpha 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lat = (0.5 - (np.arange(height) + 0.5) / height) * np.pi          # +pi/2 .. -pi/2
    lon = ((np.arange(width) + 0.5) / width - 0.5) * 2.0 * np.pi       # -pi .. pi
    LON, LAT = np.meshgrid(lon, lat)
    up = np.clip(np.sin(LAT), 0.0, 1.0)[..., None]
    zenith, horizon, ground = np.array([0.22, 0.42, 0.85]), np.array([0.85, 0.82, 0.78]), np.array([0.32, 0.29, 0.25])
    col = np.where(LAT[..., None] >= 0, horizon + (zenith - horizon) * up ** 0.6, ground)
    clouds = np.zeros_like(LAT)
    for _ in range(6):
        kx, ky = rng.integers(1, 6), rng.integers(1, 4)
        clouds += rng.uniform(0.2, 1.0) * np.sin(kx * LON + rng.uniform(0, 2 * np.pi)) * \
            np.cos(ky * LAT * 2 + rng.uniform(0, 2 * np.pi))
    clouds = np.clip(clouds / 3.0, 0.0, 1.0) * (LAT > 0)
    col = col * (1.0 - 0.5 * clouds[..., None]) + 0.9 * clouds[..., None] * 0.5
    az, el = rng.uniform(-np.pi, np.pi), rng.uniform(np.radians(20), np.radians(60))
    sun = np.array([np.cos(el) * np.cos(az), np.sin(el), np.cos(el) * np.sin(az)])
    dirs = np.stack([np.cos(LAT) * np.cos(LON), np.sin(LAT), np.cos(LAT) * np.sin(LON)], -1)
    cosang = np.clip(dirs @ sun, -1.0, 1.0)
    col = col + 4.0 * np.exp(-(1.0 - cosang) / 2e-3)[..., None] * np.array([1.0, 0.95, 0.85])
    out = np.ones((height, width, 4), np.float32)
    out[..., :3] = col
    return f32(out)


def animated_scene(width: int = 1280, height: int = 720) -> tuple[Workload, np.ndarray]:
    """The animated loop: the paper-structure scene (five spheres, one spherical
    light, plane, Blinn-Phong, hard shadows, bounce limit 1: the paper's real-time
    setting) with the synthetic sky, its spheres lifted 1-3 units above their seeded
    places and given a seeded horizontal velocity, to fall and bounce under Verlet
    physics (Section 3.8).  Returns the workload and the previous positions [N, 3]
    (one step of 1/60 s back along the velocity)."""
    w = paper_scene(width, height, 1, 1)
    rng = np.random.Generator(np.random.PCG64(42))
    sph = w.scene.spheres.astype(np.float64).copy()
    n = sph.shape[0]
    sph[:, 1] += rng.uniform(1.0, 3.0, n)
    vel = np.zeros((n, 3))
    vel[:, 0], vel[:, 2] = rng.uniform(-1.0, 1.0, n), rng.uniform(-1.0, 1.0, n)
    prev = sph[:, :3] - vel / 60.0
    w.scene = Scene(spheres=f32(sph), plane=w.scene.plane, lights=w.scene.lights, scale=w.scene.scale,
                    sky=sky_texture())
    w.name = f"animated_{width}x{height}_5sph_1sphlight_sky_d1_rgba8"
    return w, f32(prev)


def perturbed_target(w: Workload, seed: int = 6) -> Scene:
    """Target scene of the inverse-rendering loop: albedo + N(0,0.1) clipped to
    [0,1], k_s + N(0,0.1) clipped to [0,1], reflectivity + N(0,0.05) clipped to
    [0,0.5], light position + N(0,0.5 s), intensity + N(0,0.1) clipped to [0.05,2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sc = w.scene
    sph = sc.spheres.astype(np.float64).copy()
    n = sph.shape[0]
    sph[:, 4:7] = np.clip(sph[:, 4:7] + rng.normal(0, 0.1, (n, 3)), 0.0, 1.0)
    sph[:, 7] = np.clip(sph[:, 7] + rng.normal(0, 0.1, n), 0.0, 1.0)
    sph[:, 9] = np.clip(sph[:, 9] + rng.normal(0, 0.05, n), 0.0, 0.5)
    lig = sc.lights.astype(np.float64).copy()
    nl = lig.shape[0]
    lig[:, 0:3] += rng.normal(0, 0.5 * sc.scale, (nl, 3))
    lig[:, 3] = np.clip(lig[:, 3] + rng.normal(0, 0.1, nl), 0.05, 2.0)
    return Scene(spheres=f32(sph), plane=None if sc.plane is None else sc.plane.copy(),
                 lights=f32(lig), scale=sc.scale)


WORKLOADS = {
    "256": whitted_256,
    "720p": whitted_720p,
    "1080p": whitted_1080p,
    "4k": area_4k,
    "4k_scene_1080p": area_scene_1080p,
    "diff512": diff_512,
}


def pixel_lattice(width: int, height: int, stride: int, seed: int = 0,
                  n_random: int = 0) -> np.ndarray:
    """int32 [n, 2] (x, y): a strided lattice plus seeded random pixels, for
    sampled parity checks on frames too large for the oracle."""
    xs, ys = np.meshgrid(np.arange(0, width, stride), np.arange(0, height, stride))
    pts = [np.stack([xs.ravel(), ys.ravel()], 1)]
    if n_random:
        rng = np.random.Generator(np.random.PCG64(seed))
        pts.append(np.stack([rng.integers(0, width, n_random),
                             rng.integers(0, height, n_random)], 1))
    return np.ascontiguousarray(np.concatenate(pts).astype(np.int32))
