"""Parity of the CUDA forward render (rt_render through the C ABI) with the FP64
oracle, element by element on the same seeded inputs."""
import copy

import numpy as np
import pytest
import torch

import oracle
from oracle_pins import light, mk, plane_rec, sphere
from paper_2305_07450_b300 import rt, scenes as S
from parity import compare_f32, compare_rgba8, oracle_reference

pytestmark = pytest.mark.gpu


def gpu_render(w, launch=None, hitrec=False, fmt=None):
    p = copy.copy(w.params)
    if fmt is not None:
        p.out_format = fmt
    ds = rt.DeviceScene(w.scene)
    hr = None
    if hitrec:
        hr = torch.empty(rt.hitrec_bytes(ds, p) // 4, dtype=torch.float32, device="cuda")
    img = rt.render(ds, w.camera, p, launch=launch, hitrec=hr)
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    out = img.cpu().numpy()
    ds.close()
    return (out, hr.cpu().numpy() if hr is not None else None)


def as_workload(name, sc, cam, p):
    return S.Workload(name, sc, cam, p)


def check_f32_full(w, min_plain=0.99):
    img, _ = gpu_render(w, fmt=S.OUT_F32)
    ref, margin, sens = oracle_reference(w)
    ok, st = compare_f32(img[..., :3].reshape(-1, 3), ref, margin, sens, w.scene.scene_scale)
    print(w.name, st)
    assert st["failing"] == 0, st
    assert st["frac_within_1e-4"] >= min_plain, st
    assert np.all(img[..., 3] == 1.0)
    return st


def test_whitted_256_full_frame():
    """256x256, 16 spheres, 1 point light, depth 1: every pixel."""
    check_f32_full(S.whitted_256(), min_plain=0.999)


def small_cases():
    cam = (0, 2.5, -8, 0, -15, 60)
    sph = [sphere((-1.5, 1, 0), 1.0, albedo=(0.9, 0.2, 0.2), refl=0.3),
           sphere((1.2, 0.8, 1.0), 0.8, albedo=(0.2, 0.9, 0.3), refl=0.5),
           sphere((0.2, 2.2, 2.5), 0.6, albedo=(0.3, 0.3, 0.9), refl=0.1)]
    lig = [light((3, 6, -2), 0.8), light((-4, 5, 1), 0.6)]
    cases = {
        "empty": mk(camera=cam, W=8, H=8),
        "no_lights_ambient": mk(spheres=sph, plane=plane_rec(refl=0.25), camera=cam, W=24, H=16, D=2),
        "plane_only": mk(plane=plane_rec(), lights=lig, camera=cam, W=16, H=16),
        "depth0": mk(spheres=sph, plane=plane_rec(), lights=lig, camera=cam, W=40, H=24, D=0),
        "ragged_37x23_d3": mk(spheres=sph, plane=plane_rec(refl=0.25), lights=lig, camera=cam, W=37, H=23, D=3),
        "one_pixel": mk(spheres=sph, plane=plane_rec(), lights=lig, camera=cam, W=1, H=1, D=2),
        "portrait_30x50": mk(spheres=sph, plane=plane_rec(refl=0.25), lights=lig, camera=cam, W=30, H=50, D=2),
        "blinn": mk(spheres=sph, plane=plane_rec(refl=0.25), lights=lig, camera=cam, W=48, H=32, D=2,
                    model=S.BLINN_PHONG),
        "area_light": mk(spheres=sph, plane=plane_rec(refl=0.25), lights=lig + [light((0, 6, 0), 0.9, area=1.5)],
                         camera=cam, W=48, H=32, D=2, samples=16, seed=77),
        "sphere_light": mk(spheres=sph, plane=plane_rec(refl=0.25), lights=[light((0, 6, 0), 0.9, srad=0.7)],
                           camera=cam, W=48, H=32, D=1, samples=20),
        "no_plane_deep": mk(spheres=sph, lights=lig, camera=cam, W=32, H=32, D=8),
        "coupled_reflectivity": mk(spheres=sph, plane=plane_rec(refl=0.25), lights=lig, camera=cam, W=40, H=32,
                                   D=3, model=S.BLINN_PHONG),
    }
    cases["coupled_reflectivity"][2].refl_coupled = 1
    cases["coupled_reflectivity"][2].max_reflectivity = 64.0
    return cases


@pytest.mark.parametrize("name", sorted(small_cases()))
def test_small_case(name):
    sc, cam, p = small_cases()[name]
    p.eps = 5e-4
    check_f32_full(as_workload(name, sc, cam, p), min_plain=0.98)


def test_empty_scene_is_black():
    sc, cam, p = small_cases()["empty"]
    img, _ = gpu_render(as_workload("e", sc, cam, p), fmt=S.OUT_F32)
    assert np.all(img[..., :3] == 0.0)


def sampled(w, n_lattice_stride, n_random, fmt):
    img, _ = gpu_render(w, fmt=fmt)
    px = S.pixel_lattice(w.params.width, w.params.height, n_lattice_stride, seed=3, n_random=n_random)
    ref, margin, sens = oracle_reference(w, px)
    g = img[px[:, 1], px[:, 0]]
    return g, ref, margin, sens


def test_720p_rgba8_sampled():
    """1280x720 RGBA8, 64 spheres, 2 lights, depth 4: lattice + random pixels."""
    w = S.whitted_720p()
    g, ref, margin, sens = sampled(w, 23, 1500, S.OUT_RGBA8)
    ok, st = compare_rgba8(g, ref, margin, sens, w.scene.scene_scale)
    print(st)
    assert st["failing"] == 0 and st["frac_within_1lsb"] >= 0.999, st


def test_720p_f32_sampled():
    w = S.whitted_720p()
    g, ref, margin, sens = sampled(w, 41, 800, S.OUT_F32)
    ok, st = compare_f32(g[:, :3], ref, margin, sens, w.scene.scene_scale)
    print(st)
    assert st["failing"] == 0 and st["frac_within_1e-4"] >= 0.98, st


def test_4k_area_light_sampled():
    """3840x2160 RGBA8, 256 spheres, 3 point + 1 area light (16 Philox samples),
    depth 8, through the one-pass kernel (rt_render) at the library's default
    launch; sampled pixels.  The bench's path (rt_render_ws at the tuned launch)
    is compared over every pixel in test_fullframe_gpu.py."""
    w = S.area_4k()
    g, ref, margin, sens = sampled(w, 191, 600, S.OUT_RGBA8)
    ok, st = compare_rgba8(g, ref, margin, sens, w.scene.scene_scale)
    print(st)
    assert st["failing"] == 0 and st["frac_within_1lsb"] >= 0.995, st


def test_4k_f32_sampled():
    w = S.area_4k()
    g, ref, margin, sens = sampled(w, 257, 300, S.OUT_F32)
    ok, st = compare_f32(g[:, :3], ref, margin, sens, w.scene.scene_scale)
    print(st)
    assert st["failing"] == 0 and st["frac_within_1e-4"] >= 0.95, st


def test_launch_shapes_and_staging_bitwise_equal():
    w = S.whitted_720p()
    w.params.width, w.params.height = 200, 120
    base, _ = gpu_render(w, launch={"block_x": 16, "block_y": 16, "staging": 1})
    for cfg in ({"block_x": 16, "block_y": 16, "staging": 2}, {"block_x": 8, "block_y": 4},
                {"block_x": 32, "block_y": 8}, {"block_x": 8, "block_y": 32}, {"staging": 3},
                {"block_x": 8, "block_y": 4, "staging": 3}):
        other, _ = gpu_render(w, launch=cfg)
        assert np.array_equal(base, other), cfg


def test_large_scene_takes_the_tiled_loop():
    """20000 spheres: the geometry table (320 KB) exceeds shared memory, so every
    warp stages it chunk by chunk; parity with the oracle on a small frame."""
    sc = S.random_scene(77, 20000, 2, 35.0)
    w = S.Workload("20000sph", sc, S.default_camera(35.0),
                   S._params(sc, width=48, height=32, max_depth=1, out_format=S.OUT_F32, seed=77))
    check_f32_full(w, min_plain=0.99)
    img_auto, _ = gpu_render(w)
    img_forced, _ = gpu_render(w, launch={"staging": 3, "block_x": 8, "block_y": 8})
    assert np.array_equal(img_auto, img_forced)


def test_rgba8_is_quantised_f32():
    """RGBA8 output = the FP32 output quantised by the same FP32 rule."""
    w = S.whitted_720p()
    w.params.width, w.params.height = 203, 117
    f, _ = gpu_render(w, fmt=S.OUT_F32)
    q, _ = gpu_render(w, fmt=S.OUT_RGBA8)
    v = np.clip(f[..., :3].astype(np.float32), np.float32(0), np.float32(1))
    codes = np.floor((v * np.float32(255.0)).astype(np.float32) + np.float32(0.5)).astype(np.uint32)
    want = codes[..., 0] | (codes[..., 1] << 8) | (codes[..., 2] << 16) | np.uint32(0xFF000000)
    assert np.array_equal(q.astype(np.uint32), want)


def test_deterministic():
    w = S.whitted_256()
    a, _ = gpu_render(w)
    b, _ = gpu_render(w)
    assert np.array_equal(a, b)


def test_hitrec_primary_hits_match_oracle():
    w = S.whitted_256()
    w.params.width = w.params.height = 64
    img, hr = gpu_render(w, hitrec=True)
    H, W, L = 64, 64, w.scene.n_lights
    rec = hr.reshape(w.params.max_depth + 1, 2 + L, H, W)
    ids = rec[0, 0].view(np.int32)
    ts = rec[0, 1]
    bad = 0
    for y in range(H):
        for x in range(W):
            o, d = oracle.primary_ray(w.scene, w.camera, w.params, x, y)
            i, t = oracle.closest(w.scene, w.camera, w.params, o, d)
            if ids[y, x] != i:
                bad += 1
            elif i >= 0:
                assert abs(ts[y, x] - t) < 1e-4 * max(1.0, t)
    assert bad <= 3


def test_device_error_word_clear_after_renders():
    gpu_render(S.whitted_256())
    assert rt.device_errors() == 0


def test_region_bands_stitch_bit_identical():
    """Row bands and an interior rectangle rendered by rt_render_region equal the
    same pixels of the full frame (RGBA8 and F32), as used to split a frame over
    GPUs."""
    from paper_2305_07450_b300 import shard
    for fmt in (S.OUT_RGBA8, S.OUT_F32):
        w = S.area_4k()
        w.params.width, w.params.height, w.params.out_format = 640, 360, fmt
        ds = rt.DeviceScene(w.scene)
        full = rt.render(ds, w.camera, w.params).cpu().numpy()
        parts = [shard.render_band(ds, w.camera, w.params, a, b).cpu().numpy()
                 for a, b in shard.row_bands(w.params.height, 3)]
        assert np.array_equal(np.concatenate(parts, 0), full)
        sub = rt.render_region(ds, w.camera, w.params, 104, 50, 203, 77).cpu().numpy()
        assert np.array_equal(sub, full[50:127, 104:307])


@pytest.mark.parametrize("samples,depth", [(1, 1), (200, 3)])
def test_paper_scene_soft_shadows(samples, depth):
    """The paper's scene structure with its two settings: hard shadows (1 sample)
    at bounce 1, and 200 sunflower samples at bounce 3 (Sections 3.6.1, 4)."""
    w = S.paper_scene(128, 72, samples, depth)
    check_f32_full(w, min_plain=0.995)


def test_maximum_lights_samples_and_depth():
    """The ABI's maxima at once: 16 lights (point, square-area and spherical), 1024
    shadow samples per sampled light, bounce limit 16 -- two large mirror spheres
    facing each other along the view axis send the central ray through all 16
    reflections; every pixel against the oracle."""
    rng = np.random.default_rng(16)
    sph = [sphere((0.0, 1.0, 6.0), 3.0, albedo=(0.2, 0.3, 0.9), refl=0.95),
           sphere((0.0, 1.0, -6.0), 3.0, albedo=(0.9, 0.3, 0.2), refl=0.95),
           sphere((-1.2, 0.6, 1.5), 0.5, albedo=(0.3, 0.9, 0.3), refl=0.5),
           sphere((1.3, 1.8, 1.0), 0.4, albedo=(0.9, 0.9, 0.2), refl=0.5),
           sphere((0.8, 0.4, -1.4), 0.35, albedo=(0.8, 0.2, 0.8), refl=0.5)]
    lig = [light((float(rng.uniform(-6, 6)), float(rng.uniform(8, 10)), float(rng.uniform(-3, 3))),
                 float(rng.uniform(0.05, 0.1))) for _ in range(12)]
    lig += [light((-2.0, 9.5, -1.0), 0.2, area=1.0), light((2.5, 9.0, 1.5), 0.2, area=0.7)]
    lig += [light((0.0, 10.0, 0.5), 0.2, srad=0.4), light((-3.0, 9.0, 2.0), 0.2, srad=0.3)]
    assert len(lig) == 16
    sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=0.6), lights=lig, camera=(0, 1, 0, 0, 0, 50),
                    W=20, H=14, D=16, samples=1024, seed=99)
    p.eps = 5e-4
    w = as_workload("max_lights_samples_depth", sc, cam, p)
    check_f32_full(w, min_plain=0.97)
    img, hr = gpu_render(w, hitrec=True)
    rec = hr.reshape(p.max_depth + 1, 2 + 16, p.height, p.width)
    assert rec[16, 0, 7, 10].view(np.int32) >= 0        # the axial ray is still hitting at bounce 16


def test_maximum_frame_dimensions():
    """Frames at the ABI's 32768-pixel limit: a 32768 x 8 strip (every pixel
    rendered, sampled parity) and 64 x 4 regions at the corners of a 32768 x 32768
    frame (the NDC of the full frame), against the oracle."""
    w = S.whitted_256()
    w.params.width, w.params.height = 32768, 8
    img, _ = gpu_render(w, fmt=S.OUT_F32)
    px = S.pixel_lattice(w.params.width, w.params.height, 997, seed=5, n_random=200)
    ref, margin, sens = oracle_reference(w, px)
    ok, st = compare_f32(img[px[:, 1], px[:, 0], :3], ref, margin, sens, w.scene.scene_scale)
    assert st["failing"] == 0, st
    w = S.whitted_256()
    w.params.width = w.params.height = 32768
    w.params.out_format = S.OUT_F32
    ds = rt.DeviceScene(w.scene)
    for x0, y0 in ((0, 0), (32768 - 64, 32768 - 4), (16384, 16382)):
        sub = rt.render_region(ds, w.camera, w.params, x0, y0, 64, 4).cpu().numpy()
        xs, ys = np.meshgrid(np.arange(x0, x0 + 64), np.arange(y0, y0 + 4))
        px = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
        ref, margin, sens = oracle_reference(w, px)
        ok, st = compare_f32(sub[..., :3].reshape(-1, 3), ref, margin, sens, w.scene.scene_scale)
        assert st["failing"] == 0, (x0, y0, st)
    ds.close()


def test_lean_kernels_follow_the_light_kinds():
    """The line-filter kernels built without the spherical-light sample code run only
    while the host knows the scene has no spherical light.  A scene that gains one by
    a host-side update, or by a device-side update (the light kinds are unknown from
    then on), renders exactly as a fresh upload of it does, in one pass and queued,
    and matches the oracle on a lattice of pixels; a host-side update that takes the
    light away again renders as the scene did before."""
    base = S.random_scene(11, 256, 3, 4.0)
    p = S._params(base, width=160, height=96, max_depth=3, shadow_samples=16, out_format=S.OUT_F32, seed=11)
    cam = S.default_camera(4.0)
    lit = copy.deepcopy(base)
    lit.lights[0, 5] = np.float32(1.5)  # light 0 becomes a sphere of radius 1.5
    launches = (None, {"block_x": 8, "block_y": 32, "queued": 1, "staging": 1})

    def frames(ds):
        out = [rt.render(ds, cam, p, launch=L).cpu().numpy() for L in launches]
        torch.cuda.synchronize()
        assert rt.device_errors() == 0
        return out

    fresh = rt.DeviceScene(lit)
    want = frames(fresh)
    fresh.close()
    assert np.array_equal(want[0], want[1])
    plain = rt.DeviceScene(base)
    before = frames(plain)
    assert not np.array_equal(before[0], want[0])  # the light's change shows
    plain.update(lit)
    for a, b in zip(frames(plain), want):
        assert np.array_equal(a, b)
    plain.update(base)  # the light kinds follow the host description back
    for a, b in zip(frames(plain), before):
        assert np.array_equal(a, b)
    plain.close()
    dev = rt.DeviceScene(base)
    frames(dev)
    dev.update(spheres=torch.from_numpy(lit.spheres).cuda(), plane=torch.from_numpy(lit.plane).cuda(),
               lights=torch.from_numpy(lit.lights).cuda())
    for a, b in zip(frames(dev), want):
        assert np.array_equal(a, b)
    dev.close()
    w = S.Workload("lean_light_kinds", lit, cam, p)
    px = S.pixel_lattice(p.width, p.height, 7, seed=11, n_random=64)
    ref, margin, sens = oracle_reference(w, px)
    got = want[0][px[:, 1], px[:, 0], :3].reshape(-1, 3)
    ok, st = compare_f32(got, ref, margin, sens, lit.scene_scale)
    assert st["failing"] == 0, st


@pytest.mark.parametrize("samples,depth", [(200, 3), (16, 2)])
def test_cleared_sampled_lights_equal_the_traced_ones(samples, depth):
    """Scenes below the line filter's size with a sampled light take light_clear: a
    light whose every segment is proved unblocked is attributed visibility 1 without
    tracing.  The tiled loop traces every segment; pixels and hit records must be
    the same bit for bit (the paper scene's spherical light, and a square area light)."""
    w = S.paper_scene(160, 90, samples, depth)
    from oracle_pins import light, mk, plane_rec, sphere
    cam = (0, 2.5, -8, 0, -15, 60)
    sph = [sphere((-1.5, 1, 0), 1.0, albedo=(0.9, 0.2, 0.2), refl=0.3),
           sphere((1.2, 0.8, 1.0), 0.8, albedo=(0.2, 0.9, 0.3), refl=0.5)]
    area = mk(spheres=sph, plane=plane_rec(refl=0.25), lights=[light((3, 6, -2), 0.8), light((0, 6, 0), 0.9, area=1.5)],
              camera=cam, W=96, H=64, D=depth, samples=int(samples ** 0.5) ** 2, seed=5)  # square strata
    for sc, camera, p in ((w.scene, w.camera, w.params), area):
        p = copy.copy(p)
        p.out_format = S.OUT_F32
        ds = rt.DeviceScene(sc)
        nb = rt.hitrec_bytes(ds, p) // 4
        h1 = torch.zeros(nb, device="cuda")
        h3 = torch.zeros(nb, device="cuda")
        a = rt.render(ds, camera, p, launch={"staging": 1}, hitrec=h1).cpu().numpy()
        b = rt.render(ds, camera, p, launch={"staging": 3}, hitrec=h3).cpu().numpy()
        torch.cuda.synchronize()
        assert rt.device_errors() == 0
        ds.close()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        assert np.array_equal(h1.cpu().numpy().view(np.uint32), h3.cpu().numpy().view(np.uint32))
