"""rt_render_ws (queued render through the C ABI): every pixel and every hit-record
entry equal, bit for bit, to rt_render's on the same inputs -- the paths handed
over between passes carry their FP32 state exactly -- for full workloads, deep
mirror scenes, workspaces too small for the queues, both output formats, a sky,
the paper's sampled spherical light, and the bounce limits 0 and 16; and the
256x256 workload against the FP64 oracle directly."""
import copy

import numpy as np
import pytest
import torch

from paper_2305_07450_b300 import rt, scenes as S
from parity import compare_f32, oracle_reference

pytestmark = pytest.mark.gpu


def render_pair(w, fmt=None, ws_bytes=None, hitrec=False, launch=None, sky=None, reps=1):
    """(rt_render image, rt_render_ws image, both hit records or None)."""
    p = copy.copy(w.params)
    if fmt is not None:
        p.out_format = fmt
    ds = rt.DeviceScene(w.scene)
    if sky is not None:
        ds.set_sky(sky)
    hb = rt.hitrec_bytes(ds, p) // 4
    # the same fill in both: entries past a path's end other than the id (t, the
    # visibilities) are left as they were by both entry points
    ha = torch.full((hb,), 7.0, device="cuda") if hitrec else None
    hq = torch.full((hb,), 7.0, device="cuda") if hitrec else None
    a = rt.render(ds, w.camera, p, hitrec=ha, launch=launch).clone()
    ws = rt.alloc_workspace(ds, p, ws_bytes)
    ws.fill_(0xA5)  # stale contents: the call must reset what it reads
    n0 = rt.launch_count()
    for _ in range(reps):
        b = rt.render(ds, w.camera, p, hitrec=hq, launch=launch, workspace=ws)
    torch.cuda.synchronize()
    launches = (rt.launch_count() - n0) // reps
    assert rt.device_errors() == 0
    out = (a.cpu().numpy(), b.cpu().numpy(),
           (ha.cpu().numpy(), hq.cpu().numpy()) if hitrec else None, launches)
    ds.close()
    return out


def assert_same(w, **kw):
    a, b, hr, launches = render_pair(w, **kw)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), \
        f"{int((a.view(np.uint32) != b.view(np.uint32)).sum())} words differ"
    if hr is not None:
        assert np.array_equal(hr[0].view(np.uint32), hr[1].view(np.uint32))
    return launches


def small(w, width, height):
    w = copy.deepcopy(w)
    w.params.width, w.params.height = width, height
    return w


def mirror_scene(n=48, seed=11, depth=16):
    """Spheres of reflectivity 0.9..1 packed near the camera's view: most paths
    bounce several times, so every queue pass has work."""
    sc = S.random_scene(seed, n, 2, 0.6)
    sc.spheres[:, 9] = np.random.default_rng(seed).uniform(0.9, 1.0, n).astype(np.float32)
    p = S._params(sc, width=320, height=200, max_depth=depth, out_format=S.OUT_F32, seed=seed)
    return S.Workload("mirror", sc, S.default_camera(0.6), p)


def test_4k_workload_full_frame_equal():
    launches = assert_same(S.area_4k())
    assert launches == S.area_4k().params.max_depth + 1


def test_720p_and_256_workloads_equal_with_hit_records():
    assert_same(S.whitted_720p(), hitrec=True)
    assert_same(S.whitted_256(), hitrec=True)


def test_4k_scene_f32_with_hit_record_equal():
    assert_same(small(S.area_4k(), 480, 270), fmt=S.OUT_F32, hitrec=True)


def test_deep_mirror_paths_equal_both_formats():
    w = mirror_scene()
    assert_same(w, hitrec=True)
    assert_same(w, fmt=S.OUT_RGBA8)


@pytest.mark.parametrize("entries", [0, 1, 37, 1000])
def test_queues_too_small_still_equal(entries):
    """Capacity = (bytes - 256) / 128 paths per queue; overflowing paths are
    finished by the lane holding them."""
    assert_same(mirror_scene(), ws_bytes=256 + 128 * entries, hitrec=True)
    assert_same(small(S.area_4k(), 640, 360), ws_bytes=256 + 128 * entries)


def test_repeated_calls_reuse_the_workspace():
    assert_same(mirror_scene(), reps=3)


def test_bounce_limits_0_and_16():
    w = mirror_scene(depth=0)
    assert assert_same(w) == 1
    assert_same(mirror_scene(depth=16), hitrec=True)


def test_sky_and_sampled_spherical_light_equal():
    assert_same(S.paper_scene(320, 180, 200, 3), sky=S.sky_texture())
    assert_same(S.paper_scene(320, 180, 200, 3), fmt=S.OUT_F32)


def test_blinn_coupled_reflection_equal():
    w = mirror_scene()
    w.params.shading_model = S.BLINN_PHONG
    w.params.refl_coupled, w.params.max_reflectivity = 1, 40.0
    assert_same(w)


def test_hierarchy_and_tiled_loop_ignore_the_workspace():
    assert_same(S.whitted_256(), launch={"staging": 3})
    w = small(S.area_4k(), 320, 180)
    p = copy.copy(w.params)
    ds = rt.DeviceScene(w.scene)
    ds.build_bvh()
    a = rt.render(ds, w.camera, p, launch={"accel": 1}).cpu().numpy()
    b = rt.render(ds, w.camera, p, launch={"accel": 1}, workspace=rt.alloc_workspace(ds, p)).cpu().numpy()
    ds.close()
    assert np.array_equal(a, b)


def test_256_workload_against_oracle():
    w = S.whitted_256()
    p = copy.copy(w.params)
    ds = rt.DeviceScene(w.scene)
    img = rt.render(ds, w.camera, p, workspace=rt.alloc_workspace(ds, p)).cpu().numpy()
    ds.close()
    ref, margin, sens = oracle_reference(w)
    ok, st = compare_f32(img[..., :3].reshape(-1, 3), ref, margin, sens, w.scene.scene_scale)
    assert st["failing"] == 0 and st["frac_within_1e-4"] >= 0.99, st


@pytest.mark.parametrize("entries", [None, 0, 37])
def test_deep_mirror_paths_with_the_line_filter(entries):
    """160 mirror spheres (the line-filter kernels; short queues run one path per
    warp): every pixel and hit-record entry equal to the one-pass kernel's."""
    w = mirror_scene(n=160, seed=12)
    assert_same(w, hitrec=True, ws_bytes=None if entries is None else 256 + 128 * entries)
    assert_same(w, fmt=S.OUT_RGBA8)


def test_maxima_in_wide_passes():
    """16 lights (point, square-area and spherical), 1024 samples per sampled light,
    bounce limit 16, and 128 filler spheres below the plane so that the line-filter
    kernels run: every queue of this small frame is short, so every pass after the
    first takes one path per warp (over 4 000 segments a hit, in chunks of 32 lanes);
    pixels and hit records equal to the one-pass kernel's."""
    from oracle_pins import light, mk, plane_rec, sphere
    rng = np.random.default_rng(16)
    sph = [sphere((0.0, 1.0, 6.0), 3.0, albedo=(0.2, 0.3, 0.9), refl=0.95),
           sphere((0.0, 1.0, -6.0), 3.0, albedo=(0.9, 0.3, 0.2), refl=0.95),
           sphere((-1.2, 0.6, 1.5), 0.5, albedo=(0.3, 0.9, 0.3), refl=0.5),
           sphere((1.3, 1.8, 1.0), 0.4, albedo=(0.9, 0.9, 0.2), refl=0.5)]
    sph += [sphere((float(x), -20.0, float(z)), 0.3) for x in range(-8, 8) for z in range(8)]
    lig = [light((float(rng.uniform(-6, 6)), float(rng.uniform(8, 10)), float(rng.uniform(-3, 3))),
                 float(rng.uniform(0.05, 0.1))) for _ in range(12)]
    lig += [light((-2.0, 9.5, -1.0), 0.2, area=1.0), light((2.5, 9.0, 1.5), 0.2, area=0.7)]
    lig += [light((0.0, 10.0, 0.5), 0.2, srad=0.4), light((-3.0, 9.0, 2.0), 0.2, srad=0.3)]
    sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=0.6), lights=lig, camera=(0, 1, 0, 0, 0, 50),
                    W=20, H=14, D=16, samples=1024, seed=99)
    p.eps = 5e-4
    p.out_format = S.OUT_F32
    assert sc.n_spheres >= 128
    assert_same(S.Workload("max_wide", sc, cam, p), hitrec=True)
