"""Rendering through the sphere hierarchy (launch accel = 1) gives the brute-force
images bit for bit: same closest hits (ties to the lower index), same shadow
verdicts, same arithmetic -- on the workloads, on the small edge cases, on a
scene beyond shared memory, with far cameras and grazing rays; plus the
staleness rules of device-side updates."""
import copy

import numpy as np
import pytest
import torch

from oracle_pins import light, mk, plane_rec, sphere
from paper_2305_07450_b300 import rt, scenes as S
from parity import compare_f32, oracle_reference
from test_render_gpu import small_cases

pytestmark = pytest.mark.gpu
ACC = {"accel": 1}


def both(w, fmt=None, launch_bf=None, launch_acc=None, hitrec=False):
    p = copy.copy(w.params)
    if fmt is not None:
        p.out_format = fmt
    ds = rt.DeviceScene(w.scene)
    info = ds.build_bvh()
    out = []
    for launch in (launch_bf, {**ACC, **(launch_acc or {})}):
        # zeroed: after a miss only the id of the later bounces is written
        hr = torch.zeros(rt.hitrec_bytes(ds, p) // 4, dtype=torch.float32, device="cuda") if hitrec else None
        img = rt.render(ds, w.camera, p, launch=launch, hitrec=hr)
        torch.cuda.synchronize()
        out.append((img.cpu().numpy(), hr.cpu().numpy() if hr is not None else None))
    assert rt.device_errors() == 0
    ds.close()
    return out[0], out[1], info


def assert_same(w, **kw):
    (a, ha), (b, hb), info = both(w, **kw)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), (w.name, info)
    if ha is not None:
        assert np.array_equal(ha.view(np.uint32), hb.view(np.uint32))
    return info


@pytest.mark.parametrize("fmt", [S.OUT_F32, S.OUT_RGBA8])
def test_whitted_256_and_720p(fmt):
    assert_same(S.whitted_256(), fmt=fmt, hitrec=True)
    assert_same(S.whitted_720p(), fmt=fmt)


def test_4k_area_light_full_frame():
    """The 3840x2160 workload (256 spheres, 16 area samples, depth 8), every pixel."""
    info = assert_same(S.area_4k())
    print(info)


def test_4k_scene_hit_record_equal():
    w = S.area_4k()
    w.params.width, w.params.height = 480, 270
    assert_same(w, fmt=S.OUT_F32, hitrec=True)


@pytest.mark.parametrize("name", sorted(small_cases()))
def test_small_cases(name):
    sc, cam, p = small_cases()[name]
    p.eps = 5e-4
    assert_same(S.Workload(name, sc, cam, p), fmt=S.OUT_F32, hitrec=True)


def test_paper_scene_soft_shadows():
    assert_same(S.paper_scene(320, 180, 200, 3), fmt=S.OUT_F32)


def test_launch_shapes_and_staging():
    w = S.whitted_720p()
    w.params.width, w.params.height = 200, 120
    for cfg in ({"staging": 2}, {"block_x": 8, "block_y": 4}, {"block_x": 32, "block_y": 8},
                {"block_x": 8, "block_y": 32, "staging": 2}):
        assert_same(w, launch_acc=cfg)


def test_large_scene_from_global_memory():
    """20000 spheres: neither the table nor the hierarchy fits shared memory, so
    both are read through the caches; brute force takes the tiled loop."""
    sc = S.random_scene(77, 20000, 2, 35.0)
    w = S.Workload("20000sph", sc, S.default_camera(35.0),
                   S._params(sc, width=160, height=96, max_depth=2, out_format=S.OUT_F32, seed=77))
    info = assert_same(w, hitrec=True)
    assert info["n_nodes"] > 1000


def test_far_narrow_camera_and_grazing_rays():
    """A camera 4000 units away with a 1.5 degree field of view over 4096 small
    spheres: ray origins far from the boxes, nearly parallel rays, many grazing
    hits -- where an under-widened box would drop a hit."""
    rng = np.random.Generator(np.random.PCG64(11))
    n = 4096
    sph = np.zeros((n, 10))
    sph[:, :3] = rng.uniform(-20, 20, (n, 3))
    sph[:, 1] = np.abs(sph[:, 1]) + 0.5
    sph[:, 3] = rng.uniform(0.02, 0.6, n)
    sph[:, 4:7] = rng.random((n, 3))
    sph[:, 7], sph[:, 8], sph[:, 9] = 0.5, 32.0, rng.uniform(0, 0.5, n)
    sc = S.Scene(spheres=S.f32(sph), plane=S.default_plane(), lights=S.f32([light((5, 200, -30), 0.9)]),
                 scale=20.0)
    for cam in ([0.0, 300.0, -4000.0, 0.0, -4.0, 1.5], [3.7, 10.0, -60.0, 12.0, -3.0, 75.0]):
        p = S._params(sc, width=320, height=240, max_depth=3, out_format=S.OUT_F32, seed=5)
        assert_same(S.Workload("far", sc, S.f32(cam), p), hitrec=True)


def test_equal_distance_ties_keep_the_lower_index():
    """Coincident spheres of different colours: both paths keep the lowest index."""
    sph = [sphere((0, 1, 0), 1.0, albedo=(1, 0, 0)), sphere((0, 1, 0), 1.0, albedo=(0, 1, 0)),
           sphere((2.5, 1, 0), 0.7, albedo=(0, 0, 1)), sphere((2.5, 1, 0), 0.7, albedo=(1, 1, 0))]
    sph += [sphere((-3 + 0.5 * i, 0.4, 3), 0.3) for i in range(12)]
    sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=0.3), lights=[light((3, 8, -4), 0.9)],
                    camera=(0, 2, -8, 0, -10, 60), W=96, H=64, D=2)
    w = S.Workload("ties", sc, cam, p)
    (a, ha), (b, hb), _ = both(w, fmt=S.OUT_F32, hitrec=True)
    assert np.array_equal(a, b) and np.array_equal(ha.view(np.uint32), hb.view(np.uint32))
    ids = ha.reshape(p.max_depth + 1, 3, 64, 96)[0, 0].view(np.int32)
    assert 0 in ids and 1 not in ids and 2 in ids and 3 not in ids


def test_oracle_parity_through_the_hierarchy():
    w = S.whitted_256()
    ds = rt.DeviceScene(w.scene)
    ds.build_bvh()
    p = copy.copy(w.params)
    p.out_format = S.OUT_F32
    img = rt.render(ds, w.camera, p, launch=ACC).cpu().numpy()
    ref, margin, sens = oracle_reference(w)
    ok, st = compare_f32(img[..., :3].reshape(-1, 3), ref, margin, sens, w.scene.scene_scale)
    assert st["failing"] == 0, st


def test_regions_stitch():
    from paper_2305_07450_b300 import shard
    w = S.area_4k()
    w.params.width, w.params.height = 640, 360
    ds = rt.DeviceScene(w.scene)
    ds.build_bvh()
    full = rt.render(ds, w.camera, w.params).cpu().numpy()
    parts = [rt.render_region(ds, w.camera, w.params, 0, a, w.params.width, b - a, launch=ACC).cpu().numpy()
             for a, b in shard.row_bands(w.params.height, 3)]
    assert np.array_equal(np.concatenate(parts, 0), full)


def test_staleness_rules():
    """No hierarchy -> refused; a device-side update makes it stale (refused); a
    host-side update rebuilds it and the images match brute force again."""
    w = S.whitted_256()
    ds = rt.DeviceScene(w.scene)
    with pytest.raises(rt.RtError) as e:
        rt.render(ds, w.camera, w.params, launch=ACC)
    assert e.value.status == 4
    ds.build_bvh()
    rt.render(ds, w.camera, w.params, launch=ACC)
    moved = copy.deepcopy(w.scene)
    moved.spheres[:, 0] += np.float32(0.75)
    ds.update(spheres=torch.from_numpy(moved.spheres).cuda(), plane=torch.from_numpy(moved.plane).cuda(),
              lights=torch.from_numpy(moved.lights).cuda())
    with pytest.raises(rt.RtError) as e:
        rt.render(ds, w.camera, w.params, launch=ACC)
    assert e.value.status == 4
    with pytest.raises(rt.RtError):
        ds.build_bvh()  # the host copy no longer holds the device contents
    ds.update(moved)
    a = rt.render(ds, w.camera, w.params).cpu().numpy()
    b = rt.render(ds, w.camera, w.params, launch=ACC).cpu().numpy()
    assert np.array_equal(a, b)
    # the tiled loop is a brute-force schedule
    with pytest.raises(rt.RtError) as e:
        rt.render(ds, w.camera, w.params, launch={"accel": 1, "staging": 3})
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    ds.close()
