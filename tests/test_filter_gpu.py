"""The line filter in front of the shadow-segment test (scenes of 128 spheres or
more) changes no verdict: every pixel and hit-record entry equals, bit for bit,
the tiled loop's (staging 3), which runs the segment test alone -- on scenes made to
stress the filter's bound: overlapping clusters (shadow origins inside other
spheres), tangent and near-tangent spheres around shadow segments, a light so far
away that |V|^2 passes 2^100 (the group falls back to the segment test), spheres
so far away that |oc|^2 overflows, a radius whose square overflows, and sampled
square and spherical lights."""
import copy

import numpy as np
import pytest
import torch

from oracle_pins import light, mk, plane_rec, sphere
from paper_2305_07450_b300 import rt, scenes as S

pytestmark = pytest.mark.gpu


def render(sc, cam, p, launch, workspace=False):
    ds = rt.DeviceScene(sc)
    hr = torch.full((rt.hitrec_bytes(ds, p) // 4,), 3.0, device="cuda")
    ws = rt.alloc_workspace(ds, p) if workspace else None
    img = rt.render(ds, cam, p, launch=launch, hitrec=hr, workspace=ws)
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    out = img.cpu().numpy().view(np.uint32).copy(), hr.cpu().numpy().view(np.uint32).copy()
    ds.close()
    return out


def assert_filter_exact(sc, cam, p):
    assert sc.n_spheres >= 128  # the filtered path
    p = copy.copy(p)
    p.out_format = S.OUT_F32
    ref_img, ref_hr = render(sc, cam, p, {"staging": 3})
    for launch, ws in (({"staging": 1}, False), ({"staging": 2, "block_x": 8, "block_y": 16}, False),
                       ({"staging": 1}, True)):
        img, hr = render(sc, cam, p, launch, ws)
        assert np.array_equal(img, ref_img), (launch, ws, int((img != ref_img).sum()))
        assert np.array_equal(hr, ref_hr), (launch, ws)


def cluster_scene(seed=3, n=160):
    """Clumps of overlapping spheres on a plane, a point light and a square light."""
    rng = np.random.default_rng(seed)
    sph = []
    for c in rng.uniform(-4, 4, (n // 8, 2)):
        for _ in range(8):
            off = rng.normal(0, 0.35, 3)
            sph.append(sphere((c[0] + off[0], 0.6 + abs(off[1]), c[1] + off[2]), rng.uniform(0.25, 0.6),
                              albedo=tuple(rng.random(3)), refl=rng.uniform(0, 0.5)))
    return mk(spheres=sph, plane=plane_rec(refl=0.2), lights=[light((2, 9, -3), 0.8), light((-1, 10, 1), 0.7, 2.0)],
              camera=(0, 6, -14, 0, -20, 55), W=192, H=128, D=3, samples=16, seed=9)


def test_overlapping_clusters():
    assert_filter_exact(*cluster_scene())


def test_tangent_spheres_around_shadow_segments():
    """Spheres placed tangent (and 1e-6 off tangent, both sides) to the segments
    from a grid of plane points to a point light, plus filler to 128 spheres."""
    L = np.array([0.0, 8.0, 0.0])
    sph = []
    rng = np.random.default_rng(5)
    for i, px in enumerate(np.linspace(-3, 3, 7)):
        for j, pz in enumerate(np.linspace(-3, 3, 7)):
            p0 = np.array([px, 0.0, pz])
            v = L - p0
            a = 0.3 + 0.1 * ((i + j) % 3)               # point along the segment
            q = p0 + a * v
            side = np.cross(v, [1.0, 0.0, 0.0])
            side /= np.linalg.norm(side)
            r = 0.2
            delta = (-1e-6, 0.0, 1e-6)[(i * 7 + j) % 3]
            c = q + side * (r + delta)
            sph.append(sphere(tuple(c), r, albedo=tuple(rng.random(3))))
    while len(sph) < 128:
        sph.append(sphere((rng.uniform(-6, 6), rng.uniform(0.5, 3), rng.uniform(6, 12)), rng.uniform(0.2, 0.5)))
    sc, cam, p = mk(spheres=sph, plane=plane_rec(), lights=[light(tuple(L), 0.9)],
                    camera=(0, 7, -9, 0, -35, 60), W=256, H=192, D=1)
    assert_filter_exact(sc, cam, p)


def test_light_beyond_the_filter_range():
    """|V|^2 > 2^100: the groups take the segment test throughout."""
    sc, cam, p = cluster_scene(seed=4)
    sc.lights[0, :3] = S.f32([3e15, 1e16, -2e15])
    assert_filter_exact(sc, cam, p)


def test_huge_coordinates_and_radius():
    """Spheres 1e20 away (|oc|^2 overflows FP32) and one whose r^2 overflows."""
    sc, cam, p = cluster_scene(seed=6)
    sph = sc.spheres.copy()
    sph[:6, 0] = S.f32([1e20, -1e20, 3e19, 1e20, -5e19, 2e20])
    sph[:6, 2] = S.f32([1e20, 1e20, -1e20, -2e20, 5e19, 0.0])
    sph[6, :4] = S.f32([4e21, 0.0, 0.0, 2e19])          # r^2 = inf in FP32
    sc.spheres = sph
    assert_filter_exact(sc, cam, p)


def test_sampled_spherical_light_and_4k_scene_crop():
    sc, cam, p = cluster_scene(seed=8)
    sc.lights[1, 4], sc.lights[1, 5] = 0.0, 0.8          # spherical light, 16 sunflower samples
    p.shading_model = S.BLINN_PHONG
    assert_filter_exact(sc, cam, p)
    w = S.area_4k()
    w.params.width, w.params.height = 480, 270
    assert_filter_exact(w.scene, w.camera, w.params)


# ---- the cone pre-pass of sampled lights (cone_pass): skipped sphere blocks change
# no verdict.  Every case below is compared with the tiled loop, which has neither
# the filter nor the pre-pass.

def test_cone_boundary_shell_of_a_square_light():
    """Spheres tangent to the segments from plane points to the corners of a square
    light (the cone's boundary), pushed 1e-3, 1e-6 or 0 outwards or inwards, plus
    filler: blocks just inside and just outside every lane's cone."""
    L, side = np.array([0.5, 9.0, -0.5]), 3.0
    corners = [L + np.array([sx * side / 2, 0.0, sz * side / 2]) for sx in (-1, 1) for sz in (-1, 1)]
    rng = np.random.default_rng(11)
    sph = []
    deltas = (-1e-3, -1e-6, 0.0, 1e-6, 1e-3)
    for i, px in enumerate(np.linspace(-3, 3, 6)):
        for j, pz in enumerate(np.linspace(-3, 3, 6)):
            p0 = np.array([px, 0.0, pz])
            axis = L - p0
            axis /= np.linalg.norm(axis)
            k = (i * 6 + j) % 4
            v = corners[k] - p0
            a = 0.25 + 0.15 * ((i + 2 * j) % 4)
            q = p0 + a * v
            out = np.cross(np.cross(axis, v), v)        # perpendicular to v, away from the axis
            out *= -np.sign(np.dot(out, axis)) / np.linalg.norm(out)
            r = float(rng.uniform(0.1, 0.4))
            c = q + out * (r + deltas[(i + j) % 5])
            sph.append(sphere(tuple(c), r, albedo=tuple(rng.random(3)), refl=0.3))
    while len(sph) < 160:
        sph.append(sphere((rng.uniform(-6, 6), rng.uniform(0.4, 4), rng.uniform(-6, 6)), rng.uniform(0.15, 0.7),
                          albedo=tuple(rng.random(3)), refl=rng.uniform(0, 0.5)))
    sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=0.2),
                    lights=[light((-4, 8, 3), 0.6), light(tuple(L), 0.9, side)],
                    camera=(0, 7, -10, 0, -32, 60), W=256, H=176, D=3, samples=16, seed=21)
    assert_filter_exact(sc, cam, p)


def test_cone_spherical_light_near_the_scene():
    """A spherical light whose radius is close to its distance from part of the
    scene: lanes of one warp with and without a usable cone."""
    sc, cam, p = cluster_scene(seed=12)
    L, R = np.array([0.3, 2.4, -0.2]), 1.4
    sph = sc.spheres.astype(np.float64)
    keep = np.linalg.norm(sph[:, :3] - L, axis=1) - R > sph[:, 3] + 0.05   # the light outside every sphere
    sph = sph[keep]
    rng = np.random.default_rng(12)
    while len(sph) < 128:
        sph = np.vstack([sph, sphere((rng.uniform(-6, 6), rng.uniform(0.5, 2), rng.uniform(6, 10)), 0.4)])
    sc.spheres = S.f32(sph)
    sc.lights[1, :3] = S.f32(L)
    sc.lights[1, 4], sc.lights[1, 5] = 0.0, R
    p.shadow_samples = 25
    assert_filter_exact(sc, cam, p)


@pytest.mark.parametrize("n", [4096, 4100])
def test_cone_table_size_limit(n):
    """4096 spheres (the largest table with a pre-pass) and 4100 (padded to 4104:
    none), with a square light."""
    rng = np.random.default_rng(n)
    sph = [sphere((rng.uniform(-30, 30), rng.uniform(0.3, 3), rng.uniform(-30, 30)), rng.uniform(0.2, 0.6),
                  albedo=tuple(rng.random(3)), refl=rng.uniform(0, 0.4)) for _ in range(n)]
    sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=0.2), lights=[light((2, 20, -4), 0.8, 4.0)],
                    camera=(0, 12, -40, 0, -18, 60), W=128, H=72, D=2, samples=16, seed=5)
    assert_filter_exact(sc, cam, p)


def test_cone_with_huge_coordinates():
    """Spheres 1e20 away (|oc|^2 overflows) with finite radii: the pre-pass stays on
    and must not clear their blocks by overflow."""
    sc, cam, p = cluster_scene(seed=13)
    sph = sc.spheres.copy()
    sph[:5, 0] = S.f32([1e20, -1e20, 3e19, 1e20, -5e19])
    sph[:5, 2] = S.f32([1e20, 1e20, -1e20, -2e20, 5e19])
    sc.spheres = sph
    assert_filter_exact(sc, cam, p)


def test_incoherent_warps_with_an_area_light():
    """160 spheres of reflectivity 0.9..1 packed in front of the camera, a point light
    and a square light, bounce limit 6: the queue passes' warps hold paths from all
    over the image (the cone groups' item mode: each lane's own blocks shared out over
    the warp), against the tiled loop, which has neither the filter nor the cones."""
    sc = S.random_scene(17, 160, 2, 0.6, area_lights=1, area_side=1.5)
    sc.spheres[:, 9] = np.random.default_rng(17).uniform(0.9, 1.0, 160).astype(np.float32)
    p = S._params(sc, width=256, height=160, max_depth=6, shadow_samples=16, out_format=S.OUT_F32, seed=17)
    assert_filter_exact(sc, S.default_camera(0.6), p)


def test_ray_cull_far_camera_and_camera_inside_a_sphere():
    """The closest-hit cull's radius grows with |o| (2^-16 (c_max + |o|)): a camera a
    million units away with a narrow field of view; and a camera inside a large sphere
    (every primary ray finds the far root of that sphere)."""
    sc, cam, p = cluster_scene(seed=19)
    far = S.f32([0.0, 3e5, -1.3e6, 0.0, -float(np.degrees(np.arctan2(3.0, 13.0))), 0.8])
    assert_filter_exact(sc, far, p)
    sph = np.vstack([sc.spheres.astype(np.float64), sphere((0.0, 6.0, -14.0), 3.0, albedo=(0.6, 0.6, 0.6), refl=0.3)])
    sc2 = S.Scene(spheres=S.f32(sph), plane=sc.plane.copy(), lights=sc.lights.copy(), scale=sc.scale)
    assert_filter_exact(sc2, cam, p)
