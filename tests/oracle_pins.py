"""Pins of the FP64 oracle against things other than itself.

Each ``pin_*`` takes the oracle module and raises AssertionError on a mismatch.
The pins come from the paper (worked example, printed constant), closed forms of
special cases derived by hand, invariants (mirror symmetry, occlusion, depth and
reflectivity reductions), brute force on tiny inputs (ray marching, recursion vs
loop on thousands of 8x8 scenes) and published known-answer vectors (Philox).
They are run one by one in test_oracle_pins.py and, against deliberately broken
builds of the oracle, in test_oracle_mutants.py.
"""
from __future__ import annotations

import math
import os

import numpy as np

from paper_2305_07450_b300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def sphere(c, r, albedo=(0.5, 0.5, 0.5), ks=0.5, ex=32.0, refl=0.0):
    return [c[0], c[1], c[2], r, *albedo, ks, ex, refl]


def plane_rec(n=(0, 1, 0), d=0.0, albedo=(0.75, 0.75, 0.75), ks=0.5, ex=32.0, refl=0.0):
    return [n[0], n[1], n[2], d, *albedo, ks, ex, refl]


def light(p, I=1.0, area=0.0, srad=0.0):
    return [p[0], p[1], p[2], I, area, srad, 0.0, 0.0]


def mk(spheres=(), plane=None, lights=(), camera=(0, 0, 0, 0, 0, 90), W=4, H=4, D=0,
       samples=1, model=S.PHONG, ka=0.1, eps=1e-4, seed=0, scale=1.0):
    sc = S.Scene(spheres=S.f32(np.array(spheres, np.float64).reshape(-1, 10)),
                 plane=None if plane is None else S.f32(plane),
                 lights=S.f32(np.array(lights, np.float64).reshape(-1, 8)), scale=scale)
    p = S.Params(width=W, height=H, max_depth=D, shadow_samples=samples, shading_model=model,
                 ambient=ka, eps=eps, seed=seed)
    return sc, S.f32(camera), p


def pix(orc, sc, cam, p, x, y, **kw):
    return orc.trace(sc, cam, p, np.array([[x, y]], np.int32), threads=1, **kw)["rgb"][0]


f32 = lambda v: float(np.float32(v))  # noqa: E731  (inputs are FP32 records)


# ----------------------------------------------------------------- camera, NDC
def pin_ndc_worked_example(orc):
    """Section 3.2 / 3.3.1: pixel (640, 360) of 1280x720 maps to NDC (0, 0)."""
    for W, H, x, y, u, v in _rows("ndc_worked_example.txt"):
        got = orc.ndc(int(W), int(H), float(x), float(y))
        assert got == (float(u), float(v)), got


def pin_ndc_shorter_side_spans_unit_square(orc):
    """Section 3.2: the viewport is the square [-1,1]^2 on the shorter side."""
    W, H = 1280, 720
    assert orc.ndc(W, H, 0, 0)[1] == 1.0 and orc.ndc(W, H, 0, H)[1] == -1.0
    assert orc.ndc(W, H, W / 2 - H / 2, 0)[0] == -1.0
    assert orc.ndc(W, H, W / 2 + H / 2, 0)[0] == 1.0
    # portrait branch = landscape branch with the axes exchanged
    for (x, y) in [(0, 0), (100, 37), (719, 1279), (360, 640)]:
        u, v = orc.ndc(720, 1280, x, y)
        u2, v2 = orc.ndc(1280, 720, y, x)
        assert abs(u + v2) < 1e-15 and abs(v + u2) < 1e-15, (x, y, u, v, u2, v2)


def pin_camera_distance(orc):
    """Section 3.2.1: b = 1 / tan(alpha / 2); 90 deg -> 1, 60 deg -> sqrt(3)."""
    assert abs(orc.camera_distance(90.0) - 1.0) < 1e-15
    assert abs(orc.camera_distance(60.0) - math.sqrt(3.0)) < 1e-14
    assert abs(orc.camera_distance(120.0) - 1.0 / math.sqrt(3.0)) < 1e-14


def pin_primary_ray(orc):
    """Section 3.3.1: centre ray is +z before rotation; the rotations turn it to the
    spherical direction (cos p sin y, sin p, cos p cos y); the ray through the
    right edge of the unit viewport at 90 deg FOV is 45 deg off axis."""
    sc, _, p = mk(W=4, H=4)
    o, d = orc.primary_ray(sc, S.f32([1, 2, 3, 0, 0, 90]), p, 2, 2)
    assert np.allclose(o, [1, 2, 3]) and np.allclose(d, [0, 0, 1], atol=1e-15)
    o, d = orc.primary_ray(sc, S.f32([0, 0, 0, 0, 0, 90]), p, 4, 2)
    assert np.allclose(d, [math.sqrt(0.5), 0, math.sqrt(0.5)], atol=1e-15)
    o, d = orc.primary_ray(sc, S.f32([0, 0, 0, 0, 0, 90]), p, 2, 0)   # top row looks up
    assert np.allclose(d, [0, math.sqrt(0.5), math.sqrt(0.5)], atol=1e-15)
    for yaw, pitch in [(30.0, 20.0), (-75.0, -12.0), (90.0, 0.0), (0.0, 90.0), (200.0, 45.0)]:
        y, q = math.radians(f32(yaw)), math.radians(f32(pitch))
        _, d = orc.primary_ray(sc, S.f32([0, 0, 0, yaw, pitch, 60]), p, 2, 2)
        want = [math.cos(q) * math.sin(y), math.sin(q), math.cos(q) * math.cos(y)]
        assert np.allclose(d, want, atol=1e-14), (yaw, pitch, d, want)


# ------------------------------------------------------------- intersections
def pin_ray_sphere_closed_forms(orc):
    """Section 3.4: roots of the ray-sphere quadratic in closed form."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        c = rng.uniform(-10, 10, 3)
        r = rng.uniform(0.1, 3.0)
        o = c + rng.normal(size=3) * 0 + (lambda v: v / np.linalg.norm(v))(rng.normal(size=3)) * rng.uniform(r + 0.5, 30)
        d = (c - o) / np.linalg.norm(c - o)
        t = orc.sphere_root(o, d, c, r)
        assert abs(t - (np.linalg.norm(c - o) - r)) < 1e-9, "through the centre: |oc| - r"
        # perpendicular offset h < r: t = D - sqrt(r^2 - h^2)
        e = np.cross(d, rng.normal(size=3))
        e /= np.linalg.norm(e)
        h = rng.uniform(0, 0.99) * r
        o2 = o + h * e
        D = float(np.dot(c - o2, d))
        t2 = orc.sphere_root(o2, d, c, r)
        assert abs(t2 - (D - math.sqrt(r * r - h * h))) < 1e-9
        # offset beyond the radius: miss; pointing away: miss
        assert orc.sphere_root(o + 1.01 * r * e, d, c, r) is None
        assert orc.sphere_root(o, -d, c, r) is None
        # from inside (the centre): the far root, t = r
        assert abs(orc.sphere_root(c, d, c, r) - r) < 1e-12
    # tangent ray: disc = 0 counts as a hit at the tangent point
    assert orc.sphere_root([1, 0, -5], [0, 0, 1], [0, 0, 0], 1.0) == 5.0


def _march(spheres, plane, o, d, tmax, n=60001):
    """Independent brute force: first sample along the ray inside a sphere or past
    the plane, refined by bisection."""
    ts = np.linspace(0, tmax, n)[1:]
    P = o[None, :] + ts[:, None] * d[None, :]
    inside = np.zeros((len(ts), len(spheres) + (plane is not None)), bool)
    for i, s in enumerate(spheres):
        inside[:, i] = np.sum((P - s[:3]) ** 2, 1) < s[3] ** 2
    if plane is not None:
        side0 = np.dot(o, plane[:3]) + plane[3]
        inside[:, -1] = np.sign(P @ plane[:3] + plane[3]) != np.sign(side0)
    anyin = inside.any(1)
    if not anyin.any():
        return -1, None
    k = int(np.argmax(anyin))
    ids = np.nonzero(inside[k])[0]
    lo, hi = (ts[k - 1] if k else 0.0), ts[k]

    def f(t, i):
        q = o + t * d
        if i < len(spheres):
            return np.sum((q - spheres[i][:3]) ** 2) < spheres[i][3] ** 2
        return np.sign(np.dot(q, plane[:3]) + plane[3]) != np.sign(np.dot(o, plane[:3]) + plane[3])
    best = None
    for i in ids:
        a, b = lo, hi
        for _ in range(60):
            m = 0.5 * (a + b)
            if f(m, i):
                b = m
            else:
                a = m
        if best is None or b < best[1]:
            best = (int(i), b)
    return best


def pin_closest_hit_brute_force(orc):
    """Section 3.4.1 against ray marching on small random scenes."""
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(40):
        n = int(rng.integers(1, 6))
        sph = [sphere(rng.uniform([-3, 0.2, -3], [3, 2, 3]), rng.uniform(0.3, 1.0)) for _ in range(n)]
        pl = plane_rec()
        sc, cam, p = mk(spheres=sph, plane=pl)
        arr = np.array(sph, np.float32).astype(np.float64)
        for _ in range(10):
            o = rng.uniform([-4, 0.5, -8], [4, 4, -5])
            tgt = rng.uniform([-3, 0, -3], [3, 2, 3])
            d = (tgt - o) / np.linalg.norm(tgt - o)
            i, t = orc.closest(sc, cam, p, o, d)
            j, tm = _march(arr, np.array(pl, np.float64), o, d, 30.0)
            if j == -1:
                assert i == -1 or t > 30.0 or _graze(arr, o, d, i), (i, t)
                continue
            if i != j:
                assert _graze(arr, o, d, i) or _graze(arr, o, d, j), (i, j, t, tm)
                continue
            assert abs(t - tm) < 2e-3, (t, tm)
            checked += 1
    assert checked > 200


def _graze(arr, o, d, i):
    if i < 0 or i >= len(arr):
        return False
    c, r = arr[i][:3], arr[i][3]
    oc = c - o
    tca = np.dot(oc, d)
    ld = np.linalg.norm(oc - tca * d)
    return abs(ld - r) < 1e-2


def pin_occlusion_brute_force(orc):
    """Section 3.6 cast-shadow test against dense sampling of the segment."""
    rng = np.random.default_rng(12)
    agree = 0
    for trial in range(30):
        n = int(rng.integers(1, 6))
        sph = [sphere(rng.uniform([-3, 0.2, -3], [3, 2, 3]), rng.uniform(0.3, 1.0)) for _ in range(n)]
        pl = plane_rec()
        sc, cam, p = mk(spheres=sph, plane=pl)
        arr = np.array(sph, np.float32).astype(np.float64)
        for _ in range(10):
            o = rng.uniform([-3, 0.05, -3], [3, 3, 3])
            if any(np.linalg.norm(o - s[:3]) < s[3] for s in arr):
                continue
            # half the segments end among the spheres, so that spheres lie beyond the end
            L = rng.uniform([-5, -1, -5], [5, 8, 5]) if rng.random() < 0.5 else \
                rng.uniform([-3, 0.1, -3], [3, 3, 3])
            if any(np.linalg.norm(L - s[:3]) < s[3] for s in arr):
                continue
            dist = float(np.linalg.norm(L - o))
            d = (L - o) / dist
            ts = np.linspace(0, dist, 20001)[1:-1]
            P = o + ts[:, None] * d
            blk = any((np.sum((P - s[:3]) ** 2, 1) < s[3] ** 2).any() for s in arr)
            blk = blk or (np.sign(P[:, 1]) != np.sign(o[1])).any()
            got = orc.occluded(sc, cam, p, o, d, dist)
            if got != blk:
                assert any(abs(np.linalg.norm(s[:3] - o - np.dot(s[:3] - o, d) * d) - s[3]) < 1e-2
                           for s in arr), (got, blk)
            else:
                agree += 1
    assert agree > 150


def pin_single_sphere_lit_side(orc):
    """A lone convex sphere never shadows itself: exactly the pixels whose surface
    faces away from the light (n.l <= 0, by test-side geometry) show ambient only,
    and exactly the others cast a shadow ray."""
    c, r = np.array([0.3, -0.2, 0.5]), 1.3
    alb = (0.7, 0.2, 0.4)
    Lp = (4.0, 3.0, -2.0)
    W = H = 48
    sc, cam, p = mk(spheres=[sphere(c, r, albedo=alb)], lights=[light(Lp, 0.9)],
                    camera=(0, 0, -6, 0, 0, 50), W=W, H=H, ka=0.15, eps=1e-4)
    res = orc.trace(sc, cam, p, counters=True)
    img = res["rgb"].reshape(H, W, 3)
    c32 = np.array([f32(v) for v in c])
    amb = f32(0.15) * np.array([f32(a) for a in alb])
    o = np.array([0.0, 0.0, -6.0])
    lit = 0
    for y in range(H):
        for x in range(W):
            _, d = orc.primary_ray(sc, cam, p, x, y)
            i, t = orc.closest(sc, cam, p, o, d)
            if i != 0:
                continue
            q = o + t * d
            n = (q - c32) / f32(r)
            l = np.array(Lp) - q
            ndl = float(np.dot(n, l / np.linalg.norm(l)))
            if ndl > 1e-9:
                lit += 1
                assert np.all(img[y, x] > amb + 1e-9), (x, y, ndl)
            elif ndl < -1e-9:
                assert np.allclose(img[y, x], amb, atol=1e-15), (x, y, ndl)
    assert lit > 50
    assert res["counters"]["shadow_rays"] == lit


def pin_ties_lowest_index(orc):
    """Reading of Section 3.4.1: two coincident spheres -> the lower index is seen."""
    sph = [sphere((0, 0, 0), 1.0, albedo=(1, 0, 0)), sphere((0, 0, 0), 1.0, albedo=(0, 1, 0))]
    sc, cam, p = mk(spheres=sph, camera=(0, 0, -5, 0, 0, 90))
    rgb = pix(orc, sc, cam, p, 2, 2)
    assert rgb[0] > 0 and rgb[1] == 0


# ------------------------------------------------------------------- shading
def _centre_sphere_scene(light_pos, model=S.PHONG, ka=0.1, I=0.8, ks=0.5, alb=(0.2, 0.4, 0.6)):
    sph = [sphere((0, 0, 0), 1.0, albedo=alb, ks=ks, ex=32.0)]
    return mk(spheres=sph, lights=[light(light_pos, I=I)], camera=(0, 0, -5, 0, 0, 90),
              model=model, ka=ka)


def pin_phong_closed_forms(orc):
    """Section 3.5.1 at the sphere's front point (n = v = (0,0,-1)):
    light at the camera: n.l = v.r = 1 -> c (k_a + I) + I k_s;
    light 60 deg off the normal: n.l = 1/2, v.r = 1/2 -> c (k_a + I/2) + I k_s 2^-32;
    light behind the surface: ambient only, k_a c."""
    alb = np.array([f32(0.2), f32(0.4), f32(0.6)])
    ka, I, ks = f32(0.1), f32(0.8), f32(0.5)
    sc, cam, p = _centre_sphere_scene((0, 0, -5))
    assert np.allclose(pix(orc, sc, cam, p, 2, 2), alb * (ka + I) + I * ks, atol=1e-12)
    q = np.array([0.0, 0.0, -1.0])
    Lp = q + 10.0 * np.array([math.sin(math.pi / 3), 0.0, -math.cos(math.pi / 3)])
    Lp32 = np.array([f32(v) for v in Lp])
    l = (Lp32 - q) / np.linalg.norm(Lp32 - q)
    sc, cam, p = _centre_sphere_scene(Lp32)
    ndl = -l[2]
    want = alb * (ka + I * ndl) + I * ks * (0.5 ** 32)
    assert abs(ndl - 0.5) < 1e-6
    assert np.allclose(pix(orc, sc, cam, p, 2, 2), want, atol=1e-7)
    sc, cam, p = _centre_sphere_scene((0, 0, 5))
    assert np.allclose(pix(orc, sc, cam, p, 2, 2), alb * ka, atol=1e-15)


def pin_blinn_closed_form(orc):
    """Section 3.5.2: light 60 deg off the normal, view along the normal -> the
    halfway vector is 30 deg off the normal: spec = cos(30 deg)^32."""
    alb = np.array([f32(0.2), f32(0.4), f32(0.6)])
    ka, I, ks = f32(0.1), f32(0.8), f32(0.5)
    q = np.array([0.0, 0.0, -1.0])
    Lp = np.array([f32(v) for v in q + 10.0 * np.array([math.sin(math.pi / 3), 0.0, -0.5])])
    sc, cam, p = _centre_sphere_scene(Lp, model=S.BLINN_PHONG)
    l = (Lp - q) / np.linalg.norm(Lp - q)
    h = (l + np.array([0, 0, -1.0]))
    h /= np.linalg.norm(h)
    assert abs(-h[2] - math.cos(math.pi / 6)) < 1e-6
    want = alb * (ka + I * (-l[2])) + I * ks * math.cos(math.pi / 6) ** 32
    assert np.allclose(pix(orc, sc, cam, p, 2, 2), want, atol=1e-6)


def pin_plane_horizon(orc):
    """Sections 3.2-3.4 together: a camera at height 2 pitched down 12 deg sees the
    plane exactly on rows with v < b tan(12 deg); with no light the plane shows
    ambient * albedo and the sky is black."""
    W = H = 64
    sc, cam, p = mk(plane=plane_rec(albedo=(0.5, 0.25, 1.0)), camera=(0, 2, 0, 0, -12, 60),
                    W=W, H=H, ka=0.3)
    img = orc.render(sc, cam, p)
    b = 1.0 / math.tan(math.radians(f32(60.0)) / 2)
    vh = b * math.tan(math.radians(f32(12.0)))
    ka = f32(0.3)
    for y in range(H):
        v = -(y / H * 2 - 1)
        row = img[y]
        if v < vh - 1e-9:
            assert np.allclose(row, [ka * 0.5, ka * 0.25, ka * 1.0], atol=1e-15), y
        elif v > vh + 1e-9:
            assert np.all(row == 0), y


def pin_occlusion_invariant(orc):
    """Section 3.6: a blocker on the segment to the only light leaves ambient * c."""
    alb = (0.5, 0.6, 0.7)
    Lp = (0.0, 6.0, 0.0)
    base = dict(plane=plane_rec(albedo=alb), lights=[light(Lp)], camera=(0, 3, -6, 0, -30, 60),
                W=16, H=16, ka=0.2)
    sc, cam, p = mk(**base)
    open_img = orc.render(sc, cam, p)
    sc2, cam2, p2 = mk(spheres=[sphere((0, 4.5, 0), 1.0)], **base)
    res = orc.trace(sc2, cam2, p2)
    img = res["rgb"].reshape(16, 16, 3)
    want = np.array([f32(0.2) * f32(a) for a in alb])
    # every pixel whose point sees the plane under the blocker's umbra
    shadowed = 0
    for y in range(16):
        for x in range(16):
            _, d = orc.primary_ray(sc2, cam2, p2, x, y)
            o = np.array(cam2[:3], np.float64)
            i, t = orc.closest(sc2, cam2, p2, o, d)
            if i != 1:
                continue
            q = o + t * d
            if np.hypot(q[0], q[2]) < 0.5:            # well inside the umbra cone
                assert np.allclose(img[y, x], want, atol=1e-15)
                assert np.all(open_img[y, x] > want + 1e-3)
                shadowed += 1
    assert shadowed > 0


def pin_mirror_symmetry(orc):
    """A scene mirrored in x, seen by a camera at x = 0 with yaw 0, renders
    mirror-symmetric: img[y][x] = img[y][W - x] (hard shadows, reflections on)."""
    rng = np.random.default_rng(5)
    half = [sphere((rng.uniform(0.5, 3), rng.uniform(0.3, 2), rng.uniform(-2, 3)), rng.uniform(0.3, 0.8),
                   albedo=tuple(rng.uniform(0, 1, 3)), refl=rng.uniform(0, 0.5)) for _ in range(4)]
    sph = half + [[-s[0]] + s[1:] for s in half]
    W = H = 32
    sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=0.25),
                    lights=[light((0, 6, -1), 0.9), light((-3, 5, 2), 0.6), light((3, 5, 2), 0.6)],
                    camera=(0, 2.5, -7, 0, -15, 60), W=W, H=H, D=3, eps=1e-4)
    img = orc.render(sc, cam, p)
    diff = np.abs(img[:, 1:] - img[:, :0:-1]).max()
    assert diff < 1e-12, diff
    assert img.max() > 0.1


def pin_depth_reductions(orc):
    """Section 3.7.1: at D = 0 the reflectivity is never read; with every
    reflectivity 0, D = 1 renders the same image as D = 0."""
    w = S.whitted_256()
    sc = w.scene
    W = H = 24
    p0 = S.Params(width=W, height=H, max_depth=0, ambient=0.1, eps=w.params.eps)
    img0 = orc.render(sc, w.camera, p0)
    sc_r = S.Scene(spheres=sc.spheres.copy(), plane=sc.plane.copy(), lights=sc.lights, scale=sc.scale)
    sc_r.spheres[:, 9] = 0.37
    assert np.array_equal(orc.render(sc_r, w.camera, p0), img0)
    sc_z = S.Scene(spheres=sc.spheres.copy(), plane=sc.plane.copy(), lights=sc.lights, scale=sc.scale)
    sc_z.spheres[:, 9] = 0.0
    sc_z.plane[9] = 0.0
    p1 = S.Params(width=W, height=H, max_depth=1, ambient=0.1, eps=w.params.eps)
    assert np.allclose(orc.render(sc_z, w.camera, p1), orc.render(sc_z, w.camera, p0),
                       atol=0, rtol=1e-15)


def pin_reflection_mixing_closed_form(orc):
    """Section 3.7.1 with no lights (shade(c) = k_a c): a camera looking straight
    down at the plane, a sphere overhead.  The centre pixel is
      D=1: k_a((1-rp) cp + rp k_a cs)
      D=2: k_a((1-rp) cp + rp k_a((1-rs) cs + rs k_a cp))
    -- the reflected colour is itself shaded, and the last bounce is not scaled."""
    cp, cs = np.array([0.9, 0.5, 0.1]), np.array([0.2, 0.7, 0.4])
    rp, rs = f32(0.3), f32(0.45)
    cp = np.array([f32(v) for v in cp])
    cs = np.array([f32(v) for v in cs])
    ka = f32(0.5)
    for D in (1, 2, 3):
        sc, cam, p = mk(spheres=[sphere((0, 10, 0), 2.0, albedo=tuple(cs), refl=rs)],
                        plane=plane_rec(albedo=tuple(cp), refl=rp),
                        camera=(0, 5, 0, 0, -90, 60), W=4, H=4, D=D, ka=ka)
        got = pix(orc, sc, cam, p, 2, 2)
        if D == 1:
            want = ka * ((1 - rp) * cp + rp * ka * cs)
        elif D == 2:
            want = ka * ((1 - rp) * cp + rp * ka * ((1 - rs) * cs + rs * ka * cp))
        else:
            inner = ka * ((1 - rp) * cp + rp * ka * cs)          # plane seen at depth 1
            want = ka * ((1 - rp) * cp + rp * ka * ((1 - rs) * cs + rs * inner))
        assert np.allclose(got, want, atol=1e-12), (D, got, want)


def pin_coupled_reflectivity(orc):
    """Section 3.7: with the paper's coupling the reflection ratio is the Phong
    exponent / MAX_REFLECTIVITY (capped at a mirror); the reflectivity field is
    then unused.  Same closed form as the depth-1 mixing pin, with exponents 16 and
    48 over MAX_REFLECTIVITY 64 (ratios 1/4 and 3/4)."""
    cp = np.array([f32(v) for v in (0.9, 0.5, 0.1)])
    cs = np.array([f32(v) for v in (0.2, 0.7, 0.4)])
    ka = f32(0.5)
    sc, cam, p = mk(spheres=[sphere((0, 10, 0), 2.0, albedo=tuple(cs), ex=48.0, refl=0.01)],
                    plane=plane_rec(albedo=tuple(cp), ex=16.0, refl=0.99),
                    camera=(0, 5, 0, 0, -90, 60), W=4, H=4, D=2, ka=ka)
    p.refl_coupled, p.max_reflectivity = 1, 64.0
    rp, rs = 0.25, 0.75
    want = ka * ((1 - rp) * cp + rp * ka * ((1 - rs) * cs + rs * ka * cp))
    got = pix(orc, sc, cam, p, 2, 2)
    assert np.allclose(got, want, atol=1e-12), (got, want)
    p.max_reflectivity = 8.0       # both ratios capped at 1: pure mirrors below the last bounce
    want = ka * (ka * (ka * cp))
    assert np.allclose(pix(orc, sc, cam, p, 2, 2), want, atol=1e-12)


def pin_recursion_equals_loop(orc, n_scenes=2000):
    """Section 3.7.1 vs 3.7.2: the literal recursion and the forward loop agree on
    thousands of random 8x8 scenes (hard, area-light and Blinn variants)."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for i in range(n_scenes):
        n = int(rng.integers(0, 6))
        sph = [sphere(rng.uniform([-3, 0.2, -3], [3, 2.5, 3]), rng.uniform(0.3, 1.2),
                      albedo=tuple(rng.uniform(0, 1, 3)), ks=rng.uniform(0, 1),
                      ex=float(rng.choice([1.0, 8.0, 32.0])), refl=rng.uniform(0, 0.9))
               for _ in range(n)]
        nl = int(rng.integers(0, 4))
        lig = [light(rng.uniform([-5, 4, -5], [5, 8, 5]), rng.uniform(0.2, 1.0),
                     area=(rng.uniform(0.5, 2) if rng.random() < 0.3 else 0.0)) for _ in range(nl)]
        sc, cam, p = mk(spheres=sph, plane=plane_rec(refl=rng.uniform(0, 0.6)) if rng.random() < 0.8 else None,
                        lights=lig, camera=(rng.uniform(-1, 1), rng.uniform(1.5, 4), -8,
                                            rng.uniform(-10, 10), rng.uniform(-25, 0), 60),
                        W=8, H=8, D=int(rng.integers(0, 5)), samples=int(rng.choice([1, 4, 9])),
                        model=int(rng.integers(0, 2)), seed=int(rng.integers(0, 2**63)))
        a = orc.trace(sc, cam, p, threads=1)["rgb"]
        b = orc.trace(sc, cam, p, mode="recursive", threads=1)["rgb"]
        worst = max(worst, float(np.abs(a - b).max()))
    assert worst < 1e-12, worst


def _plane_pixels(orc, sc, cam, p, plane_id):
    """(x, y, hit point) of every pixel whose primary ray hits the plane first."""
    o = np.array(cam[:3], np.float64)
    out = []
    for y in range(p.height):
        for x in range(p.width):
            _, d = orc.primary_ray(sc, cam, p, x, y)
            i, t = orc.closest(sc, cam, p, o, d)
            if i == plane_id:
                out.append((x, y, o + t * d))
    return out


def pin_area_light(orc):
    """Area light (square, stratified): unblocked it equals a point light at its
    centre; inside a blocker's umbra it contributes nothing; in the penumbra the
    visible fraction is a multiple of 1/n."""
    alb = (0.6, 0.5, 0.4)
    cam = (0, 3, -6, 0, -30, 60)
    base = dict(plane=plane_rec(albedo=alb), camera=cam, W=12, H=12, ka=0.1, samples=16, seed=99)
    sc_a, c, p = mk(lights=[light((0, 6, 0), 0.9, area=1.5)], **base)
    sc_p, _, _ = mk(lights=[light((0, 6, 0), 0.9)], **base)
    assert np.array_equal(orc.render(sc_a, c, p), orc.render(sc_p, c, p))
    ambient = f32(0.1) * np.array([f32(a) for a in alb])
    blocker = sphere((0, 4.0, 0), 1.5)
    sc_b, _, _ = mk(spheres=[blocker], lights=[light((0, 6.2, 0), 0.9, area=1.0)], **base)
    img_b = orc.render(sc_b, c, p)
    umbra = 0
    for x, y, q in _plane_pixels(orc, sc_b, c, p, 1):
        if np.hypot(q[0], q[2]) < 1.0:
            assert np.allclose(img_b[y, x], ambient, atol=1e-15)
            umbra += 1
    assert umbra > 0
    part = sphere((0.3, 5.2, 0.2), 0.45)
    low = sphere((0.3, -50, 0.2), 0.45)                 # same sphere moved out of the way
    sc_pt, _, _ = mk(spheres=[part], lights=[light((0, 6, 0), 0.9, area=1.2)], **base)
    sc_fu, _, _ = mk(spheres=[low], lights=[light((0, 6, 0), 0.9, area=1.2)], **base)
    img, full = orc.render(sc_pt, c, p), orc.render(sc_fu, c, p)
    fracs = []
    for x, y, _ in _plane_pixels(orc, sc_pt, c, p, 1):
        fr = (img[y, x, 0] - ambient[0]) / (full[y, x, 0] - ambient[0])
        k = fr * 16
        assert abs(k - round(k)) < 1e-6, k
        fracs.append(round(k))
    assert len(set(fracs)) > 2, fracs


def pin_philox_kat(orc):
    """Philox4x32-10 against the published known-answer vectors."""
    for row in _rows("philox4x32_10_kat.txt"):
        v = [int(h, 16) for h in row]
        got = orc.philox4x32_10(v[0:4], v[4:6])
        assert got.tolist() == v[6:10], [hex(g) for g in got]


def pin_counters(orc):
    """Brute force does exactly (N + 1) tests per traced ray; every lit point light
    casts one shadow ray; an area light casts n samples from n / 2 Philox calls."""
    w = S.whitted_256()
    p = S.Params(width=32, height=32, max_depth=2, ambient=0.1, eps=w.params.eps)
    r = orc.trace(w.scene, w.camera, p, counters=True)["counters"]
    rays = r["primary_rays"] + r["reflection_rays"]
    assert r["primary_rays"] == 32 * 32
    assert r["closest_sphere_tests"] == rays * w.scene.n_spheres
    assert r["closest_plane_tests"] == rays
    assert r["shadow_rays"] == r["lit_lights"]
    assert r["shadow_sphere_tests"] <= r["shadow_rays"] * w.scene.n_spheres
    w4 = S.area_4k()
    p4 = S.Params(width=16, height=9, max_depth=1, shadow_samples=16, ambient=0.1, eps=w4.params.eps)
    r = orc.trace(w4.scene, w4.camera, p4, counters=True)["counters"]
    assert r["light_samples"] == 16 * r["philox_calls"] // 8
    assert r["shadow_rays"] == r["lit_lights"] + r["light_samples"] - r["philox_calls"] // 8


def pin_margin_grazing(orc):
    """Margin of a ray passing at distance h from a sphere of radius r is |h - r|."""
    sc, cam, p = mk(spheres=[sphere((0, 0, 0), 1.0)], camera=(0, 0, -20, 0, 0, 2.0), W=64, H=64, scale=100.0)
    # ray of pixel (x, 32): lateral offset at the sphere ~ 20 * u * tan(1 deg)
    for x in (0, 10, 40, 63):
        _, d = orc.primary_ray(sc, cam, p, x, 32)
        o = np.array([0, 0, -20.0])
        tca = np.dot(-o, d)
        h = np.linalg.norm(-o - tca * d)
        m = orc.trace(sc, cam, p, np.array([[x, 32]], np.int32), margin=True, threads=1)["margin"][0]
        assert abs(m - abs(h - 1.0)) < 1e-9, (x, m, h)


H_GRAZE = 2.0 ** -7        # a small distance exact in FP32


def _close(a, b, tol=1e-12):
    return abs(a - b) <= tol * max(1.0, abs(b))


def pin_margin_closest_terms(orc):
    """Margins of one closest-hit ray (the distances below which FP32 could decide
    the hit differently: Section 3.4's closest-hit decision), in closed form along
    the +z axis from the origin:
      gap to the second primitive: spheres at depth 9 and 9 + h -> h, in either
      index order; the plane at depth 9 + h behind a sphere hit at 9 -> h;
      plane horizon: a ray at slope s to the plane y = 0 -> s * scene scale, hit or
      miss (the scene scale being the sphere box's half-extent, 5 length units
      per unit of scale); a root near the origin: the plane h below -> h, a sphere surface h
      behind -> h, neither counted when the ray leaves that primitive;
      a silhouette grazed at distance h in front of the hit -> h, but not behind
      the hit and not behind the origin."""
    h = H_GRAZE
    o, z = np.zeros(3), np.array([0.0, 0.0, 1.0])
    A, B = sphere((0, 0, 10), 1.0), sphere((0, 0, 10 + h), 1.0)
    for sph in ([A, B], [B, A]):
        sc, cam, p = mk(spheres=sph)
        i, t, m = orc.closest(sc, cam, p, o, z, margin=True)
        assert sph[i] is A and t == 9.0 and _close(m, h), (i, t, m)
    sc, cam, p = mk(spheres=[A], plane=plane_rec(n=(0, 0, 1), d=-(9 + h)))
    i, t, m = orc.closest(sc, cam, p, o, z, margin=True)
    assert i == 0 and _close(m, h), (i, m)
    s = 0.01
    for scale in (1.0, 2.0):
        sc, cam, p = mk(plane=plane_rec(), scale=scale)
        for sign, want_id in ((-1.0, 0), (1.0, -1)):
            d = np.array([math.sqrt(1 - s * s), sign * s, 0.0])
            i, t, m = orc.closest(sc, cam, p, np.array([0.0, 1.0, 0.0]), d, margin=True)
            assert i == want_id and _close(m, s * sc.scene_scale), (scale, sign, i, m)
    sc, cam, p = mk(plane=plane_rec(), scale=1.0)
    assert sc.scene_scale > 1.0
    down = np.array([0.0, -1.0, 0.0])
    i, t, m = orc.closest(sc, cam, p, np.array([0.0, h, 0.0]), down, margin=True)
    assert i == 0 and _close(t, h) and _close(m, h), (i, t, m)
    i, t, m = orc.closest(sc, cam, p, np.array([0.0, h, 0.0]), down, origin=0, margin=True)
    assert i == 0 and _close(m, sc.scene_scale), m
    sc, cam, p = mk(spheres=[sphere((0, 0, -1 - h), 1.0)])
    i, t, m = orc.closest(sc, cam, p, o, z, margin=True)
    assert i == -1 and _close(m, h), (i, m)
    i, t, m = orc.closest(sc, cam, p, o, z, origin=0, margin=True)
    assert i == -1 and math.isinf(m), m
    for cz, want in ((5.0, h), (20.0, 9.0)):
        sc, cam, p = mk(spheres=[A, sphere((1 + h, 0, cz), 1.0)])
        i, t, m = orc.closest(sc, cam, p, o, z, margin=True)
        assert i == 0 and _close(m, want), (cz, i, m)
    sc, cam, p = mk(spheres=[sphere((1 + h, 0, -5), 1.0)])
    i, t, m = orc.closest(sc, cam, p, o, z, margin=True)
    assert i == -1 and math.isinf(m), m


def pin_margin_shadow_terms(orc):
    """Margins of one shadow segment o + t z, 0 < t < dist (Section 3.6's
    cast-shadow decision), in closed form: a sphere spanning depths 9..11 and
    the light h before its near surface, h inside it, or h beyond its far
    surface -> h; a sphere surface h ahead of the origin -> h (not counted when
    the segment leaves that sphere: then the silhouette term, r = 1); a
    silhouette grazed at h between origin and light -> h, but not beyond the
    light or behind the origin; the plane y = 0 crossed h before or after the
    light -> h; the plane h behind the origin -> h, not counted when the
    segment leaves the plane."""
    h = H_GRAZE
    o, z = np.zeros(3), np.array([0.0, 0.0, 1.0])
    sc, cam, p = mk(spheres=[sphere((0, 0, 10), 1.0)])
    for dist, blocked in ((9 - h, False), (9 + h, True), (11 + h, True)):
        b, m = orc.occluded(sc, cam, p, o, z, dist, margin=True)
        assert b == blocked and _close(m, h), (dist, b, m)
    sc, cam, p = mk(spheres=[sphere((0, 0, 1 + h), 1.0)])
    b, m = orc.occluded(sc, cam, p, o, z, 100.0, margin=True)
    assert b and _close(m, h), (b, m)
    b, m = orc.occluded(sc, cam, p, o, z, 100.0, origin=0, margin=True)
    assert b and _close(m, 1.0), (b, m)
    for cz, want in ((5.0, h), (15.0, math.inf), (-5.0, math.inf)):
        sc, cam, p = mk(spheres=[sphere((1 + h, 0, cz), 1.0)])
        b, m = orc.occluded(sc, cam, p, o, z, 10.0, margin=True)
        assert not b and (_close(m, want) if want < math.inf else math.isinf(m)), (cz, b, m)
    sc, cam, p = mk(plane=plane_rec())
    down = np.array([0.0, -1.0, 0.0])
    for dist, blocked in ((1 - h, False), (1 + h, True)):
        b, m = orc.occluded(sc, cam, p, np.array([0.0, 1.0, 0.0]), down, dist, margin=True)
        assert b == blocked and _close(m, h), (dist, b, m)
    up = np.array([0.0, 1.0, 0.0])
    b, m = orc.occluded(sc, cam, p, np.array([0.0, h, 0.0]), up, 5.0, margin=True)
    assert not b and _close(m, h), (b, m)
    b, m = orc.occluded(sc, cam, p, np.array([0.0, h, 0.0]), up, 5.0, origin=0, margin=True)
    assert not b and _close(m, 5.0 + h), (b, m)


def pin_margin_light_gate(orc):
    """The light gate n.l > 0 (Section 3.5 with the shadow rays of Section 3.6)
    decides whether a light contributes at all; its margin is |n.l| x scene scale.
    A camera looking straight down at the plane y = 0 from height 10 sees the
    origin in its centre pixel; a light at (10, +-y_l, 0) grazes it, n.l =
    y_l / |L|, and every other term of that pixel's path is larger."""
    yl = 0.0625
    for scale in (1.0, 2.0):
        for sgn in (1.0, -1.0):
            Lp = (10.0, sgn * yl, 0.0)
            sc, cam, p = mk(plane=plane_rec(), lights=[light(Lp)], camera=(0, 10, 0, 0, -90, 60), W=4, H=4,
                            scale=scale)
            m = orc.trace(sc, cam, p, np.array([[2, 2]], np.int32), margin=True, threads=1)["margin"][0]
            want = yl / math.hypot(10.0, yl) * sc.scene_scale
            assert _close(m, want, 1e-9), (scale, sgn, m, want)


# pixels of the 3840x2160 seeded workload whose paths run six to nine bounces
# between spheres (found by scanning the frame): chains where rounding in the
# hit geometry is amplified most from bounce to bounce
DEEP_4K_PIXELS = [(1849, 695), (2767, 705), (1535, 707), (1558, 707), (2044, 711), (2642, 712), (2643, 712),
                  (1549, 714), (2395, 717), (2412, 717), (2056, 725), (1660, 730)]


def pin_path_geometry_invariants(orc):
    """Along every ray path (Sections 3.4, 3.5, 3.7.1): each hit point lies on its
    primitive (|p - c| = r, or the plane equation), each normal and direction has
    unit length, the normal faces the incoming ray, and the next ray leaves from
    p + eps n along the mirror direction d - 2 (d.n) n.  Checked on deep
    reflection chains of the 4K workload and on a lattice of its pixels."""
    w = S.area_4k()
    sph = np.asarray(w.scene.spheres, np.float64).reshape(-1, 10)
    pl = np.asarray(w.scene.plane, np.float64)
    eps = float(w.params.eps)
    pixels = DEEP_4K_PIXELS + [(x, y) for y in range(0, 2160, 157) for x in range(0, 3840, 263)]
    deep = 0
    for x, y in pixels:
        P = orc.trace_path(w.scene, w.camera, w.params, x, y)
        o0, d0 = orc.primary_ray(w.scene, w.camera, w.params, x, y)
        assert np.array_equal(P[0, 2:5], o0) and np.array_equal(P[0, 5:8], d0)
        for k, row in enumerate(P):
            i = int(row[0])
            o, d, p, n = row[2:5], row[5:8], row[8:11], row[11:14]
            assert abs(np.linalg.norm(d) - 1.0) < 1e-12, (x, y, k, np.linalg.norm(d))
            if i < 0:
                assert k == len(P) - 1
                continue
            assert np.allclose(p, o + row[1] * d, rtol=0, atol=1e-12 * (1 + np.abs(p).max()))
            if i < len(sph):
                assert abs(np.linalg.norm(p - sph[i, :3]) / sph[i, 3] - 1.0) < 1e-9, (x, y, k, i)
            else:
                assert abs(np.dot(pl[:3], p) + pl[3]) < 1e-9 * (1 + np.abs(p).max()), (x, y, k)
            assert abs(np.linalg.norm(n) - 1.0) < 1e-12, (x, y, k, np.linalg.norm(n))
            assert np.dot(n, d) <= 0.0, (x, y, k)
            if k + 1 < len(P):
                nxt = P[k + 1]
                assert np.allclose(nxt[5:8], d - 2 * np.dot(d, n) * n, rtol=0, atol=1e-14)
                assert np.allclose(nxt[2:5], p + eps * n, rtol=0, atol=1e-13 * (1 + np.abs(p).max()))
        deep += len(P) >= 7
    assert deep >= 8


def pin_rgba8(orc):
    """toInt reading: clamp, x 255, round half up, alpha 255, 0xAABBGGRR."""
    rgb = np.array([[0.5, 0.25, 1.5], [-1.0, 0.0, 1.0], [0.2, 0.6, 0.999]])
    got = orc.to_rgba8(rgb)
    assert got[0] == (0xFF << 24) | (255 << 16) | (64 << 8) | 128
    assert got[1] == (0xFF << 24) | (255 << 16) | (0 << 8) | 0
    assert got[2] == (0xFF << 24) | (255 << 16) | (153 << 8) | 51


def pin_area_samples_stratified(orc):
    """Stratified square light: sample s lies in cell (s mod g, s div g) of the
    g x g grid over the light's square (centred on the light, horizontal); the
    in-cell offsets are uniform over pixels; pixels, bounces and lights get
    independent samples."""
    a, g = 1.5, 4
    Lp = np.array([f32(1.0), f32(6.0), f32(-2.0)])
    sc, cam, p = mk(lights=[light((0, 9, 0)), light(Lp, 1.0, area=a)], W=64, H=64, samples=g * g,
                    seed=1234567)
    offs = []
    seen = set()
    for (x, y, k) in [(x, y, k) for x in range(0, 64, 3) for y in range(0, 64, 7) for k in (0, 1)]:
        pts = orc.light_samples(sc, cam, p, 1, x, y, k)
        assert pts.shape == (16, 3)
        assert np.all(pts[:, 1] == Lp[1])
        fx = (pts[:, 0] - (Lp[0] - f32(a) / 2)) / (f32(a) / g)
        fz = (pts[:, 2] - (Lp[2] - f32(a) / 2)) / (f32(a) / g)
        cell_i, cell_j = np.floor(fx + 1e-12), np.floor(fz + 1e-12)
        s_idx = np.arange(16)
        assert np.array_equal(cell_i, s_idx % g) and np.array_equal(cell_j, s_idx // g), (fx, fz)
        offs.append(np.concatenate([fx - cell_i, fz - cell_j]))
        seen.add(tuple(np.round(pts[:, 0], 9)))
    offs = np.concatenate(offs)
    assert abs(offs.mean() - 0.5) < 0.02 and abs(offs.var() - 1 / 12) < 0.01
    assert len(seen) == len(offs) // 32          # no two (pixel, bounce) alike
    assert orc.light_samples(sc, cam, p, 0, 0, 0, 0).shape[0] == 0   # point light: none


def pin_vogel_sunflower(orc):
    """Section 3.6.1: sunflower points on the great circle facing the point, radius
    R sqrt(i/n), successive angles one golden angle apart (the printed constant)."""
    (deg, decimals), = _rows("golden_angle.txt")
    R, n = 0.8, 50
    Lp = np.array([f32(0.5), f32(7.0), f32(1.0)])
    sc, cam, p = mk(lights=[light(Lp, 1.0, srad=R)], W=8, H=8, samples=n)
    q = np.array([2.0, 0.3, -1.0])
    pts = orc.light_samples(sc, cam, p, 0, 3, 3, 0, q)
    assert pts.shape == (n, 3)
    w = (q - Lp) / np.linalg.norm(q - Lp)
    rel = pts - Lp
    assert np.abs(rel @ w).max() < 1e-12                       # in the plane facing q
    radii = np.linalg.norm(rel, axis=1)
    assert np.allclose(radii, f32(R) * np.sqrt(np.arange(n) / n), atol=1e-12)
    ang = np.arctan2(rel @ np.cross(w, rel[1] / radii[1]), rel @ (rel[1] / radii[1]))
    step = np.degrees(np.mod(np.diff(ang[1:]), 2 * np.pi))
    assert np.allclose(step, step[0], atol=1e-9)
    golden = min(float(step[0]), 360.0 - float(step[0]))      # orientation-free
    assert abs(golden - float(deg)) < 10.0 ** -int(decimals), golden

# ----------------------------------------------------------------- sky (NEXT-3)
def _sky_tex(seed, W=16, H=8):
    t = np.random.default_rng(seed).random((H, W, 4)).astype(np.float32)
    t[..., 3] = 1.0
    return t


def _unit(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def pin_sky_invariants(orc):
    """Section 3.8 sky, equirectangular UV mapping (u = longitude, v = latitude from
    the top), bilinear between texel centres.  Checked by properties only: a constant
    panorama is constant; turning the direction by one texel of longitude (2 pi / W
    about y) equals shifting the panorama by one column; flipping the latitude
    equals flipping the rows; a panorama symmetric under column mirror i -> W-1-i
    gives z-mirror symmetric colours (this fixes the half-texel offset); the
    cardinal directions of the convention u = 1/2 + atan2(d_z, d_x) / 2 pi land on
    the columns it names; a panorama that varies only by row gives its top row
    straight up and the mean of the two middle rows on the horizon."""
    rng = np.random.default_rng(5)
    W, H = 16, 8
    const = np.ones((H, W, 4), np.float32) * np.float32(0.3)
    for d in _unit(rng, 20):
        assert np.allclose(orc.sky(const, d), 0.3, atol=1e-7)
    T = _sky_tex(1, W, H)
    shifted = np.ascontiguousarray(np.roll(T, -1, axis=1))
    fl = np.ascontiguousarray(T[::-1])
    mir = np.ascontiguousarray(0.5 * (T + T[:, ::-1]))
    a = 2 * np.pi / W
    rot = np.array([[math.cos(a), 0, -math.sin(a)], [0, 1, 0], [math.sin(a), 0, math.cos(a)]])
    for d in _unit(rng, 40):
        # rot turns atan2(z, x) by +a
        assert np.allclose(orc.sky(T, rot @ d), orc.sky(shifted, d), atol=1e-9), d
        assert np.allclose(orc.sky(T, d * [1, -1, 1]), orc.sky(fl, d), atol=1e-9), d
        assert np.allclose(orc.sky(mir, d), orc.sky(mir, d * [1, 1, -1]), atol=1e-9), d
    # columns by index, rows constant: longitude -> column
    C = np.zeros((H, W, 4), np.float32)
    C[..., 0] = np.arange(W, dtype=np.float32)[None, :]
    for d, col in (((1, 0, 0), W / 2 - 0.5), ((0, 0, 1), 3 * W / 4 - 0.5), ((0, 0, -1), W / 4 - 0.5)):
        assert abs(orc.sky(C, d)[0] - col) < 1e-9, (d, orc.sky(C, d))
    # -x is the seam: halfway between the last and the first column
    assert abs(orc.sky(C, (-1, 1e-12, -1e-15))[0] - 0.5 * (W - 1)) < 1e-6
    R = np.zeros((H, W, 4), np.float32)
    R[..., 1] = np.arange(H, dtype=np.float32)[:, None]
    assert abs(orc.sky(R, (0, 1, 0))[1] - 0.0) < 1e-12 and abs(orc.sky(R, (0, -1, 0))[1] - (H - 1)) < 1e-12
    assert abs(orc.sky(R, (0.3, 0.0, -0.7))[1] - (H / 2 - 0.5)) < 1e-9
    # interpolation weights: the stored row (column) index rises strictly as the
    # direction sweeps down in latitude (east in longitude, away from the seam)
    lat = np.radians(np.linspace(75, -75, 301))
    rows = [orc.sky(R, (math.cos(b) * 0.6, math.sin(b), math.cos(b) * 0.8))[1] for b in lat]
    assert np.all(np.diff(rows) > 0), "row weights"
    lon = np.radians(np.linspace(-160, 160, 301))
    cols = [orc.sky(C, (math.cos(l), 0.2, math.sin(l)))[0] for l in lon]
    assert np.all(np.diff(cols) > 0), "column weights"


def pin_sky_on_misses(orc):
    """A ray that leaves the scene shows the sky (Section 3.8); through the bounce
    recursion (Section 3.7.1) a perfect mirror sphere (reflectivity 1, no lights)
    shows k_a times the sky in the mirror direction, computed here from the
    closed-form hit point of the sphere."""
    T = _sky_tex(2, 32, 16)
    cam = (0, 0, -5, 0, 0, 60)
    sc, c, p = mk(camera=cam, W=8, H=6)
    sc.sky = T
    for x, y in ((0, 0), (3, 2), (7, 5)):
        o, d = orc.primary_ray(sc, c, p, x, y)
        assert np.allclose(pix(orc, sc, c, p, x, y), orc.sky(T, d), atol=1e-12)
    ka = 0.25
    sc, c, p = mk(spheres=[sphere((0, 0, 0), 1.0, albedo=(0.9, 0.1, 0.4), refl=1.0)], camera=cam, W=9, H=9,
                  D=1, ka=ka)
    sc.sky = T
    for x, y in ((4, 4), (3, 5), (5, 3)):
        o, d = orc.primary_ray(sc, c, p, x, y)
        b = float(np.dot(o, d))
        disc = b * b - (float(np.dot(o, o)) - 1.0)
        assert disc > 0
        t = -b - math.sqrt(disc)
        n = o + t * d                                   # unit sphere at the origin
        r = d - 2 * np.dot(d, n) * n
        want = ka * orc.sky(T, r)
        for mode in ("forward", "recursive"):
            got = orc.trace(sc, c, p, np.array([[x, y]], np.int32), mode=mode, threads=1)["rgb"][0]
            assert np.allclose(got, want, atol=1e-9), (mode, got, want)


# ------------------------------------------------------------- physics (NEXT-3)
def pin_verlet_free_fall(orc):
    """Position Verlet is exact for constant acceleration: from x_0 and x_{-1} =
    x_0 - v_0 dt, x_n = x_0 + n v_0 dt - g dt^2 n (n + 1) / 2 (y), with no plane."""
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-5, 5, (6, 3))
    v0 = rng.uniform(-2, 2, (6, 3))
    dt, g, n = 1.0 / 60.0, 9.81, 240
    pos, prev = orc.verlet(x0, x0 - v0 * dt, np.ones(6), None, dt, g, 0.5, n)
    want = x0 + n * v0 * dt
    want[:, 1] -= g * dt * dt * n * (n + 1) / 2
    assert np.allclose(pos, want, rtol=0, atol=1e-9), np.abs(pos - want).max()
    assert np.allclose(pos - prev, v0 * dt + np.array([0, -g * dt * dt * n, 0]), atol=1e-9)


def pin_verlet_ground_contact(orc):
    """Contact with the ground plane: a resting sphere stays exactly at rest; with
    restitution 0 a dropped sphere ends touching the plane and keeps its horizontal
    velocity; with restitution 1 it bounces back to within a step of its drop
    height; a tilted plane leaves the sphere touching it after the contact step."""
    dt, g = 1.0 / 120.0, 9.81
    plane = (0.0, 1.0, 0.0, 0.0)
    r = np.array([0.5])
    x = np.array([[1.0, 0.5, -2.0]])
    pos, prev = orc.verlet(x, x, r, plane, dt, g, 0.7, 1000)
    assert np.array_equal(pos, x) and np.array_equal(prev, x)
    h = 3.0
    x = np.array([[0.0, h, 0.0]])
    vx = 0.4
    pos, prev = orc.verlet(x, x - [[vx * dt, 0, 0]], r, plane, dt, g, 0.0, 300)
    assert abs(pos[0, 1] - 0.5) < 1e-12 and abs(pos[0, 1] - prev[0, 1]) < 1e-12
    assert abs((pos[0, 0] - prev[0, 0]) - vx * dt) < 1e-12
    pos, prev = x.copy(), x.copy()
    top, seen_ground = 0.0, False
    for _ in range(400):                                  # ~ two bounces
        pos, prev = orc.verlet(pos, prev, r, plane, dt, g, 1.0, 1)
        if pos[0, 1] < 0.5 + 1e-9:
            seen_ground = True
        if seen_ground:
            top = max(top, pos[0, 1])
    v_impact = math.sqrt(2 * g * (h - 0.5))
    assert seen_ground and abs(top - h) < 2 * v_impact * dt, (top, h)
    nrm = np.array([0.3, 1.0, -0.2]) / np.linalg.norm([0.3, 1.0, -0.2])
    tilted = (*nrm, 0.4)
    x = np.array([[0.2, 1.0, 0.1]]) - nrm * (np.dot(nrm, [0.2, 1.0, 0.1]) + 0.4 - 0.5 - 1e-3)
    pos, prev = orc.verlet(x, x + nrm * 0.05, r, tilted, dt, g, 0.5, 1)
    assert abs(np.dot(nrm, pos[0]) + 0.4 - 0.5) < 1e-12


PINS = {k: v for k, v in globals().items() if k.startswith("pin_")}
