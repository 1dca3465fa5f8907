"""The animated loop on the GPU (Section 3.8 sky and physics): sky parity with the
FP64 oracle, the sky through the batch and the hierarchy (bit-identical), one-step
parity of the Verlet kernel with the oracle's step, and animated frames equal to
the same positions uploaded from the host."""
import copy

import numpy as np
import pytest
import torch

import oracle
from oracle_pins import light, mk, plane_rec, sphere
from paper_2305_07450_b300 import animate, rt, scenes as S
from parity import compare_f32, compare_rgba8, oracle_reference
from test_render_gpu import check_f32_full, gpu_render, small_cases

pytestmark = pytest.mark.gpu
SKY = S.sky_texture()


def with_sky(w, tex=SKY):
    w = copy.deepcopy(w)
    w.scene.sky = tex
    w.name += "_sky"
    return w


@pytest.mark.parametrize("name", ["empty", "ragged_37x23_d3", "no_plane_deep", "area_light", "blinn"])
def test_small_cases_with_sky(name):
    sc, cam, p = small_cases()[name]
    p.eps = 5e-4
    check_f32_full(with_sky(S.Workload(name, sc, cam, p)), min_plain=0.98)


def test_whitted_256_with_sky():
    check_f32_full(with_sky(S.whitted_256()), min_plain=0.995)


def test_paper_scene_with_sky_200_samples():
    w = with_sky(S.paper_scene(128, 72, 200, 3))
    check_f32_full(w, min_plain=0.99)


def test_720p_with_sky_sampled_rgba8():
    w = with_sky(S.whitted_720p())
    img, _ = gpu_render(w)
    px = S.pixel_lattice(w.params.width, w.params.height, 29, seed=4, n_random=800)
    ref, margin, sens = oracle_reference(w, px)
    ok, st = compare_rgba8(img[px[:, 1], px[:, 0]], ref, margin, sens, w.scene.scene_scale)
    print(st)
    assert st["failing"] == 0 and st["frac_within_1lsb"] >= 0.999, st


def test_sky_through_batch_and_hierarchy_bitwise():
    ws = [with_sky(S.whitted_256()), with_sky(S.paper_scene(160, 90, 16, 2)), S.whitted_256()]
    for w in ws:
        w.params.out_format = S.OUT_F32
    dss = [rt.DeviceScene(w.scene) for w in ws]
    outs, pitches = rt.alloc_batch_outputs([w.params for w in ws])
    rt.render_batch(dss, [w.camera for w in ws], [w.params for w in ws], outs=outs, pitches=pitches)
    for w, d, o in zip(ws, dss, outs):
        single = rt.render(d, w.camera, w.params)
        d.build_bvh()
        acc = rt.render(d, w.camera, w.params, launch={"accel": 1})
        torch.cuda.synchronize()
        assert torch.equal(o, single) and torch.equal(acc, single), w.name
    assert rt.device_errors() == 0


def test_removing_the_sky_gives_black_misses():
    w = with_sky(S.whitted_256())
    ds = rt.DeviceScene(w.scene)
    ds.set_sky(None)
    a = rt.render(ds, w.camera, w.params).cpu().numpy()
    b, _ = gpu_render(S.whitted_256())
    assert np.array_equal(a, b)


def test_verlet_one_step_parity():
    """From the device's own FP32 state, each step equals the oracle's FP64 step of
    that state to FP32 rounding, over 400 steps with falls and bounces."""
    w, prev = S.animated_scene(64, 36)
    sph = torch.from_numpy(w.scene.spheres.copy()).cuda()
    pv = torch.from_numpy(prev.copy()).cuda()
    r = w.scene.spheres[:, 3].astype(np.float64)
    plane = w.scene.plane
    dt, g, e = 1.0 / 60.0, 9.81, 0.7
    worst = 0.0
    for _ in range(400):
        x0 = sph[:, :3].cpu().numpy().astype(np.float64)
        p0 = pv.cpu().numpy().astype(np.float64)
        rt.verlet_step(sph, pv, plane, dt=dt, gravity=g, restitution=e, steps=1)
        want_x, want_p = oracle.verlet(x0, p0, r, plane, dt, g, e, 1)
        got_x = sph[:, :3].cpu().numpy()
        got_p = pv.cpu().numpy()
        err = max(np.abs(got_x - want_x).max(), np.abs(got_p - want_p).max())
        worst = max(worst, err)
        assert err < 4e-6 * max(1.0, np.abs(want_x).max()), err
    print("worst step error", worst)
    assert np.all(sph[:, 1].cpu().numpy() >= w.scene.spheres[:, 3] - 1e-4)  # never below the plane


def test_verlet_free_fall_many_steps():
    rng = np.random.default_rng(9)
    n = 1000
    rec = np.zeros((n, 10), np.float32)
    rec[:, :3] = rng.uniform(-5, 5, (n, 3))
    rec[:, 3] = 0.5
    v0 = rng.uniform(-2, 2, (n, 3))
    dt, g, steps = 1.0 / 60.0, 9.81, 120
    prev = (rec[:, :3] - v0 * dt).astype(np.float32)
    sph = torch.from_numpy(rec).cuda()
    pv = torch.from_numpy(prev).cuda()
    rt.verlet_step(sph, pv, None, dt=dt, gravity=g, restitution=0.5, steps=steps)
    want, _ = oracle.verlet(rec[:, :3].astype(np.float64), prev.astype(np.float64), rec[:, 3], None, dt, g, 0.5,
                            steps)
    got = sph[:, :3].cpu().numpy()
    # FP32 rounding of a step (a few ulps of |x|) carries into every later position
    # once per remaining step: bound 3 u max|x| n (n + 1) / 2, u = 2^-24
    bound = 3 * 2.0 ** -24 * np.abs(want).max() * steps * (steps + 1) / 2
    err = np.abs(got - want).max()
    print("free fall error", err, "bound", bound)
    assert err < bound, (err, bound)


def test_animated_frames_equal_host_upload_and_oracle():
    w, prev = S.animated_scene(160, 96)
    w.params.out_format = S.OUT_F32
    an = animate.Animation(w, prev)
    for _ in range(45):
        an.step(readback=False)
    frame = an.step(readback=True)
    torch.cuda.synchronize()
    got = frame.numpy().copy()
    rec = an.spheres.cpu().numpy()
    moved = copy.deepcopy(w)
    moved.scene.spheres = np.ascontiguousarray(rec)
    fresh, _ = gpu_render(moved)
    assert np.array_equal(got, fresh)                       # device update == host upload
    ref, margin, sens = oracle_reference(moved)
    ok, st = compare_f32(got[..., :3].reshape(-1, 3), ref, margin, sens, moved.scene.scene_scale)
    print(st)
    assert st["failing"] == 0, st
    assert not np.allclose(rec[:, 1], w.scene.spheres[:, 1])  # the bodies moved
    an.close()


def test_refusals():
    w = with_sky(S.whitted_256())
    ds = rt.DeviceScene(w.scene)
    p = copy.copy(w.params)
    dl = torch.zeros((p.height, p.width, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(rt.RtError) as e:
        rt.render_backward(ds, w.camera, p, dl)
    assert e.value.status == 4
    sph = torch.zeros((2, 10), dtype=torch.float32, device="cuda")
    pv = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    for kw in ({"restitution": 1.5}, {"dt": 0.0}, {"dt": -1.0}):
        with pytest.raises(rt.RtError) as e:
            rt.verlet_step(sph, pv, None, **kw)
        assert e.value.status == 1
    with pytest.raises(rt.RtError):
        rt.verlet_step(sph, pv, [0.0, 2.0, 0.0, 0.0])   # non-unit plane normal
    bad = SKY.copy()
    bad[3, 5, 1] = np.inf
    with pytest.raises(rt.RtError):
        ds.set_sky(bad)
    ds.close()
