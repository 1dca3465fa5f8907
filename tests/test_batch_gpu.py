"""Batched persistent render (rt_render_batch, rt_batch_* CUDA graph): output
bit-identical to per-frame rt_render, replays identical, parity with the oracle on
a small batch and on every pixel of the 64-scene batch."""
import numpy as np
import pytest
import torch

from paper_2305_07450_b300 import rt, scenes as S
from parity import compare_f32, oracle_reference

pytestmark = pytest.mark.gpu


def per_frame(ws, dss, launch=None):
    outs = []
    for w, d in zip(ws, dss):
        outs.append(rt.render(d, w.camera, w.params, launch=launch).cpu().numpy())
    return outs


def test_batch_64_scenes_bitwise_equal_per_frame():
    """The 64-scene batch (sphere counts log-uniform in [8, 512], 1-4 lights,
    depth 1-6, four resolutions) in one graph launch equals 64 rt_render calls."""
    ws = S.batch_scenes()
    dss = [rt.DeviceScene(w.scene) for w in ws]
    ref = per_frame(ws, dss)
    b = rt.Batch(dss, [w.camera for w in ws], [w.params for w in ws])
    b.launch()
    torch.cuda.synchronize()
    got = [o.cpu().numpy() for o in b.outputs()]
    for i, (a, c) in enumerate(zip(ref, got)):
        assert np.array_equal(a, c), (i, ws[i].name)
    # replay: identical again (the graph resets the work counter)
    for o in b.outs:
        o.zero_()
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    for i, (a, o) in enumerate(zip(ref, b.outputs())):
        assert np.array_equal(a, o.cpu().numpy()), i
    assert rt.device_errors() == 0
    b.close()


def test_render_batch_workspace_path_and_staging_modes():
    ws = S.batch_scenes(12, seed0=300)
    dss = [rt.DeviceScene(w.scene) for w in ws]
    ref = per_frame(ws, dss)
    for launch in (None, {"staging": 2}, {"block_x": 8, "block_y": 8, "min_blocks_per_sm": 1}, {"block_x": 32, "block_y": 4},
                   {"staging": 3}):
        outs, _ = rt.render_batch(dss, [w.camera for w in ws], [w.params for w in ws], launch=launch)
        torch.cuda.synchronize()
        for i, (a, o) in enumerate(zip(ref, outs)):
            assert np.array_equal(a, o.cpu().numpy()), (launch, i)
    assert rt.device_errors() == 0


def test_small_batch_matches_oracle():
    ws = S.batch_scenes(6, seed0=500)
    for w in ws:
        w.params.width, w.params.height = 64, 48
    dss = [rt.DeviceScene(w.scene) for w in ws]
    outs, _ = rt.render_batch(dss, [w.camera for w in ws], [w.params for w in ws])
    torch.cuda.synchronize()
    for w, o in zip(ws, outs):
        ref, margin, sens = oracle_reference(w)
        ok, st = compare_f32(o.cpu().numpy()[..., :3].reshape(-1, 3), ref, margin, sens, w.scene.scene_scale)
        assert st["failing"] == 0 and st["frac_within_1e-4"] >= 0.98, (w.name, st)


def test_bounce_queues_rgba8_and_deep_mirrors():
    """Frames of the line-filter class with bounce limits 1..16 defer their
    bounce-1 paths to the batch's bounce queues; RGBA8 frames (four lanes share a
    store, a deferred pixel is overwritten by the pass that finishes it) and a
    scene of mirror spheres whose paths run to bounce 16 equal rt_render bit for
    bit, and so do the frames of the segment-test class in the same batch."""
    ws = S.batch_scenes(10, seed0=800)
    sc = S.random_scene(901, 160, 2, 3.0)
    sc.spheres = sc.spheres.copy()
    sc.spheres[:, 9] = np.float32(0.9)                  # mirrors: long reflection chains
    ws.append(S.Workload("mirrors_d16", sc, S.default_camera(3.0),
                         S._params(sc, width=200, height=120, max_depth=16, seed=901)))
    for i, w in enumerate(ws):
        if i % 2 == 0:
            w.params.out_format = S.OUT_RGBA8
    assert any(w.scene.n_spheres >= 121 and w.params.max_depth >= 1 for w in ws)
    dss = [rt.DeviceScene(w.scene) for w in ws]
    ref = per_frame(ws, dss)
    outs, _ = rt.render_batch(dss, [w.camera for w in ws], [w.params for w in ws])
    b = rt.Batch(dss, [w.camera for w in ws], [w.params for w in ws])
    b.launch()
    torch.cuda.synchronize()
    for i, (a, o, g) in enumerate(zip(ref, outs, b.outputs())):
        assert np.array_equal(a, o.cpu().numpy()), (i, ws[i].name)
        assert np.array_equal(a, g.cpu().numpy()), (i, ws[i].name)
    assert rt.device_errors() == 0
    b.close()


def test_batch_64_scenes_every_pixel_against_oracle():
    """The 64-scene batch through one graph launch (the bench's batched path): every
    pixel of every frame in FP32 within 1e-4 of the oracle or exempt, the exempt share
    of the batch bounded as for the 4K frame."""
    from parity import EXEMPT_SHARE_MAX
    ws = S.batch_scenes()
    dss = [rt.DeviceScene(w.scene) for w in ws]
    b = rt.Batch(dss, [w.camera for w in ws], [w.params for w in ws])
    b.launch()
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    got = [o.cpu().numpy() for o in b.outputs()]
    b.close()
    pixels = exempt = 0
    for w, img in zip(ws, got):
        ref, margin, sens = oracle_reference(w)
        ok, st = compare_f32(img[..., :3].reshape(-1, 3), ref, margin, sens, w.scene.scene_scale)
        assert st["failing"] == 0, (w.name, st)
        pixels += st["pixels"]
        exempt += st["pixels"] - st["plain"]
    print(f"batch: {pixels} pixels, {exempt} exempt")
    assert exempt <= EXEMPT_SHARE_MAX * pixels
