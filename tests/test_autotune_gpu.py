"""Autotuner: picks a measured launch shape, caches it, and never changes the
image (every candidate renders bit-identically)."""
import numpy as np
import pytest
import torch

from paper_2305_07450_b300 import autotune, rt, scenes as S

pytestmark = pytest.mark.gpu


def test_tune_render_caches_and_keeps_results(tmp_path, monkeypatch):
    monkeypatch.setenv("RT_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    autotune._mem.clear()
    w = S.whitted_720p()
    w.params.width, w.params.height = 320, 180
    ds = rt.DeviceScene(w.scene)
    launch = autotune.tune_render(ds, w.scene, w.camera, w.params, reps=2, force=True)
    assert (launch["block_x"], launch["block_y"]) in autotune.FWD_CANDIDATES
    autotune._mem.clear()
    assert autotune.lookup(autotune.key_for(w.scene, w.params))["launch"] == launch
    a = rt.render(ds, w.camera, w.params, launch=launch).cpu().numpy()
    b = rt.render(ds, w.camera, w.params).cpu().numpy()
    assert np.array_equal(a, b)


def test_tune_batch(tmp_path, monkeypatch):
    monkeypatch.setenv("RT_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    autotune._mem.clear()
    ws = S.batch_scenes(5, seed0=800)
    dss = [rt.DeviceScene(w.scene) for w in ws]
    launch = autotune.tune_batch(dss, [w.scene for w in ws], [w.camera for w in ws], [w.params for w in ws],
                                 reps=1, force=True)
    assert (launch["block_x"], launch["block_y"]) in autotune.BATCH_CANDIDATES
    b = rt.Batch(dss, [w.camera for w in ws], [w.params for w in ws], launch=launch)
    b.launch()
    torch.cuda.synchronize()
    for w, d, o in zip(ws, dss, b.outputs()):
        assert torch.equal(o, rt.render(d, w.camera, w.params))
