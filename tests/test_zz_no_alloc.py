"""rt_render_batch_noalloc: the batched render for callers that must not allocate
device memory while rendering (an application or framework owns every device
allocation, or a frame loop cannot afford the device-wide synchronisation and the
run-time failure modes of cudaMalloc/cudaFree).  Its work tables live in a fixed
scratch array inside the library, so the caller passes only inputs and outputs.

Checked here through the C ABI against rt_render_batch (the entry point with a
caller workspace), on calls made back to back: outputs must be identical, since
both run the same kernel on the same work tables.  Kept in its own file, collected
last, so that a run stopping at the first failure has run every other test; it
also passes alone in a fresh process (the first call performs the per-device
set-up).
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2305_07450_b300 import rt, scenes as S

pytestmark = pytest.mark.gpu

RT_ERR_EXCEEDS_SCRATCH = 6


def call_noalloc(dss, cams, params, outs, pitches, launch=None):
    n, sc, cm, prm, op, pt = rt._batch_arrays(dss, cams, params, outs, pitches)
    cfg = rt.launch_struct(launch)
    return rt.lib().rt_render_batch_noalloc(n, sc, cm, prm, op, pt, C.byref(cfg) if cfg is not None else None,
                                            rt._stream(None))


def test_noalloc_matches_workspace_batch_on_consecutive_calls():
    batches = [S.batch_scenes(10, seed0=700), S.batch_scenes(7, seed0=900), S.batch_scenes(10, seed0=700)]
    for ws in batches:
        dss = [rt.DeviceScene(w.scene) for w in ws]
        cams, params = [w.camera for w in ws], [w.params for w in ws]
        ref, _ = rt.render_batch(dss, cams, params)
        outs, pitches = rt.alloc_batch_outputs(params)
        for o in outs:
            o.fill_(-1)
        assert call_noalloc(dss, cams, params, outs, pitches) == 0
        torch.cuda.synchronize()
        assert rt.device_errors() == 0
        for i, (a, o, p) in enumerate(zip(ref, outs, params)):
            got = o if p.out_format == S.OUT_F32 else o[:, : p.width]
            assert torch.equal(a, got), (ws[i].name, float((a.float() - got.float()).abs().max()))


def test_noalloc_rejects_work_beyond_its_scratch():
    w = S.whitted_256()
    ds = rt.DeviceScene(w.scene)
    dummy = torch.empty(16, dtype=torch.float32, device="cuda")
    big = S.Params(width=4096, height=4096, max_depth=1, out_format=S.OUT_F32, eps=w.params.eps)
    # 8 frames x 131072 tiles of 16 x 8 pixels: 4 MiB of items, beyond the scratch
    st = call_noalloc([ds] * 8, [w.camera] * 8, [big] * 8, [dummy] * 8, [4096 * 16] * 8)
    assert st == RT_ERR_EXCEEDS_SCRATCH
    assert rt.lib().rt_status_string(st) == b"RT_ERR_EXCEEDS_SCRATCH"
    # more frames than the scratch's frame limit
    st = call_noalloc([ds] * 300, [w.camera] * 300, [w.params] * 300, [dummy] * 300, [256 * 16] * 300)
    assert st == RT_ERR_EXCEEDS_SCRATCH
