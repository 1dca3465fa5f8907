"""rt_render_batch_noalloc: the batched render for callers that must not allocate
device memory while rendering (an application or framework owns every device
allocation, or a frame loop cannot afford the device-wide synchronisation and the
run-time failure modes of cudaMalloc/cudaFree).  Its work tables live in a fixed
scratch array inside the library, so the caller passes only inputs and outputs.

Checked here through the C ABI against rt_render_batch (the entry point with a
caller workspace), on calls made back to back: outputs must be identical, since
both run the same kernel on the same work tables.  The limits are exercised at
their edges (exactly the frame limit, tables a few items under the scratch size)
and just beyond them; calls that must be refused still get real output buffers of
the size each frame needs.  Kept in its own file, collected last, so that a run
stopping at the first failure has run every other test; it also passes alone in a
fresh process (the first call performs the per-device set-up).
"""
import ctypes as C
import os
import re

import pytest
import torch

from paper_2305_07450_b300 import rt, scenes as S

pytestmark = pytest.mark.gpu

RT_ERR_UNSUPPORTED = 4
RT_ERR_EXCEEDS_SCRATCH = 6
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rt.h")


def header_limits():
    """(scratch bytes, frame limit) as the header defines them."""
    txt = open(HEADER).read()
    nb = re.search(r"#define RT_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", txt)
    nf = re.search(r"#define RT_NOALLOC_MAX_FRAMES (\d+)", txt)
    return int(nb.group(1)) << int(nb.group(2)), int(nf.group(1))


def call_noalloc(dss, cams, params, outs, pitches, launch=None, stream=None):
    n, sc, cm, prm, op, pt = rt._batch_arrays(dss, cams, params, outs, pitches)
    cfg = rt.launch_struct(launch)
    return rt.lib().rt_render_batch_noalloc(n, sc, cm, prm, op, pt, C.byref(cfg) if cfg is not None else None,
                                            rt._stream(stream))


TILE = {"block_x": 16, "block_y": 8}     # one work item per 16 x 8 pixels


def check_against_workspace_batch(dss, cams, params, launch=None):
    ref, _ = rt.render_batch(dss, cams, params, launch=launch)
    outs, pitches = rt.alloc_batch_outputs(params)
    for o in outs:
        o.fill_(-1)
    assert call_noalloc(dss, cams, params, outs, pitches, launch=launch) == 0
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    for i, (a, o, p) in enumerate(zip(ref, outs, params)):
        got = o if p.out_format == S.OUT_F32 else o[:, : p.width]
        assert torch.equal(a, got), (i, float((a.float() - got.float()).abs().max()))
    del ref, outs


def test_noalloc_matches_workspace_batch_on_consecutive_calls():
    batches = [S.batch_scenes(10, seed0=700), S.batch_scenes(7, seed0=900), S.batch_scenes(10, seed0=700)]
    for ws in batches:
        dss = [rt.DeviceScene(w.scene) for w in ws]
        check_against_workspace_batch(dss, [w.camera for w in ws], [w.params for w in ws])


def frames_filling_scratch(ds, eps, cap, spare_items):
    """Frame sizes (RGBA8, bounce limit 0) whose work tables -- header, frame records
    and one 4-byte item per 16 x 8 tile -- end exactly `spare_items` items under the
    scratch size (a negative count: that many items beyond it): 4096 x 4096 frames,
    one 4096-wide frame and one 16-wide frame for the remainder."""
    def prm(w, h):
        return S.Params(width=w, height=h, max_depth=0, out_format=S.OUT_RGBA8, eps=eps)
    tiny = prm(16, 8)

    def items_offset(n):
        return rt.batch_workspace_bytes([ds] * n, [tiny] * n, TILE) - 4 * n
    big = 256 * 512
    for k in range(64):
        n = k + 2
        avail = (cap - items_offset(n)) // 4 - spare_items
        if avail - k * big < big:
            break
    rem = avail - k * big
    mid, last = rem // 256, rem % 256
    if last == 0:
        mid, last = mid - 1, 256
    frames = [prm(4096, 4096)] * k + [prm(4096, 8 * mid), prm(16, 8 * last)]
    assert 0 < mid < 4096 and 0 < last <= 256
    need = rt.batch_workspace_bytes([ds] * len(frames), frames, TILE)
    assert need == cap - 4 * spare_items - (cap - items_offset(len(frames))) % 4, (need, cap)
    return frames


def test_noalloc_at_its_limits():
    """Exactly the frame limit, and tables three items under the scratch size, are
    accepted and equal the workspace batch."""
    cap, max_frames = header_limits()
    w = S.whitted_256()
    ds = rt.DeviceScene(w.scene)
    small = S.Params(width=16, height=8, max_depth=1, out_format=S.OUT_F32, eps=w.params.eps)
    check_against_workspace_batch([ds] * max_frames, [w.camera] * max_frames, [small] * max_frames, TILE)
    frames = frames_filling_scratch(ds, w.params.eps, cap, 3)
    check_against_workspace_batch([ds] * len(frames), [w.camera] * len(frames), frames, TILE)


def test_noalloc_rejects_work_beyond_its_scratch():
    cap, max_frames = header_limits()
    w = S.whitted_256()
    ds = rt.DeviceScene(w.scene)
    # tables one item beyond the scratch (sizes checked on the host above); every
    # frame still gets a real framebuffer of its full size
    frames = frames_filling_scratch(ds, w.params.eps, cap, -1)
    n = len(frames)
    outs, pitches = rt.alloc_batch_outputs(frames)
    st = call_noalloc([ds] * n, [w.camera] * n, frames, outs, pitches, launch=TILE)
    assert st == RT_ERR_EXCEEDS_SCRATCH
    assert rt.lib().rt_status_string(st) == b"RT_ERR_EXCEEDS_SCRATCH"
    del outs
    # one frame more than the frame limit, each with a real 16 x 8 framebuffer
    m = max_frames + 1
    small = S.Params(width=16, height=8, max_depth=1, out_format=S.OUT_F32, eps=w.params.eps)
    outs, pitches = rt.alloc_batch_outputs([small] * m)
    st = call_noalloc([ds] * m, [w.camera] * m, [small] * m, outs, pitches, launch=TILE)
    assert st == RT_ERR_EXCEEDS_SCRATCH
    torch.cuda.synchronize()
    assert rt.device_errors() == 0


def test_noalloc_refuses_stream_capture():
    """Under stream capture the call returns RT_ERR_UNSUPPORTED and enqueues nothing
    (the captured graph stays empty of its work and the outputs keep their fill)."""
    ws = S.batch_scenes(3, seed0=700)
    dss = [rt.DeviceScene(w.scene) for w in ws]
    cams, params = [w.camera for w in ws], [w.params for w in ws]
    outs, pitches = rt.alloc_batch_outputs(params)
    for o in outs:
        o.fill_(-7)
    torch.cuda.synchronize()
    n0 = rt.launch_count()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        g.capture_begin()
        st = call_noalloc(dss, cams, params, outs, pitches, stream=side)
        g.capture_end()
    assert st == RT_ERR_UNSUPPORTED
    assert rt.launch_count() == n0
    g.replay()
    torch.cuda.synchronize()
    for o in outs:
        assert bool((o == -7).all())
    # the entry point works again outside the capture
    check_against_workspace_batch(dss, cams, params)
