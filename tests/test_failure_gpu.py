"""Failure detection without a GPU fault: a bounded device wait that nothing
satisfies gives up, reports RT_ERR_TIMEOUT through the error word, and the
context keeps working; invalid arguments are refused before any launch."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2305_07450_b300 import rt, scenes as S

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    assert rt.device_errors() == 0
    st = rt.lib().rt_selftest_wait_timeout(4096, rt._stream(None))
    assert st == 0
    bits = C.c_uint32(0)
    assert rt.lib().rt_device_errors(rt._stream(None), C.byref(bits)) == 5  # RT_ERR_TIMEOUT
    assert bits.value & 1
    assert rt.device_errors() == 0  # read clears the word
    # the context is still usable: a render runs and is correct
    w = S.whitted_256()
    w.params.width = w.params.height = 32
    ds = rt.DeviceScene(w.scene)
    img = rt.render(ds, w.camera, w.params)
    torch.cuda.synchronize()
    assert np.isfinite(img.cpu().numpy()).all() and img.abs().sum() > 0


def test_invalid_arguments_are_refused_on_the_host():
    w = S.whitted_256()
    ds = rt.DeviceScene(w.scene)
    n0 = rt.launch_count()
    bad = S.Params(width=0, height=16)
    with pytest.raises(rt.RtError):
        rt.render(ds, w.camera, bad, out=torch.empty(16, 4, device="cuda"), pitch=16)
    with pytest.raises(rt.RtError):
        rt.render(ds, w.camera, w.params, out=torch.empty(64, device="cuda")[1:], pitch=20)
    assert rt.lib().rt_selftest_wait_timeout(0, None) == 1
    assert rt.launch_count() == n0
