"""The C-ABI library loads, exports every function include/*.h declares, agrees
with the Python structures on layout, and rejects bad arguments on the host
before touching the device (CPU only: no compute call is made)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2305_07450_b300 import build, rt
    build.build()
    return rt.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(rt_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 8, names
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\S+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_struct_layouts_match_header(tmp_path):
    from paper_2305_07450_b300 import rt
    probe = tmp_path / "probe.c"
    probe.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{ROOT}/include/rt.h"
int main(void) {{
  printf("%zu %zu %zu %zu\\n", sizeof(rt_scene_desc), sizeof(rt_camera), sizeof(rt_render_params), sizeof(rt_launch_config));
  printf("%zu %zu %zu\\n", offsetof(rt_scene_desc, lights), offsetof(rt_render_params, seed), offsetof(rt_render_params, eps));
  return 0;
}}''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(probe)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")[:2]
    assert [int(v) for v in a.split()] == [C.sizeof(rt.SceneDesc), C.sizeof(rt.Camera), C.sizeof(rt.RenderParams),
                                           C.sizeof(rt.LaunchConfig)]
    assert [int(v) for v in b.split()] == [rt.SceneDesc.lights.offset, rt.RenderParams.seed.offset,
                                           rt.RenderParams.eps.offset]


def test_status_strings(L):
    assert L.rt_status_string(0) == b"RT_OK"
    assert L.rt_status_string(1) == b"RT_ERR_INVALID_ARG"
    assert L.rt_status_string(5) == b"RT_ERR_TIMEOUT"
    assert L.rt_launch_count() >= 0


def test_host_validation_rejects_before_any_launch(L):
    from paper_2305_07450_b300 import rt
    import numpy as np
    before = L.rt_launch_count()
    h = C.c_void_p()
    assert L.rt_scene_upload(None, None, C.byref(h)) == 1
    d = rt.SceneDesc()
    d.n_spheres = -1
    assert L.rt_scene_upload(C.byref(d), None, C.byref(h)) == 1
    # a sphere with a negative radius, and one with NaN
    for bad in ([0, 0, 0, -1, 1, 1, 1, 0.5, 32, 0], [0, 0, float("nan"), 1, 1, 1, 1, 0.5, 32, 0]):
        sph = np.array(bad, np.float32)
        d = rt.SceneDesc()
        d.n_spheres, d.spheres = 1, sph.ctypes.data
        assert L.rt_scene_upload(C.byref(d), None, C.byref(h)) == 1
    # a light inside a sphere: valid input the library does not handle
    sph = np.array([0, 5, 0, 2, 1, 1, 1, 0.5, 32, 0], np.float32)
    lig = np.array([0, 5.5, 0, 1, 0, 0, 0, 0], np.float32)
    d = rt.SceneDesc()
    d.n_spheres, d.spheres, d.n_lights, d.lights = 1, sph.ctypes.data, 1, lig.ctypes.data
    assert L.rt_scene_upload(C.byref(d), None, C.byref(h)) == 4
    # render without a scene / params
    cam = rt.Camera()
    p = rt.RenderParams()
    assert L.rt_render(None, C.byref(cam), C.byref(p), None, 0, None, None, None) == 1
    assert L.rt_hitrec_bytes(None, C.byref(p)) == 0
    # queued render: no workspace, a misaligned one, one below the 256-byte control block
    buf = (C.c_uint8 * 4096)()
    base = (C.addressof(buf) + 255) // 256 * 256
    assert L.rt_render_ws(None, C.byref(cam), C.byref(p), None, 0, None, None, None, 4096, None) == 1
    assert L.rt_render_ws(None, C.byref(cam), C.byref(p), None, 0, None, None, base + 16, 2048, None) == 1
    assert L.rt_render_ws(None, C.byref(cam), C.byref(p), None, 0, None, None, base, 255, None) == 1
    assert L.rt_render_ws(None, C.byref(cam), C.byref(p), None, 0, None, None, base, 2048, None) == 1
    assert L.rt_render_workspace_bytes(None, C.byref(p)) == 0
    assert L.rt_launch_count() == before
