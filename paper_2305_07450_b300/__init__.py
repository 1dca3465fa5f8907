"""B300 (sm_103a) per-pixel Whitted ray tracer of arXiv 2305.07450 (Section 3).

``scenes`` (seeded inputs) imports without CUDA.  The device binding (``rt``) is
loaded on first use of one of its names; it raises if ``librt.so`` is missing.
"""
from . import scenes  # noqa: F401

_RT_NAMES = {"DeviceScene", "render", "alloc_output", "hitrec_bytes", "device_errors",
             "launch_count", "RtError", "lib"}


def __getattr__(name):
    if name in _RT_NAMES:
        from . import rt
        return getattr(rt, name)
    raise AttributeError(name)
