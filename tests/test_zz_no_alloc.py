"""sonar_render_noalloc: the render entry point for callers that cannot
allocate device memory (a fixed-budget engine that owns all its device
memory, or real-time code where an allocation could block or synchronise).
Its scratch is a fixed array inside the library, so these tests check that
consecutive calls, which reuse that array, give the same images as
sonar_render, and that frames too large for the array are refused.

This file is collected last on purpose; it also runs on its own in a fresh
process (it creates its own context and scene)."""
import ctypes as C

import numpy as np
import pytest

from paper_2503_01074_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300 import sonar as SB  # noqa: E402
from paper_2503_01074_gb300.sonar import RenderParams, Sonar  # noqa: E402

RTOL, ATOL = 1e-4, 1e-6      # the bin tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    son = Sonar(0)
    mesh, mu = S.tiny_scene()
    sid = son.upload_mesh(mesh)
    yield son, sid, mu
    son.close()


def noalloc(son, sid, spec, theta, prm, seed, frame, polar, fan=None, noised=None):
    out = SB.Outputs(polar.data_ptr(), noised.data_ptr() if noised is not None else None, None, None,
                     fan.data_ptr() if fan is not None else None,
                     fan.shape[1] if fan is not None else 0, fan.shape[0] if fan is not None else 0)
    sensor = SB.to_sensor(spec)
    p = prm.c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return son.lib.sonar_render_noalloc(son.h, sid, C.byref(sensor), C.byref(p), C.c_void_p(theta.data_ptr()),
                                        theta.shape[0] - 2, seed, frame, C.byref(out), stream)


def test_consecutive_calls_match_sonar_render(env):
    son, sid, mu = env
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    cases = []
    a = S.sensor_tiny(40.0)                                  # with a fan
    b = S.sensor_tiny(35.0)
    b.n_range_bins, b.n_az_bins, b.fan_w, b.fan_h = 300, 96, 0, 0   # another shape, no fan
    cases = [(a, 1, 2), (b, 7, 9), (a, 3, 4)]
    for spec, seed, frame in cases:
        polar = torch.full((spec.n_range_bins, spec.n_az_bins), -7.0, device=son.device)
        fan = torch.full((spec.fan_h, spec.fan_w), -7.0, device=son.device) if spec.fan_w else None
        st = noalloc(son, sid, spec, theta, prm, seed, frame, polar, fan)
        assert st == SB.OK, son.lib.sonar_last_error(son.h)
        ref = son.render(sid, spec, theta, prm, seed, frame, fan=bool(spec.fan_w))
        torch.cuda.synchronize()
        assert torch.allclose(polar, ref["polar"], rtol=RTOL, atol=ATOL)
        if fan is not None:
            assert torch.allclose(fan, ref["fan"], rtol=RTOL, atol=ATOL)
    st, bits = son.check()
    assert st == 0 and bits == 0


def test_oversized_frame_is_refused(env):
    son, sid, mu = env
    theta = son.theta(0.05, 1.0, mu)
    spec = S.sensor_tiny(40.0)
    spec.n_range_bins, spec.n_az_bins, spec.fan_w, spec.fan_h = 4000, 1024, 0, 0   # 4.1M bins > 1M words
    polar = torch.empty((4000, 1024), device=son.device)
    st = noalloc(son, sid, spec, theta, RenderParams(), 0, 0, polar)
    assert st == SB.ERR_ARG
    assert b"scratch" in son.lib.sonar_last_error(son.h)
    # with the caller's own noised buffer only the row maxima need the fixed scratch
    noised = torch.empty_like(polar)
    st = noalloc(son, sid, spec, theta, RenderParams(), 0, 0, polar, noised=noised)
    assert st == SB.OK, son.lib.sonar_last_error(son.h)
    ref = son.render(sid, spec, theta, RenderParams(), 0, 0, fan=False)
    torch.cuda.synchronize()
    assert torch.allclose(polar, ref["polar"], rtol=RTOL, atol=ATOL)
