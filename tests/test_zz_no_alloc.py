"""sonar_render_noalloc: the render entry point for callers that cannot
allocate device memory (a fixed-budget engine that owns all its device
memory, or real-time code where an allocation could block or synchronise).
Its scratch is a fixed array inside the library.  Consecutive calls reuse
that array, so these tests check, call after call, that the images are bit
for bit those of sonar_render (the same kernels and launch shapes), including
the whole-image maximum that lives in the array and must be cleared on every
call; that warm calls leave the device's free memory unchanged; and that
frames too large for the array are refused.

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


@pytest.fixture(scope="module")
def env():
    son = Sonar(0)
    mesh, mu = S.tiny_scene()
    sid = son.upload_mesh(mesh)
    soup = S.random_soup(300, seed=4)
    sid2 = son.upload_mesh(soup)
    yield son, sid, mu, sid2, np.array([0.2, 0.4, 0.6, 0.8], np.float32)
    son.close()


def noalloc(son, sid, spec, theta, prm, seed, frame, polar, fan=None, noised=None, hits=None):
    out = SB.Outputs(polar.data_ptr(), noised.data_ptr() if noised is not None else None, None,
                     hits.data_ptr() if hits is not None else None,
                     fan.data_ptr() if fan is not None else None,
                     fan.shape[1] if fan is not None else 0, fan.shape[0] if fan is not None else 0)
    sensor = SB.to_sensor(spec)
    p = prm.c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return son.lib.sonar_render_noalloc(son.h, sid, C.byref(sensor), C.byref(p), C.c_void_p(theta.data_ptr()),
                                        theta.shape[0] - 2, seed, frame, C.byref(out), stream)


def fresh(spec, dev, fan=True):
    polar = torch.full((spec.n_range_bins, spec.n_az_bins), -7.0, device=dev)
    f = torch.full((spec.fan_h, spec.fan_w), -7.0, device=dev) if (fan and spec.fan_w) else None
    return polar, f


def assert_same_as_render(son, sid, spec, theta, prm, seed, frame, polar, fan=None, hits=None):
    ref = son.render(sid, spec, theta, prm, seed, frame, hits=hits is not None, fan=fan is not None)
    torch.cuda.synchronize()
    assert torch.equal(polar, ref["polar"]), (seed, frame, "polar")
    if fan is not None:
        assert torch.equal(fan, ref["fan"]), (seed, frame, "fan")
    if hits is not None:
        assert torch.equal(hits, ref["hits"]), (seed, frame, "hits")


def test_consecutive_calls_match_sonar_render(env):
    """Three calls in a row, two sensor shapes, hit records and I~ kept in
    the fixed array, with and without a fan: each equals sonar_render."""
    son, sid, mu, _, _ = env
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    a = S.sensor_tiny(40.0)                                  # with a fan
    b = S.sensor_tiny(35.0)
    b.n_range_bins, b.n_az_bins, b.fan_w, b.fan_h = 300, 96, 0, 0   # another shape, no fan
    for spec, seed, frame in [(a, 1, 2), (b, 7, 9), (a, 3, 4)]:
        polar, fan = fresh(spec, son.device)
        st = noalloc(son, sid, spec, theta, prm, seed, frame, polar, fan)
        assert st == SB.OK, son.lib.sonar_last_error(son.h)
        assert_same_as_render(son, sid, spec, theta, prm, seed, frame, polar, fan)
    st, bits = son.check()
    assert st == 0 and bits == 0


def test_caller_hit_records_and_fan(env):
    """The caller's own hit-record buffer (the records then do not use the
    array) and a fan: records, image and fan equal sonar_render's, twice."""
    son, sid, mu, _, _ = env
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    spec = S.sensor_tiny(40.0)
    for seed in (5, 6):
        polar, fan = fresh(spec, son.device)
        hits = torch.full((spec.n_rays, 4), -1, dtype=torch.int32, device=son.device)
        st = noalloc(son, sid, spec, theta, prm, seed, seed, polar, fan, hits=hits)
        assert st == SB.OK, son.lib.sonar_last_error(son.h)
        assert_same_as_render(son, sid, spec, theta, prm, seed, seed, polar, fan, hits)


def test_global_maximum_cleared_between_calls(env):
    """Whole-image normalisation keeps its running maximum in word 0 of the
    array.  A large gain first, then small gains on two scenes: a maximum
    left over from the previous call would scale the later images wrongly."""
    son, sid, mu, sid2, mu2 = env
    prm = RenderParams(normalise=2)
    spec = S.sensor_tiny(40.0)
    soup_spec = S.sensor_tiny(20.0)      # looks into the soup at 6 m ahead
    for scene, m, gain, spec_k in [(sid, mu, 20.0, spec), (sid, mu, 0.5, spec), (sid2, mu2, 0.25, soup_spec),
                                   (sid2, mu2, 0.25, soup_spec)]:
        theta = son.theta(0.05, gain, m)
        polar, fan = fresh(spec_k, son.device)
        st = noalloc(son, scene, spec_k, theta, prm, 11, 12, polar, fan)
        assert st == SB.OK, son.lib.sonar_last_error(son.h)
        assert_same_as_render(son, scene, spec_k, theta, prm, 11, 12, polar, fan)
        assert float(polar.max()) == 1.0


def test_warm_calls_leave_device_memory_unchanged(env):
    """After one warm-up call (which may load device code), further calls
    change neither the device's free memory nor torch's allocations."""
    son, sid, mu, _, _ = env
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    spec = S.sensor_tiny(40.0)
    polar, fan = fresh(spec, son.device)
    assert noalloc(son, sid, spec, theta, prm, 0, 0, polar, fan) == SB.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(son.device)
    alloc0 = torch.cuda.memory_allocated(son.device)
    for k in range(4):
        assert noalloc(son, sid, spec, theta, prm, k, k, polar, fan) == SB.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(son.device)
    assert free1 == free0 and torch.cuda.memory_allocated(son.device) == alloc0


def test_oversized_frame_is_refused(env):
    son, sid, mu, _, _ = env
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
    assert torch.equal(polar, ref["polar"])
