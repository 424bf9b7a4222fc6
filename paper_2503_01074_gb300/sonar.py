"""Python binding of libsonar (include/sonar.h), argument marshalling only.

Every step of the sonar path runs in the CUDA library; PyTorch supplies
device memory and the current stream.  There is no CPU fallback: if the
library is missing or fails to load, the first call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsonar.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_DEVICE, ERR_STATE = range(7)
DEVERR_STACK, DEVERR_INDEX, DEVERR_TIMEOUT = 1, 2, 4
NO_KEY = 0xFFFFFFFF


class SonarError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libsonar status {status}: {message}")
        self.status = status


# ---- C structs ----------------------------------------------------------------

class Sensor(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("rot", C.c_float * 9), ("n_beams", C.c_int32),
                ("n_elev", C.c_int32), ("n_range_bins", C.c_int32), ("n_az_bins", C.c_int32),
                ("hfov", C.c_float), ("vfov", C.c_float), ("r_min", C.c_float), ("r_max", C.c_float)]


class Params(C.Structure):
    _fields_ = [("sigma_sa", C.c_float), ("sigma_sm", C.c_float), ("sigma_phi", C.c_float),
                ("normalise", C.c_int32), ("two_sided", C.c_int32), ("clip_tmax", C.c_int32),
                ("accumulate", C.c_int32), ("reserved", C.c_int32)]


class Outputs(C.Structure):
    _fields_ = [("polar", C.c_void_p), ("noised", C.c_void_p), ("binned", C.c_void_p),
                ("hits", C.c_void_p), ("fan", C.c_void_p), ("fan_w", C.c_int32),
                ("fan_h", C.c_int32)]


class BatchItem(C.Structure):
    _fields_ = [("scene_id", C.c_int32), ("fan_w", C.c_int32), ("fan_h", C.c_int32),
                ("reserved", C.c_int32), ("sensor", Sensor), ("seed", C.c_uint64),
                ("frame", C.c_uint64), ("polar_offset", C.c_int64), ("hits_offset", C.c_int64),
                ("fan_offset", C.c_int64)]


class BatchOutputs(C.Structure):
    _fields_ = [("polar", C.c_void_p), ("noised", C.c_void_p), ("binned", C.c_void_p),
                ("hits", C.c_void_p), ("fan", C.c_void_p)]


class DvlParams(C.Structure):
    """DVL configuration (include/sonar.h: sonar_dvl_params)."""
    _fields_ = [("tilt", C.c_float), ("r_min", C.c_float), ("r_max", C.c_float), ("min_beams", C.c_int32),
                ("sigma_b", C.c_float), ("t0", C.c_float), ("t1", C.c_float), ("t_lost", C.c_float)]

    def __init__(self, tilt=math.radians(30.0), r_min=0.3, r_max=50.0, min_beams=3, sigma_b=0.01, t0=0.05,
                 t1=4.0 * 2.0 / 1500.0, t_lost=1.0):
        super().__init__(tilt, r_min, r_max, min_beams, sigma_b, t0, t1, t_lost)


HIT_DTYPE = np.dtype([("key", "<u4"), ("tri", "<u4"), ("r", "<f4"), ("cos", "<f4")])

# name -> (restype, argtypes); every symbol declared in include/sonar.h
_SIG = {
    "sonar_version": (C.c_char_p, []),
    "sonar_create": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p)]),
    "sonar_destroy": (C.c_int, [C.c_void_p]),
    "sonar_last_error": (C.c_char_p, [C.c_void_p]),
    "sonar_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32)]),
    "sonar_scene_upload": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_int64, C.c_void_p, C.POINTER(C.c_int32)]),
    "sonar_scene_release": (C.c_int, [C.c_void_p, C.c_int32]),
    "sonar_scene_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "sonar_render": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Sensor), C.POINTER(Params),
                               C.c_void_p, C.c_int32, C.c_uint64, C.c_uint64,
                               C.POINTER(Outputs), C.c_void_p]),
    "sonar_render_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Sensor), C.POINTER(Params),
                                       C.c_void_p, C.c_int32, C.c_uint64, C.c_uint64,
                                       C.POINTER(Outputs), C.c_void_p]),
    "sonar_fan_resample": (C.c_int, [C.c_void_p, C.POINTER(Sensor), C.c_void_p, C.c_int32,
                                     C.c_int32, C.c_void_p, C.c_void_p]),
    "sonar_render_backward": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Sensor), C.POINTER(Params),
                                        C.c_void_p, C.c_int32, C.c_uint64, C.c_uint64, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sonar_batch_create": (C.c_int, [C.c_void_p, C.POINTER(BatchItem), C.c_int32,
                                     C.POINTER(C.c_void_p)]),
    "sonar_batch_update": (C.c_int, [C.c_void_p, C.POINTER(BatchItem), C.c_int32, C.c_void_p]),
    "sonar_render_batch": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_int32,
                                     C.POINTER(BatchOutputs), C.c_void_p]),
    "sonar_render_batch_backward": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_int32,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p]),
    "sonar_render_batch_step": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_int32,
                                          C.POINTER(BatchOutputs), C.c_void_p, C.c_void_p, C.c_void_p]),
    "sonar_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "sonar_batch_kernels": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "sonar_batch_timings": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "sonar_batch_destroy": (C.c_int, [C.c_void_p]),
    "sonar_autotune": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_int32,
                                 C.POINTER(BatchOutputs), C.c_void_p]),
    "sonar_tune_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32,
                                 C.POINTER(C.c_int32)]),
    "sonar_tune_set": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "sonar_uw_image": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float),
                                 C.c_void_p, C.c_void_p]),
    "sonar_dvl": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(DvlParams),
                            C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sonar_dvl_schedule": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_float, C.c_void_p,
                                     C.c_void_p]),
    "sonar_trace_stats": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Sensor), C.POINTER(Params),
                                    C.c_void_p, C.POINTER(C.c_int64)]),
    "sonar_probe_l2_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int32,
                                      C.c_void_p]),
    "sonar_philox": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p]),
}

_LIB = None


def load_library(path: str = LIB_PATH):
    """Loads libsonar.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise ImportError(f"libsonar.so not built ({path}); run __graft_entry__.build() or "
                              "python paper_2503_01074_gb300/build.py")
        L = C.CDLL(path)
        for name, (res, args) in _SIG.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIG)


# ---- helpers ----------------------------------------------------------------

def to_sensor(spec) -> Sensor:
    s = Sensor()
    s.pos[:] = [float(x) for x in np.asarray(spec.pos, np.float32).reshape(3)]
    s.rot[:] = [float(x) for x in np.asarray(spec.rot, np.float32).reshape(9)]
    s.n_beams, s.n_elev = int(spec.n_beams), int(spec.n_elev)
    s.n_range_bins, s.n_az_bins = int(spec.n_range_bins), int(spec.n_az_bins)
    s.hfov, s.vfov = float(spec.hfov), float(spec.vfov)
    s.r_min, s.r_max = float(spec.r_min), float(spec.r_max)
    return s


@dataclass
class RenderParams:
    sigma_sa: float = 0.3
    sigma_sm: float = 0.01
    sigma_phi: float = 1.0
    normalise: int = 1
    two_sided: int = 1
    clip_tmax: int = 1      # 1: the cast ends at r_max; 0: unbounded (same images)
    accumulate: int = 0

    def c(self) -> Params:
        return Params(self.sigma_sa, self.sigma_sm, self.sigma_phi, self.normalise, self.two_sided,
                      self.clip_tmax, self.accumulate, 0)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _keep(tmp, orig, stream):
    """A contiguous copy `tmp` of `orig` that a call reads on `stream`: when it
    is a new tensor and the stream is not torch's current one, the caching
    allocator is told that the stream uses it, so that its memory is not
    handed to other work before the queued kernels have read it."""
    if stream is not None and tmp.data_ptr() != orig.data_ptr():
        tmp.record_stream(stream)
    return tmp


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Sonar:
    """A libsonar context on one CUDA device (torch tensors in, torch tensors out)."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        h = C.c_void_p()
        st = self.lib.sonar_create(device, C.byref(h))
        if st != OK:
            raise SonarError(st, "sonar_create failed")
        self.h = h
        self._scenes = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.sonar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise SonarError(st, self.lib.sonar_last_error(self.h).decode())

    def check(self):
        bits = C.c_uint32()
        st = self.lib.sonar_check(self.h, C.byref(bits))
        return st, bits.value

    # ---- scenes ----
    def upload(self, verts, tris, mat, stream=None) -> int:
        t = self.torch
        v = t.as_tensor(np.ascontiguousarray(verts, np.float32) if isinstance(verts, np.ndarray) else verts,
                        device=self.device, dtype=t.float32).contiguous()
        f = t.as_tensor(np.ascontiguousarray(tris, np.int32) if isinstance(tris, np.ndarray) else tris,
                        device=self.device, dtype=t.int32).contiguous()
        m = t.as_tensor(np.ascontiguousarray(mat, np.int32) if isinstance(mat, np.ndarray) else mat,
                        device=self.device, dtype=t.int32).contiguous()
        sid = C.c_int32()
        self._check(self.lib.sonar_scene_upload(self.h, _ptr(v), v.shape[0], _ptr(f), _ptr(m), f.shape[0],
                                                _stream(stream), C.byref(sid)))
        return sid.value

    def upload_mesh(self, mesh, stream=None) -> int:
        return self.upload(mesh.verts, mesh.tris, mesh.mat, stream)

    def scene_info(self, sid):
        out = (C.c_int64 * 5)()
        self._check(self.lib.sonar_scene_info(self.h, sid, out))
        return dict(zip(("n_tris", "n_pairs", "height", "max_mat", "bytes"), list(out)))

    def release(self, sid):
        self._check(self.lib.sonar_scene_release(self.h, sid))

    # ---- rendering ----
    def theta(self, alpha, gain, mu):
        t = self.torch
        return t.cat([t.tensor([alpha, gain], dtype=t.float32),
                      t.as_tensor(np.asarray(mu, np.float32))]).to(self.device)

    def render(self, sid, spec, theta, params: RenderParams = RenderParams(), seed=0, frame=0,
               hits=False, binned=False, fan=True, outputs=None, stream=None):
        """Renders one frame; returns a dict of device tensors (polar, noised,
        and optionally binned, hits [N_b*N_e, 4] int32 view of sonar_hit, fan)."""
        t = self.torch
        nr, naz = spec.n_range_bins, spec.n_az_bins
        o = outputs or {}

        def buf(name, shape, dtype=t.float32):
            return o[name] if name in o else t.empty(shape, dtype=dtype, device=self.device)

        polar = buf("polar", (nr, naz))
        noised = buf("noised", (nr, naz))
        P = buf("binned", (nr, naz)) if binned else None
        H = buf("hits", (spec.n_beams * spec.n_elev, 4), t.int32) if hits else None
        fw, fh = (spec.fan_w, spec.fan_h) if fan and spec.fan_w > 0 else (0, 0)
        F = buf("fan", (fh, fw)) if fw else None
        out = Outputs(polar.data_ptr(), noised.data_ptr(), P.data_ptr() if P is not None else None,
                      H.data_ptr() if H is not None else None, F.data_ptr() if F is not None else None,
                      fw, fh)
        sensor = to_sensor(spec)
        prm = params.c()
        n_mat = theta.shape[0] - 2
        self._check(self.lib.sonar_render(self.h, sid, C.byref(sensor), C.byref(prm), _ptr(theta), n_mat,
                                          seed, frame, C.byref(out), _stream(stream)))
        res = {"polar": polar, "noised": noised}
        if P is not None:
            res["binned"] = P
        if H is not None:
            res["hits"] = H
        if F is not None:
            res["fan"] = F
        return res

    def fan_resample(self, spec, polar, fan_w, fan_h, stream=None):
        t = self.torch
        F = t.empty((fan_h, fan_w), dtype=t.float32, device=self.device)
        sensor = to_sensor(spec)
        src = _keep(polar.contiguous(), polar, stream)
        self._check(self.lib.sonar_fan_resample(self.h, C.byref(sensor), _ptr(src), fan_w,
                                                fan_h, _ptr(F), _stream(stream)))
        return F

    def backward(self, sid, spec, theta, params: RenderParams, seed, frame, grad_polar, noised,
                 hits=None, stream=None):
        t = self.torch
        d = t.empty_like(theta)
        sensor = to_sensor(spec)
        prm = params.c()
        g = _keep(grad_polar.contiguous(), grad_polar, stream)
        self._check(self.lib.sonar_render_backward(
            self.h, sid, C.byref(sensor), C.byref(prm), _ptr(theta), theta.shape[0] - 2, seed, frame,
            _ptr(g), _ptr(noised), _ptr(hits), _ptr(d), _stream(stream)))
        return d

    def trace_stats(self, sid, spec, params: RenderParams = RenderParams(), stream=None):
        out = (C.c_int64 * 6)()
        sensor = to_sensor(spec)
        prm = params.c()
        self._check(self.lib.sonar_trace_stats(self.h, sid, C.byref(sensor), C.byref(prm), _stream(stream), out))
        return dict(zip(("visits", "tests", "nodes_touched", "tris_touched", "rays", "exact_tests"),
                        list(out)))

    def uw_image(self, J, depth, coef, out=None, stream=None):
        """Underwater image (Eq. 1) of in-air image J [..., 3] and depth [...]
        (float32 CUDA tensors); coef = beta_attn (RGB), beta_bs (RGB), B_inf
        (RGB).  Returns I [..., 3] (out may be J itself)."""
        t = self.torch
        if J.dtype != t.float32 or depth.dtype != t.float32 or J.shape[-1] != 3 or J.shape[:-1] != depth.shape:
            raise ValueError("J must be float32 [..., 3] and depth float32 [...] of the same leading shape")
        J = J.contiguous()
        depth = depth.contiguous()
        I = t.empty_like(J) if out is None else out
        k = (C.c_float * 9)(*[float(x) for x in coef])
        self._check(self.lib.sonar_uw_image(self.h, _ptr(J), _ptr(depth), depth.numel(), k, _ptr(I),
                                            _stream(stream)))
        return I

    def dvl(self, sid, poses, vel_world, params=None, seed=0, stream=None):
        """DVL measurements of poses [n, 12] (position, sensor->world rotation)
        with world velocities [n, 3] (float32 CUDA tensors).  Returns a dict of
        ranges [n, 4], vel [n, 3] (sensor frame), flags [n] (int32; bit k beam k
        valid, bit 4 velocity valid), period [n]."""
        t = self.torch
        params = params or DvlParams()
        poses = poses.contiguous()
        vel_world = vel_world.contiguous()
        n = poses.shape[0]
        if poses.shape != (n, 12) or vel_world.shape != (n, 3) or poses.dtype != t.float32:
            raise ValueError("poses must be float32 [n, 12] and vel_world [n, 3]")
        out = {"ranges": t.empty(n, 4, device=self.device), "vel": t.empty(n, 3, device=self.device),
               "flags": t.empty(n, dtype=t.int32, device=self.device), "period": t.empty(n, device=self.device)}
        self._check(self.lib.sonar_dvl(self.h, sid, _ptr(poses), _ptr(vel_world), n, C.byref(params),
                                       C.c_uint64(seed), _ptr(out["ranges"]), _ptr(out["vel"]), _ptr(out["flags"]),
                                       _ptr(out["period"]), _stream(stream)))
        return out

    def dvl_schedule(self, period, dt, stream=None):
        """Measurement steps [n_veh, n_steps] (int32 0/1) of periods [n_veh, n_steps]."""
        period = period.contiguous()
        n_veh, n_steps = period.shape
        emit = self.torch.empty(n_veh, n_steps, dtype=self.torch.int32, device=self.device)
        self._check(self.lib.sonar_dvl_schedule(self.h, _ptr(period), n_veh, n_steps, C.c_float(dt), _ptr(emit),
                                                _stream(stream)))
        return emit

    def philox(self, counters, seed, stream=None):
        """Philox4x32-10 words of counters [n, 4] (an int32 CUDA tensor holding
        the uint32 bits) under key = seed; returns [n, 4] int32 (the bits)."""
        counters = counters.contiguous()
        if counters.dtype != self.torch.int32 or counters.dim() != 2 or counters.shape[1] != 4:
            raise ValueError("counters must be an int32 tensor [n, 4]")
        out = self.torch.empty_like(counters)
        self._check(self.lib.sonar_philox(self.h, _ptr(counters), counters.shape[0], C.c_uint64(seed), _ptr(out),
                                          _stream(stream)))
        return out

    def probe_l2_read(self, buf, passes, n_blocks, stream=None):
        """Reads the CUDA tensor `buf` (16-byte aligned, size a multiple of 16
        bytes) `passes` times with L2-cached, L1-bypassing loads on n_blocks
        blocks; returns the per-block sums (float32 [n_blocks])."""
        sums = self.torch.empty(n_blocks, dtype=self.torch.float32, device=self.device)
        self._check(self.lib.sonar_probe_l2_read(self.h, _ptr(buf), buf.numel() * buf.element_size(), passes,
                                                 _ptr(sums), n_blocks, _stream(stream)))
        return sums

    def tune_get(self):
        cnt = C.c_int32()
        self._check(self.lib.sonar_tune_get(self.h, None, 0, C.byref(cnt)))
        rows = (C.c_int32 * (8 * max(1, cnt.value)))()
        self._check(self.lib.sonar_tune_get(self.h, rows, cnt.value, C.byref(cnt)))
        return np.array(list(rows), np.int32).reshape(-1, 8)[: cnt.value]

    def tune_set(self, rows):
        rows = np.ascontiguousarray(rows, np.int32).reshape(-1, 8)
        buf = (C.c_int32 * rows.size)(*rows.ravel().tolist())
        self._check(self.lib.sonar_tune_set(self.h, buf, rows.shape[0]))

    def batch(self, items):
        return Batch(self, items)


class Batch:
    """A planned batch of (scene id, SensorSpec, seed, frame) items with packed outputs."""

    def __init__(self, sonar: Sonar, items):
        self.sonar = sonar
        self.lib = sonar.lib
        t = sonar.torch
        self.items = list(items)
        n = len(self.items)
        arr = (BatchItem * n)()
        pol = hit = fan = 0
        self.layout = []
        for k, (sid, spec, seed, frame) in enumerate(self.items):
            it = arr[k]
            it.scene_id = sid
            it.fan_w, it.fan_h = int(spec.fan_w), int(spec.fan_h)
            it.sensor = to_sensor(spec)
            it.seed, it.frame = seed, frame
            it.polar_offset, it.hits_offset, it.fan_offset = pol, hit, fan
            self.layout.append((pol, hit, fan))
            pol += spec.n_range_bins * spec.n_az_bins
            hit += spec.n_beams * spec.n_elev
            fan += spec.fan_w * spec.fan_h
        self.n_polar, self.n_hits, self.n_fan = pol, hit, fan
        self._arr = arr
        h = C.c_void_p()
        sonar._check(self.lib.sonar_batch_create(sonar.h, arr, n, C.byref(h)))
        self.h = h
        dev = sonar.device
        self.polar = t.empty(pol, dtype=t.float32, device=dev)
        self.noised = t.empty(pol, dtype=t.float32, device=dev)
        self.hits = t.empty((hit, 4), dtype=t.int32, device=dev)
        self.fan = t.empty(max(fan, 1), dtype=t.float32, device=dev)
        self.binned = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.sonar_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, items, stream=None):
        n = len(items)
        arr = (BatchItem * n)()
        for k, (sid, spec, seed, frame) in enumerate(items):
            it = arr[k]
            it.scene_id = sid
            it.fan_w, it.fan_h = int(spec.fan_w), int(spec.fan_h)
            it.sensor = to_sensor(spec)
            it.seed, it.frame = seed, frame
            it.polar_offset, it.hits_offset, it.fan_offset = self.layout[k]
        self.items = list(items)
        self.sonar._check(self.lib.sonar_batch_update(self.h, arr, n, _stream(stream)))

    def outputs(self, hits=True, fan=True, binned=False):
        if binned and self.binned is None:
            self.binned = self.sonar.torch.empty_like(self.polar)
        return BatchOutputs(self.polar.data_ptr(), self.noised.data_ptr(),
                            self.binned.data_ptr() if binned else None,
                            self.hits.data_ptr() if hits else None,
                            self.fan.data_ptr() if (fan and self.n_fan) else None)

    def render(self, theta, params: RenderParams = RenderParams(), hits=True, fan=True, binned=False,
               stream=None):
        out = self.outputs(hits, fan, binned)
        prm = params.c()
        self.sonar._check(self.lib.sonar_render_batch(self.h, C.byref(prm), _ptr(theta), theta.shape[0] - 2,
                                                      C.byref(out), _stream(stream)))

    def backward(self, theta, params: RenderParams, grad_polar, hits=True, stream=None, out=None):
        t = self.sonar.torch
        d = t.empty_like(theta) if out is None else out
        prm = params.c()
        self.sonar._check(self.lib.sonar_render_batch_backward(
            self.h, C.byref(prm), _ptr(theta), theta.shape[0] - 2, _ptr(grad_polar), _ptr(self.noised),
            _ptr(self.hits) if hits else None, _ptr(d), _stream(stream)))
        return d

    def step(self, theta, params: RenderParams, grad_polar, hits=True, fan=True, stream=None, out=None):
        """Forward into the batch's buffers and the adjoint of `grad_polar` in one
        graph (sonar_render_batch_step); returns dtheta."""
        t = self.sonar.torch
        d = t.empty_like(theta) if out is None else out
        o = self.outputs(hits, fan)
        prm = params.c()
        self.sonar._check(self.lib.sonar_render_batch_step(self.h, C.byref(prm), _ptr(theta), theta.shape[0] - 2,
                                                           C.byref(o), _ptr(grad_polar), _ptr(d), _stream(stream)))
        return d

    def autotune(self, theta, params: RenderParams = RenderParams(), stream=None, hits=True):
        out = self.outputs(hits, True)
        prm = params.c()
        self.sonar._check(self.lib.sonar_autotune(self.h, C.byref(prm), _ptr(theta), theta.shape[0] - 2,
                                                  C.byref(out), _stream(stream)))

    def kernels(self):
        """Kernel launches per replay of the current forward and adjoint graphs."""
        out = (C.c_int32 * 2)()
        self.sonar._check(self.lib.sonar_batch_kernels(self.h, out))
        return {"forward": out[0], "adjoint": out[1]}

    def info(self):
        out = (C.c_int64 * 5)()
        self.sonar._check(self.lib.sonar_batch_info(self.h, out))
        return dict(zip(("units", "rays", "grid", "block", "graphs"), list(out)))

    def timings(self):
        """Phase durations (ms) of the last forward/backward graph replays."""
        ms = (C.c_float * 5)()
        self.sonar._check(self.lib.sonar_batch_timings(self.h, ms))
        return dict(zip(("trace", "bin_noise", "normalise_fan", "adjoint_rows", "adjoint_gather"), list(ms)))

    def view(self, k):
        """Per-item views (polar [nr, naz], noised, hits [rays, 4], fan [h, w]) of the packed outputs."""
        sid, spec, _, _ = self.items[k]
        p, h, f = self.layout[k]
        npol = spec.n_range_bins * spec.n_az_bins
        res = {"polar": self.polar[p:p + npol].view(spec.n_range_bins, spec.n_az_bins),
               "noised": self.noised[p:p + npol].view(spec.n_range_bins, spec.n_az_bins),
               "hits": self.hits[h:h + spec.n_beams * spec.n_elev]}
        if spec.fan_w:
            res["fan"] = self.fan[f:f + spec.fan_w * spec.fan_h].view(spec.fan_h, spec.fan_w)
        if self.binned is not None:
            res["binned"] = self.binned[p:p + npol].view(spec.n_range_bins, spec.n_az_bins)
        return res


def hits_numpy(h):
    """Device hit records [N, 4] int32 -> numpy structured array (key, tri, r, cos)."""
    return np.ascontiguousarray(h.cpu().numpy()).view(HIT_DTYPE).reshape(-1)
