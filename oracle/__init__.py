"""FP64 CPU oracle for the imaging-sonar path (OceanSim, arXiv 2503.01074).

TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
bench's CPU-baseline leg may import this module.  It shares no code with
the CUDA path and never imports it; inputs come from the seeded generators.

The arithmetic lives in sonar_oracle.c (plain FP64 definitions, one
function per step of the method, each citing the passage it follows).  This
wrapper only marshals arrays and derives the edge/tie flags used to decide
which rays a comparison may exclude:

  edge     the hit's barycentric min(u, v, 1-u-v) < 1e-6
  tie      the nearest hit on another triangle is within 1e-6 * t
  graze    |d . n_hat| < 1e-6
  binedge  the range lies within 1e-4 m of a range-bin edge (r_min, r_max included)
  limit    (a cast bounded at r_max) the nearest return lies within 1e-5 * r_max
           of the bound, on either side of it

Parity status: every step is pinned by tests/test_oracle_*.py (closed forms,
invariants, brute force, an independent Philox implementation, moment tests,
finite differences).  The fan geometry conventions, the sigma_phi default and
the noise-before-normalisation order are readings of the paper that no
external source fixes: parity unpinned with respect to the paper for those
conventions (they are pinned against their own closed forms only).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle()
        L = C.CDLL(path)
        P = np.ctypeslib.ndpointer
        f64, i64, i32, u32, u8 = (P(np.float64, flags="C"), P(np.int64, flags="C"),
                                   P(np.int32, flags="C"), P(np.uint32, flags="C"),
                                   P(np.uint8, flags="C"))
        f32 = P(np.float32, flags="C")
        L.oracle_philox_batch.argtypes = [u32, C.c_int64, u32, u32]
        L.oracle_noise_draws.argtypes = [C.c_int64, C.c_uint64, C.c_uint64, C.c_double,
                                         C.c_double, f64, f64]
        L.oracle_ray_dirs.argtypes = [f64, f64]
        L.oracle_closest_hits.argtypes = [f32, C.c_int64, f64, f64, C.c_int64, C.c_double,
                                          C.c_int, i32, f64, f64, f64, f64, f64]
        L.oracle_closest_hits.restype = C.c_int
        L.oracle_scores.argtypes = [C.c_int64, i32, f64, f64, i32, f64, C.c_double,
                                    C.c_double, C.c_int, f64]
        L.oracle_bin_keys.argtypes = [f64, C.c_int64, i64, i32, f64, i64]
        L.oracle_accumulate.argtypes = [C.c_int64, i64, f64, C.c_int64, f64]
        L.oracle_noise.argtypes = [f64, f64, C.c_uint64, C.c_uint64, C.c_double, C.c_double,
                                   C.c_double, f64]
        L.oracle_normalise.argtypes = [f64, f64, C.c_int, f64, i64, f64]
        L.oracle_fan.argtypes = [f64, f64, C.c_int, C.c_int, f64, u8]
        L.oracle_grad.argtypes = [f64, C.c_int, f64, f64, C.c_uint64, C.c_uint64, C.c_double,
                                  C.c_double, C.c_int64, i64, i32, f64, f64, i32, f64, C.c_int,
                                  C.c_double, C.c_double, C.c_int, f64]
        L.oracle_uw_image.argtypes = [f32, f32, C.c_int64, f64, f64]
        L.oracle_dvl_beams.argtypes = [f64, C.c_int64, C.c_double, f64]
        L.oracle_dvl_measure.argtypes = [C.c_int64, f64, f64, f64, C.c_double, C.c_double, C.c_double, C.c_int,
                                         C.c_double, C.c_double, C.c_double, C.c_double, C.c_uint64, f64, i32, f64]
        L.oracle_dvl_schedule.argtypes = [C.c_int64, C.c_int64, f64, C.c_double, i32]
        _LIB = L
    return _LIB


@dataclass
class Params:
    """Non-differentiable sonar configuration (mirrors the C-ABI sonar_params)."""
    sigma_sa: float = 0.3      # Rayleigh scale of the additive term, Eq. 4
    sigma_sm: float = 0.01     # std dev of the multiplicative term, Eq. 6
    sigma_phi: float = 1.0     # beam-pattern width (rad^2), Eq. 3
    normalise: int = 1         # 0 none, 1 range-row max, 2 global max
    two_sided: int = 1
    clip_tmax: int = 1         # 1: the cast ends at r_max; 0: unbounded


# relative width of the band around r_max inside which a bounded cast's
# decision is left to rounding (the range tolerance of the parity tests)
LIMIT_RTOL = 1e-5


def sensor_desc(s) -> np.ndarray:
    d = np.zeros(20, np.float64)
    d[0:3] = np.asarray(s.pos, np.float32).reshape(3)
    d[3:12] = np.asarray(s.rot, np.float32).reshape(9)
    d[12:20] = [s.n_beams, s.n_elev, s.n_range_bins, s.n_az_bins,
                np.float32(s.hfov), np.float32(s.vfov), np.float32(s.r_min), np.float32(s.r_max)]
    return d


def philox(ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(np.asarray(ctr, np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().oracle_philox_batch(ctr, ctr.shape[0], key, out)
    return out


def noise_draws(n_bins, seed, frame, sigma_sa, sigma_sm):
    w_sa = np.empty(n_bins, np.float64)
    w_sm = np.empty(n_bins, np.float64)
    lib().oracle_noise_draws(n_bins, seed, frame, sigma_sa, sigma_sm, w_sa, w_sm)
    return w_sa, w_sm


def ray_dirs(sensor) -> np.ndarray:
    out = np.empty((sensor.n_beams * sensor.n_elev, 3), np.float64)
    lib().oracle_ray_dirs(sensor_desc(sensor), out)
    return out


def tri_verts(mesh) -> np.ndarray:
    """[T, 9] FP32 vertex triples: plain gathering of the input arrays."""
    return np.ascontiguousarray(mesh.verts[mesh.tris].reshape(-1, 9), np.float32)


def closest_hits(tv, origin, dirs, t_max=np.inf, nthreads=0):
    dirs = np.ascontiguousarray(dirs, np.float64)
    n = dirs.shape[0]
    out = {k: np.empty(n, np.float64) for k in ("t", "u", "v", "t2", "dn")}
    out["tri"] = np.empty(n, np.int32)
    used = lib().oracle_closest_hits(tv, tv.shape[0], np.asarray(origin, np.float64).copy(), dirs,
                                     n, float(t_max), int(nthreads), out["tri"], out["t"],
                                     out["u"], out["v"], out["t2"], out["dn"])
    out["threads"] = used
    return out


def flags(sensor, hits, limit=None):
    """C13 flags: edge, tie, graze, binedge, limit (bool arrays per ray).
    `limit` marks rays whose nearest return lies within the range tolerance of
    the cast's r_max bound, on either side of it (None: an unbounded cast)."""
    hit = hits["tri"] >= 0
    u, v, t = hits["u"], hits["v"], hits["t"]
    edge = hit & (np.minimum(np.minimum(u, v), 1.0 - u - v) < 1e-6)
    with np.errstate(invalid="ignore"):
        tie = hit & ((hits["t2"] - t) < 1e-6 * t)
    graze = hit & (np.abs(hits["dn"]) < 1e-6)
    rmin, rmax = float(np.float32(sensor.r_min)), float(np.float32(sensor.r_max))
    dr = (rmax - rmin) / sensor.n_range_bins
    with np.errstate(invalid="ignore"):
        e = np.clip(np.round((t - rmin) / dr), 0, sensor.n_range_bins)
        near = np.abs(t - (rmin + e * dr)) < 1e-4
    binedge = hit & (t > rmin - 1e-3) & (t < rmax + 1e-3) & near
    lim = np.zeros_like(hit) if limit is None else limit
    return {"edge": edge, "tie": tie, "graze": graze, "binedge": binedge, "limit": lim}


def render(mesh, mu, alpha, gain, sensor, params: Params = Params(), seed=0, frame=0,
           ray_ids=None, nthreads=0, fan=True, tv=None):
    """Full FP64 render.  With `ray_ids` only those rays are cast and only the
    per-ray quantities (hits, scores, keys, flags) are returned."""
    L = lib()
    sd = sensor_desc(sensor)
    dirs_all = ray_dirs(sensor)
    ids = np.arange(dirs_all.shape[0], dtype=np.int64) if ray_ids is None else \
        np.ascontiguousarray(np.asarray(ray_ids, np.int64))
    dirs = np.ascontiguousarray(dirs_all[ids])
    tv = tri_verts(mesh) if tv is None else tv
    limit = None
    if params.clip_tmax:
        # the cast ends at the sonar's maximum range (Sec. III-A-2: r_max, the
        # range that scales Eq. 3).  It runs a hair past r_max so that returns
        # within the range tolerance of the bound, on either side, are flagged;
        # a nearest return at or beyond the bound then becomes a miss, which
        # is exactly the cast bounded at r_max.
        t_max = float(np.float32(sensor.r_max))
        h = closest_hits(tv, sd[0:3], dirs, t_max * (1.0 + LIMIT_RTOL), nthreads)
        limit = (h["tri"] >= 0) & (np.abs(h["t"] - t_max) <= LIMIT_RTOL * t_max)
        far = (h["tri"] >= 0) & ~(h["t"] < t_max)
        h["tri"][far] = -1
        h["t"][far] = np.inf
        h["u"][far] = 0.0
        h["v"][far] = 0.0
        h["dn"][far] = 0.0
        h["t2"][~(h["t2"] < t_max)] = np.inf
    else:
        h = closest_hits(tv, sd[0:3], dirs, np.inf, nthreads)
    n = ids.shape[0]
    mu64 = np.ascontiguousarray(mu, np.float64)
    mat = np.ascontiguousarray(mesh.mat, np.int32)
    s = np.empty(n, np.float64)
    L.oracle_scores(n, h["tri"], h["t"], h["dn"], mat, mu64, float(alpha), float(gain),
                    int(params.two_sided), s)
    key = np.empty(n, np.int64)
    L.oracle_bin_keys(sd, n, ids, h["tri"], h["t"], key)
    out = {"ray_ids": ids, "dirs": dirs, "hits": h, "score": s, "key": key,
           "flags": flags(sensor, h, limit)}
    if ray_ids is not None:
        return out
    nb = sensor.n_range_bins * sensor.n_az_bins
    P = np.empty(nb, np.float64)
    L.oracle_accumulate(n, key, s, nb, P)
    In = np.empty(nb, np.float64)
    L.oracle_noise(sd, P, seed, frame, params.sigma_sa, params.sigma_sm, params.sigma_phi, In)
    N, am, sc = normalise(sensor, In, params.normalise)
    shape = (sensor.n_range_bins, sensor.n_az_bins)
    out.update(P=P.reshape(shape), noised=In.reshape(shape), polar=N.reshape(shape),
               argmax=am, scale=sc)
    if fan and sensor.fan_w > 0:
        out["fan"], out["fan_flag"] = fan_image(sensor, N, sensor.fan_w, sensor.fan_h)
    return out


def noise(sensor, P, seed, frame, params: Params = Params()):
    In = np.empty(P.size, np.float64)
    lib().oracle_noise(sensor_desc(sensor), np.ascontiguousarray(P, np.float64).ravel(),
                       seed, frame, params.sigma_sa, params.sigma_sm, params.sigma_phi, In)
    return In.reshape(sensor.n_range_bins, sensor.n_az_bins)


def normalise(sensor, In, mode):
    In = np.ascontiguousarray(In, np.float64).ravel()
    out = np.empty_like(In)
    g = sensor.n_range_bins if mode == 1 else 1
    am = np.zeros(g, np.int64)
    sc = np.zeros(g, np.float64)
    lib().oracle_normalise(sensor_desc(sensor), In, int(mode), out, am, sc)
    return out, am, sc


def fan_image(sensor, polar, W, H):
    fan = np.empty(W * H, np.float64)
    flag = np.empty(W * H, np.uint8)
    lib().oracle_fan(sensor_desc(sensor), np.ascontiguousarray(polar, np.float64).ravel(),
                     int(W), int(H), fan, flag)
    return fan.reshape(H, W), flag.reshape(H, W).astype(bool)


def grad(mesh, mu, alpha, gain, sensor, params: Params, seed, frame, G, noised, fwd):
    """dtheta = (dL/dalpha, dL/dgain, dL/dmu[...]) for upstream G = dL/dN, the
    noised image `noised` and the per-ray results `fwd` of render()."""
    n_mat = len(mu)
    out = np.empty(n_mat + 2, np.float64)
    h = fwd["hits"]
    lib().oracle_grad(sensor_desc(sensor), int(params.normalise),
                      np.ascontiguousarray(G, np.float64).ravel(),
                      np.ascontiguousarray(noised, np.float64).ravel(), seed, frame,
                      params.sigma_sa, params.sigma_sm, fwd["key"].shape[0], fwd["key"],
                      h["tri"], h["t"], h["dn"], np.ascontiguousarray(mesh.mat, np.int32),
                      np.ascontiguousarray(mu, np.float64), n_mat, float(alpha), float(gain),
                      int(params.two_sided), out)
    return out


def loss_from_hits(mesh, mu, alpha, gain, sensor, params, seed, frame, fwd, target):
    """MSE between the normalised image rendered from fixed hits and `target`
    (used for finite differences: hits do not depend on mu, alpha, gain)."""
    L = lib()
    sd = sensor_desc(sensor)
    h = fwd["hits"]
    n = fwd["key"].shape[0]
    s = np.empty(n, np.float64)
    L.oracle_scores(n, h["tri"], h["t"], h["dn"], np.ascontiguousarray(mesh.mat, np.int32),
                    np.ascontiguousarray(mu, np.float64), float(alpha), float(gain),
                    int(params.two_sided), s)
    nb = sensor.n_range_bins * sensor.n_az_bins
    P = np.empty(nb, np.float64)
    L.oracle_accumulate(n, fwd["key"], s, nb, P)
    In = np.empty(nb, np.float64)
    L.oracle_noise(sd, P, seed, frame, params.sigma_sa, params.sigma_sm, params.sigma_phi, In)
    N, _, _ = normalise(sensor, In, params.normalise)
    d = N - np.asarray(target, np.float64).ravel()
    return float(np.mean(d * d)), In


def uw_image(J, depth, coef):
    """Eq. 1 per pixel and channel: J [..., 3] f32, depth [...] f32, coef (9,):
    beta_attn (RGB), beta_bs (RGB), B_inf (RGB).  Returns I [..., 3] f64."""
    J = np.ascontiguousarray(J, np.float32)
    d = np.ascontiguousarray(depth, np.float32)
    assert J.shape[-1] == 3 and J.shape[:-1] == d.shape
    out = np.empty(J.shape, np.float64)
    lib().oracle_uw_image(J.reshape(-1), d.reshape(-1), d.size, np.ascontiguousarray(coef, np.float64), out.reshape(-1))
    return out


@dataclass
class DvlParams:
    """DVL readings (the paper fixes none of these): beam tilt off the down axis
    (rad), valid range [r_min, r_max] (m), beams needed for a velocity, beam
    velocity noise (m/s), ping period t0 + t1 * farthest valid range (s), and
    the period after a dropout (s)."""
    tilt: float = math.radians(30.0)
    r_min: float = 0.3
    r_max: float = 50.0
    min_beams: int = 3
    sigma_b: float = 0.01
    t0: float = 0.05
    t1: float = 4.0 * 2.0 / 1500.0
    t_lost: float = 1.0


def dvl_beams(R, tilt):
    """World directions [n, 4, 3] of the four beams of poses R [n, 3, 3]."""
    R = np.ascontiguousarray(R, np.float64).reshape(-1, 9)
    out = np.empty((R.shape[0], 4, 3), np.float64)
    lib().oracle_dvl_beams(R.reshape(-1), R.shape[0], float(tilt), out.reshape(-1))
    return out


def dvl_ranges(tv, pos, R, tilt, nthreads=0):
    """Closest-hit distance of every beam [n, 4] (+inf for a miss), with the
    hit records (for the edge/tie flags)."""
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    dirs = dvl_beams(R, tilt)
    t = np.empty((pos.shape[0], 4))
    recs = []
    for p in range(pos.shape[0]):
        h = closest_hits(tv, pos[p], dirs[p], nthreads=nthreads)
        t[p] = np.where(h["tri"] >= 0, h["t"], np.inf)
        recs.append(h)
    return t, recs


def dvl_measure(R, v_world, t, params: "DvlParams", seed):
    R = np.ascontiguousarray(R, np.float64).reshape(-1, 9)
    n = R.shape[0]
    vel = np.empty((n, 3))
    flags = np.empty(n, np.int32)
    period = np.empty(n)
    lib().oracle_dvl_measure(n, R.reshape(-1), np.ascontiguousarray(v_world, np.float64).reshape(-1),
                             np.ascontiguousarray(t, np.float64).reshape(-1), params.tilt, params.r_min,
                             params.r_max, int(params.min_beams), params.sigma_b, params.t0, params.t1,
                             params.t_lost, int(seed), vel.reshape(-1), flags, period)
    return vel, flags, period


def dvl_schedule(period, dt):
    period = np.ascontiguousarray(period, np.float64)
    n_veh, n_steps = period.shape
    emit = np.empty((n_veh, n_steps), np.int32)
    lib().oracle_dvl_schedule(n_veh, n_steps, period.reshape(-1), float(dt), emit.reshape(-1))
    return emit
