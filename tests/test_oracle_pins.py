"""Pins for the FP64 oracle against things other than itself: an independent
Philox implementation, distribution moments, closed forms (flat seabed,
sphere, fan geometry), brute force through a different intersection
formulation, exact rational bin arithmetic, invariants and finite
differences.  CPU only."""
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------
# Philox4x32-10 against Triton's implementation (run in Triton's interpreter)
# --------------------------------------------------------------------------

def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(40, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [1, 0, 0, 0]
    for seed in (0, 1, 0x1234_5678_9ABC_DEF0 & 0x7FFF_FFFF_FFFF_FFFF):
        req = json.dumps({"ctr": ctr.tolist(), "seed": seed})
        env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
        res = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox.py"), req],
                             capture_output=True, text=True, env=env, timeout=300)
        assert res.returncode == 0, res.stderr[-2000:]
        ref = np.asarray(json.loads(res.stdout.strip().splitlines()[-1]), np.uint64)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
        got = O.philox(ctr.astype(np.uint32), key).astype(np.uint64)
        assert np.array_equal(got, ref), f"seed {seed}: first mismatch row {np.argwhere(got != ref)[:1]}"


def test_philox_counter_sensitivity():
    # distinct counters give distinct outputs; each output bit ~ fair over many counters
    ctr = np.zeros((4096, 4), np.uint32)
    ctr[:, 0] = np.arange(4096)
    out = O.philox(ctr, np.array([7, 9], np.uint32))
    assert len({tuple(r) for r in out}) == 4096
    bits = np.unpackbits(out.view(np.uint8)).reshape(-1, 128).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.05)


# --------------------------------------------------------------------------
# noise draws: Rayleigh(sigma) and N(0, sigma) moments and KS
# --------------------------------------------------------------------------

def test_noise_draw_distributions():
    scipy_stats = pytest.importorskip("scipy.stats")
    n = 1_000_000
    sa, sm = 0.3, 0.01
    w_sa, w_sm = O.noise_draws(n, seed=123, frame=4, sigma_sa=sa, sigma_sm=sm)
    # Rayleigh: mean sigma sqrt(pi/2), variance (4 - pi) sigma^2 / 2
    m, v = sa * math.sqrt(math.pi / 2), (4 - math.pi) * sa * sa / 2
    assert abs(w_sa.mean() - m) < 5 * math.sqrt(v / n)
    assert abs(w_sa.var() - v) < 0.01 * v
    assert (w_sa >= 0).all()
    assert abs(w_sm.mean()) < 5 * sm / math.sqrt(n)
    assert abs(w_sm.var() - sm * sm) < 0.01 * sm * sm
    assert scipy_stats.kstest(w_sa[:200000], scipy_stats.rayleigh(loc=0, scale=sa).cdf).pvalue > 1e-3
    assert scipy_stats.kstest(w_sm[:200000], scipy_stats.norm(loc=0, scale=sm).cdf).pvalue > 1e-3
    # different frame -> independent stream
    w2, _ = O.noise_draws(1000, seed=123, frame=5, sigma_sa=sa, sigma_sm=sm)
    assert abs(np.corrcoef(w_sa[:1000], w2)[0, 1]) < 0.15
    # the additive and multiplicative draws of a bin are independent, and so are
    # the four bins that share one Philox block of the additive stream
    assert abs(np.corrcoef(w_sa, w_sm)[0, 1]) < 5 / math.sqrt(n)
    q = w_sa.reshape(-1, 4)
    for i in range(4):
        for j in range(i + 1, 4):
            assert abs(np.corrcoef(q[:, i], q[:, j])[0, 1]) < 5 / math.sqrt(n / 4)
    # the additive draws are the Rayleigh inverse of the words of counters
    # (bin / 4, frame lo, 1, frame hi), bin b taking word b mod 4
    ctr = np.zeros((256, 4), np.uint32)
    ctr[:, 0] = np.arange(256)
    ctr[:, 1] = 4
    ctr[:, 2] = 1
    words = O.philox(ctr, np.array([123, 0], np.uint32)).reshape(-1).astype(np.float64)
    assert np.allclose(w_sa[:1024], sa * np.sqrt(-2.0 * np.log((words + 1.0) / 2.0 ** 32)), rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# rays
# --------------------------------------------------------------------------

def test_ray_directions_angles():
    s = S.sensor_tiny(33.0)
    s = s.replace_pose((1.0, 2.0, 3.0), S.pose_matrix(0.7, math.radians(33.0)))
    d = O.ray_dirs(s)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    R = s.rot.astype(np.float64)
    # back to the sensor frame (R is orthonormal up to its FP32 rounding)
    ds = d @ R
    ds /= np.linalg.norm(ds, axis=1, keepdims=True)
    H, V = float(np.float32(s.hfov)), float(np.float32(s.vfov))
    i = np.arange(s.n_beams).repeat(s.n_elev)
    j = np.tile(np.arange(s.n_elev), s.n_beams)
    phi = -H / 2 + (i + 0.5) * H / s.n_beams
    th = -V / 2 + (j + 0.5) * V / s.n_elev
    assert np.allclose(np.arctan2(ds[:, 0], ds[:, 1]), phi, atol=1e-6)
    assert np.allclose(np.arcsin(ds[:, 2]), th, atol=1e-6)
    # identity pose: exact to rounding
    s0 = s.replace_pose((0, 0, 0), np.eye(3))
    d0 = O.ray_dirs(s0)
    assert np.allclose(np.arctan2(d0[:, 0], d0[:, 1]), phi, atol=1e-14)
    assert np.allclose(np.arcsin(d0[:, 2]), th, atol=1e-12)


def test_azimuth_bin_integer_formula_exact():
    # floor((2i+1) N_az / (2 N_b)) equals the bin of the beam's own angle,
    # floor((phi_i + H/2) / (H / N_az)), in exact rational arithmetic
    for nb, naz in ((128, 128), (512, 512), (3000, 220), (100, 37), (7, 64)):
        m = O.render  # noqa: F841 (module import check)
        for i in range(nb):
            frac = (Fraction(2 * i + 1, 2 * nb)) * naz   # (phi + H/2)/(H/naz) with H cancelling
            assert math.floor(frac) == ((2 * i + 1) * naz) // (2 * nb)


# --------------------------------------------------------------------------
# closest hit: flat seabed closed form
# --------------------------------------------------------------------------

@pytest.mark.parametrize("clip", [1, 0])
@pytest.mark.parametrize("n_az", [64, 24])
def test_flat_seabed_closed_form(n_az, clip):
    h = 5.0
    mesh = S.quad(-h, 500.0, 0)
    p = math.radians(30.0)
    s = S.SensorSpec(np.zeros(3, np.float32), S.pose_matrix(0.0, p), 64, 16, 200, n_az,
                     math.radians(130.0), math.radians(20.0), 0.5, 30.0)
    r = O.render(mesh, np.array([0.7], np.float32), 0.05, 1.3, s, O.Params(clip_tmax=clip), fan=False)
    H, V = float(np.float32(s.hfov)), float(np.float32(s.vfov))
    i = np.arange(s.n_beams).repeat(s.n_elev)
    j = np.tile(np.arange(s.n_elev), s.n_beams)
    phi = -H / 2 + (i + 0.5) * H / s.n_beams
    th = -V / 2 + (j + 0.5) * V / s.n_elev
    R = s.rot.astype(np.float64)
    # depression of the world ray: -(z component), from the pitch rotation rows
    dsx, dsy, dsz = np.sin(phi) * np.cos(th), np.cos(phi) * np.cos(th), np.sin(th)
    dz = R[2, 0] * dsx + R[2, 1] * dsy + R[2, 2] * dsz
    nrm = np.sqrt((R[0, 0] * dsx + R[0, 1] * dsy + R[0, 2] * dsz) ** 2 +
                  (R[1, 0] * dsx + R[1, 1] * dsy + R[1, 2] * dsz) ** 2 + dz ** 2)
    sin_dep = -dz / nrm
    expect_r = h / sin_dep
    hits = r["hits"]
    rmax = float(np.float32(s.r_max))
    if clip:
        # the cast bounded at the sonar's maximum range returns exactly the rays
        # whose closed-form range is below it (some reach the plane beyond it)
        assert (expect_r >= rmax).sum() > 20 and (expect_r < rmax).sum() > 500
        assert np.array_equal(hits["tri"] >= 0, expect_r < rmax)
        assert np.array_equal(r["flags"]["limit"], np.abs(expect_r - rmax) <= O.LIMIT_RTOL * rmax)
    else:
        assert (hits["tri"] >= 0).all() and not r["flags"]["limit"].any()
    ok = ~(r["flags"]["edge"] | r["flags"]["tie"]) & (hits["tri"] >= 0)
    assert np.allclose(hits["t"][ok], expect_r[ok], rtol=1e-12)
    # incidence cosine of a horizontal plane is the sine of the depression
    assert np.allclose(np.abs(hits["dn"][ok]), sin_dep[ok], rtol=1e-12)
    # intensity s = mu |cos| e^{-2 alpha r} gain with cos = h / r
    expect_s = 0.7 * (h / expect_r) * np.exp(-2 * 0.05 * expect_r) * 1.3
    assert np.allclose(r["score"][ok], expect_s[ok], rtol=1e-10)
    # range bins from the closed-form range (rays away from bin edges)
    dr = (np.float64(np.float32(30.0)) - 0.5) / 200
    expect_br = np.floor((expect_r - 0.5) / dr)
    valid = (expect_r >= 0.5) & (expect_r < 30.0) & ~r["flags"]["binedge"]
    assert np.array_equal(r["key"][valid] // s.n_az_bins, expect_br[valid].astype(np.int64))
    # azimuth bin of each binned return from the angle of its own direction in the
    # sensor frame (for these N_b, N_az every beam centre is >= 1/16 bin from an edge)
    dsen = r["dirs"] @ R
    az = np.arctan2(dsen[:, 0], dsen[:, 1])
    expect_ba = np.floor((az + H / 2) / (H / s.n_az_bins)).astype(np.int64)
    b = r["key"] >= 0
    assert np.array_equal(r["key"][b] % s.n_az_bins, expect_ba[b])
    # invariant: the noise-free polar total equals the sum of binned scores
    assert np.isclose(r["P"].sum(), r["score"][r["key"] >= 0].sum(), rtol=1e-12)



def test_bounded_cast_changes_records_only():
    """Returns at or beyond the sonar's maximum range fall outside the polar
    grid (Sec. III-A-2), so a cast bounded at r_max differs from an unbounded
    one only in the records of those rays, which become misses: the binned,
    noised and normalised images and the fan are the same values."""
    mesh, mu = S.tiny_scene()
    spec = S.sensor_tiny(28.0)
    spec.n_beams, spec.n_elev, spec.n_range_bins, spec.n_az_bins = 64, 8, 96, 48
    spec.fan_w, spec.fan_h = 160, 120
    a = O.render(mesh, mu, 0.05, 1.0, spec, O.Params(clip_tmax=0), seed=3, frame=2)
    b = O.render(mesh, mu, 0.05, 1.0, spec, O.Params(clip_tmax=1), seed=3, frame=2)
    far = (a["hits"]["tri"] >= 0) & (a["hits"]["t"] >= np.float32(spec.r_max))
    assert far.sum() > 100 and (b["key"] >= 0).sum() > 100          # both kinds of ray occur
    assert (b["hits"]["tri"][far] == -1).all() and np.isinf(b["hits"]["t"][far]).all()
    for k in ("tri", "t", "dn"):
        assert np.array_equal(a["hits"][k][~far], b["hits"][k][~far])
    assert np.array_equal(a["key"], b["key"])
    for k in ("P", "noised", "polar", "fan"):
        assert np.array_equal(a[k], b[k]), k

def test_accumulate_per_bin_closed_form():
    """oracle_accumulate bin by bin: on a flat seabed every ray's range, score,
    range bin and azimuth bin have closed forms, so the polar image P is the
    closed-form scores summed at the closed-form keys (np.add.at).  Several
    beams share a column (N_b = 3 N_az + 1) and several elevations share range
    bins, so a transposed index, a dropped or doubled score or a misplaced
    column fails here even though the image total would still agree."""
    h = 4.0
    mesh = S.quad(-h, 500.0, 0)
    s = S.SensorSpec(np.zeros(3, np.float32), S.pose_matrix(0.3, math.radians(25.0)), 97, 24, 60, 32,
                     math.radians(120.0), math.radians(18.0), 0.5, 25.0)
    mu, alpha, gain = float(np.float32(0.45)), 0.03, 2.0     # the reflectivity table is FP32
    r = O.render(mesh, np.array([mu], np.float32), alpha, gain, s, O.Params(), fan=False)
    H, V = float(np.float32(s.hfov)), float(np.float32(s.vfov))
    i = np.arange(s.n_beams).repeat(s.n_elev)
    j = np.tile(np.arange(s.n_elev), s.n_beams)
    phi = -H / 2 + (i + 0.5) * H / s.n_beams
    th = -V / 2 + (j + 0.5) * V / s.n_elev
    R = s.rot.astype(np.float64)
    ds = np.stack([np.sin(phi) * np.cos(th), np.cos(phi) * np.cos(th), np.sin(th)], axis=1)
    dw = ds @ R.T
    sin_dep = -dw[:, 2] / np.linalg.norm(dw, axis=1)
    rr = h / sin_dep
    score = mu * (h / rr) * np.exp(-2 * alpha * rr) * gain
    rmin, rmax = 0.5, float(np.float32(25.0))
    dr = (rmax - rmin) / s.n_range_bins
    br = np.floor((rr - rmin) / dr).astype(np.int64)
    ba = ((2 * i + 1) * s.n_az_bins) // (2 * s.n_beams)
    inside = (rr >= rmin) & (rr < rmax)
    key = br * s.n_az_bins + ba
    expect = np.zeros(s.n_range_bins * s.n_az_bins)
    np.add.at(expect, key[inside], score[inside])
    # bins a return within 1e-4 m of a range-bin edge may reach are not compared
    near = np.abs(rr - (rmin + np.round((rr - rmin) / dr) * dr)) < 1e-4
    skip = np.zeros_like(expect, bool)
    for k in np.flatnonzero(near & (rr > rmin - 1e-3) & (rr < rmax + 1e-3)):
        for kk in (key[k] - s.n_az_bins, key[k], key[k] + s.n_az_bins):
            if 0 <= kk < skip.size:
                skip[kk] = True
    P = r["P"].ravel()
    assert inside.sum() > 0.5 * s.n_rays and (expect > 0).sum() > 300     # not vacuous
    assert np.allclose(P[~skip], expect[~skip], rtol=1e-11, atol=0)
    assert (np.bincount(ba, minlength=s.n_az_bins) > s.n_elev).any()      # columns hold several beams


# --------------------------------------------------------------------------
# closest hit: icosphere vs analytic sphere bounds
# --------------------------------------------------------------------------

def _sphere_t(o, d, c, rad):
    oc = c - o
    b = d @ oc
    cc = (oc @ oc) - rad * rad
    disc = b * b - cc
    t = np.where(disc >= 0, b - np.sqrt(np.maximum(disc, 0)), np.inf)
    return t


def test_icosphere_against_analytic_sphere():
    c = np.array([0.0, 4.0, -3.5])
    ico = S.icosphere(3, 1.0, c, 0)
    v = ico.verts.astype(np.float64)
    t3 = v[ico.tris]
    n = np.cross(t3[:, 1] - t3[:, 0], t3[:, 2] - t3[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = float(np.min(np.einsum("ij,ij->i", n, t3[:, 0] - c)))     # inner sphere of the facets
    r_out = float(np.max(np.linalg.norm(v - c, axis=1)))            # vertices (FP32-rounded)
    assert 0.99 < r_in < 1.0 <= r_out + 1e-6
    s = S.sensor_tiny(40.0)
    r = O.render(ico, np.array([1.0], np.float32), 0.0, 1.0, s, O.Params(), fan=False)
    d = r["dirs"]
    o = np.zeros(3)
    t_out = _sphere_t(o, d, c, r_out)
    t_in = _sphere_t(o, d, c, r_in)
    hit = r["hits"]["tri"] >= 0
    assert np.all(hit[np.isfinite(t_in)])          # rays through the inner sphere hit the mesh
    assert not np.any(hit[~np.isfinite(t_out)])    # rays missing the outer sphere miss it
    tm = r["hits"]["t"]
    sel = np.isfinite(t_in)
    assert np.all(tm[sel] >= t_out[sel] - 1e-9) and np.all(tm[sel] <= t_in[sel] + 1e-9)
    # incidence cosine within the facet angular size of the sphere's
    p = o + d[sel] * tm[sel, None]
    ns = (p - c) / np.linalg.norm(p - c, axis=1, keepdims=True)
    cos_sphere = np.abs(np.einsum("ij,ij->i", d[sel], ns))
    facet_angle = math.acos(r_in / r_out)
    assert np.all(np.abs(np.abs(r["hits"]["dn"][sel]) - cos_sphere) <= math.sin(facet_angle) + 1e-9)
    assert sel.sum() > 200


# --------------------------------------------------------------------------
# closest hit: brute force through a different formulation (linear solve)
# --------------------------------------------------------------------------

def _solve_hits(tv, o, dirs):
    """Nearest hit by solving o + t d = v0 + u e1 + v e2 with numpy.linalg.solve.
    Also returns, per ray, whether the answer is ambiguous at the 1e-6 level:
    some triangle at or before the nearest hit has a barycentric within 1e-6 of
    its edge, or two triangles are within 1e-6 t of each other."""
    nt = tv.shape[0]
    v0 = tv[:, 0:3].astype(np.float64)
    e1 = tv[:, 3:6].astype(np.float64) - v0
    e2 = tv[:, 6:9].astype(np.float64) - v0
    best_t = np.full(dirs.shape[0], np.inf)
    best = np.full(dirs.shape[0], -1)
    ambiguous = np.zeros(dirs.shape[0], bool)
    for k, d in enumerate(dirs):
        A = np.stack([e1, e2, -np.broadcast_to(d, e1.shape)], axis=2)     # [nt,3,3]
        det = np.linalg.det(A)
        ok = np.abs(det) > 1e-12 * (np.linalg.norm(e1, axis=1) * np.linalg.norm(e2, axis=1))
        x = np.full((nt, 3), np.nan)
        x[ok] = np.linalg.solve(A[ok], (o - v0[ok])[..., None])[..., 0]
        u, v, t = x[:, 0], x[:, 1], x[:, 2]
        with np.errstate(invalid="ignore"):
            good = ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
            near = ok & (t > 0) & (np.abs(np.minimum(np.minimum(u, v), 1 - u - v)) < 1e-6)
        tt = np.where(good, t, np.inf)
        if good.any():
            f = int(np.argmin(tt))
            best_t[k], best[k] = tt[f], f
            ambiguous[k] = np.sum(tt <= best_t[k] * (1 + 1e-6)) > 1
        with np.errstate(invalid="ignore"):
            ambiguous[k] |= bool(np.any(near & (t <= best_t[k] * (1 + 1e-6))))
    return best, best_t, ambiguous


@pytest.mark.parametrize("seed,n", [(1, 1), (2, 17), (3, 300), (4, 2000)])
def test_brute_force_random_soups(seed, n):
    mesh = S.random_soup(n, seed)
    s = S.SensorSpec(np.zeros(3, np.float32), S.pose_matrix(0.1, math.radians(15)), 24, 8,
                     64, 24, math.radians(100.0), math.radians(30.0), 0.5, 20.0)
    r = O.render(mesh, np.ones(4, np.float32), 0.0, 1.0, s, O.Params(), fan=False)
    tv = O.tri_verts(mesh)
    best, bt, amb = _solve_hits(tv, np.zeros(3), r["dirs"])
    ok = ~amb          # exclusions decided by the independent solver, not by the oracle
    assert ok.mean() > 0.9
    assert np.array_equal(r["hits"]["tri"][ok], best[ok])
    hit = ok & (best >= 0)
    assert np.allclose(r["hits"]["t"][hit], bt[hit], rtol=1e-9)


def test_exact_tie_goes_to_lower_index():
    # two coincident triangles: same t, lower id wins, tie flag set
    v = np.array([[-5, 5, -5], [5, 5, -5], [0, 5, 5]], np.float32)
    mesh = S.Mesh(np.concatenate([v, v]), np.array([[3, 4, 5], [0, 1, 2]], np.int32),
                  np.array([0, 1], np.int32))
    s = S.SensorSpec(np.zeros(3, np.float32), np.eye(3, dtype=np.float32), 4, 2, 16, 4,
                     math.radians(20), math.radians(10), 0.5, 10.0)
    r = O.render(mesh, np.ones(2, np.float32), 0.0, 1.0, s, O.Params(), fan=False)
    assert (r["hits"]["tri"] == 0).all()
    assert r["flags"]["tie"].all()
    assert np.allclose(r["hits"]["t"], 5.0 / r["dirs"][:, 1])


# --------------------------------------------------------------------------
# noise path closed forms
# --------------------------------------------------------------------------

def test_noise_free_closed_form():
    s = S.sensor_tiny(40.0)
    m, mu = S.tiny_scene()
    p0 = O.Params(sigma_sa=0.0, sigma_sm=0.0, normalise=0)
    r = O.render(m, mu, 0.05, 1.0, s, p0, fan=False)
    H = float(np.float32(s.hfov))
    rmin, rmax = float(np.float32(s.r_min)), float(np.float32(s.r_max))
    rc = rmin + (np.arange(s.n_range_bins) + 0.5) * (rmax - rmin) / s.n_range_bins
    expect = 0.5 * r["P"] + (rc * rc / (rmax * rmax))[:, None]
    assert np.allclose(r["noised"], expect, rtol=1e-14, atol=1e-15)
    assert np.allclose(r["polar"], r["noised"])
    # additive term alone: Rayleigh draws modulated by the beam pattern exp(-phi_c^2/sigma_phi)
    p1 = O.Params(sigma_sa=0.3, sigma_sm=0.0, sigma_phi=0.25, normalise=0)
    P0 = np.zeros((s.n_range_bins, s.n_az_bins))
    In = O.noise(s, P0, seed=3, frame=9, params=p1)
    w_sa, _ = O.noise_draws(P0.size, 3, 9, 0.3, 0.0)
    phic = -H / 2 + (np.arange(s.n_az_bins) + 0.5) * H / s.n_az_bins
    base = (rc * rc / (rmax * rmax))[:, None]
    recovered = (In / base - 1.0) / (0.5 * np.exp(-phic ** 2 / 0.25))[None, :]
    assert np.allclose(recovered.ravel(), w_sa, rtol=1e-10, atol=1e-12)


def test_multiplicative_term_scales_signal():
    # with sigma_sa = 0 the signal part is P (0.5 + w_sm) with w_sm ~ N(0, sigma_sm)
    s = S.sensor_tiny(40.0)
    rng = np.random.default_rng(0)
    P = rng.uniform(1.0, 2.0, size=(s.n_range_bins, s.n_az_bins))
    In = O.noise(s, P, seed=1, frame=2, params=O.Params(sigma_sa=0.0, sigma_sm=0.05))
    rmin, rmax = float(np.float32(s.r_min)), float(np.float32(s.r_max))
    rc = rmin + (np.arange(s.n_range_bins) + 0.5) * (rmax - rmin) / s.n_range_bins
    w = (In - (rc * rc / rmax ** 2)[:, None]) / P - 0.5
    assert abs(w.mean()) < 5 * 0.05 / math.sqrt(w.size)
    assert abs(w.std() - 0.05) < 0.003


# --------------------------------------------------------------------------
# normalisation
# --------------------------------------------------------------------------

def test_normalisation_modes():
    s = S.sensor_tiny(40.0)
    rng = np.random.default_rng(1)
    In = rng.uniform(0.1, 3.0, size=(s.n_range_bins, s.n_az_bins))
    In[3, 5] = In[3, 9] = In[3].max() + 1.0          # tie for the maximum
    In[7] = -np.abs(In[7])                           # row with max <= 0 stays unchanged
    N, am, sc = O.normalise(s, In, 1)
    N = N.reshape(In.shape)
    rows = np.arange(In.shape[0]) != 7
    assert np.allclose(N[rows].max(axis=1), 1.0)
    assert np.allclose(sc[rows], In[rows].max(axis=1))
    assert am[3] == 5
    assert np.array_equal(N[7], In[7])
    N2, am2, sc2 = O.normalise(s, In, 2)
    assert np.isclose(N2.max(), 1.0) and sc2[0] == In.max() and am2[0] == np.argmax(In)


# --------------------------------------------------------------------------
# fan geometry closed forms
# --------------------------------------------------------------------------

def _fan_xy(s, W, Hpx):
    H, rmax = float(np.float32(s.hfov)), float(np.float32(s.r_max))
    scale = min(W / (2 * rmax * math.sin(H / 2)), Hpx / rmax)
    u = np.arange(W) + 0.5 - W / 2
    v = Hpx - np.arange(Hpx) - 0.5
    X, Y = np.meshgrid(u / scale, v / scale)
    return X, Y


@pytest.mark.parametrize("hfov", [60.0, 130.0])
def test_fan_reproduces_linear_fields(hfov):
    s = S.sensor_tiny(40.0)
    s.hfov = math.radians(hfov)
    W, Hpx = 400, 300
    H = float(np.float32(s.hfov))
    rmin, rmax = float(np.float32(s.r_min)), float(np.float32(s.r_max))
    dr, da = (rmax - rmin) / s.n_range_bins, H / s.n_az_bins
    rc = rmin + (np.arange(s.n_range_bins) + 0.5) * dr
    pc = -H / 2 + (np.arange(s.n_az_bins) + 0.5) * da
    X, Y = _fan_xy(s, W, Hpx)
    R = np.hypot(X, Y)
    PH = np.arctan2(X, Y)
    inside = (R >= rmin) & (R <= rmax) & (np.abs(PH) <= H / 2)
    interior = (R >= rc[0]) & (R <= rc[-1]) & (np.abs(PH) <= pc[-1])
    # constant -> constant inside the fan, 0 outside
    f, flag = O.fan_image(s, np.full((s.n_range_bins, s.n_az_bins), 2.5), W, Hpx)
    assert np.allclose(f[inside & ~flag], 2.5) and np.all(f[~inside & ~flag] == 0)
    # bilinear interpolation reproduces fields linear in r or in phi exactly
    f, _ = O.fan_image(s, np.repeat(rc[:, None], s.n_az_bins, 1), W, Hpx)
    assert np.allclose(f[interior], R[interior], rtol=1e-12)
    f, _ = O.fan_image(s, np.repeat(pc[None, :], s.n_range_bins, 0), W, Hpx)
    assert np.allclose(f[interior], PH[interior], atol=1e-12)
    # the fan fills the image: full height along phi = 0, or full width at r_max
    assert inside[:, W // 2].sum() >= Hpx * (1 - rmin / rmax) - 2 or \
        (inside[:, 0].any() and inside[:, -1].any())


# --------------------------------------------------------------------------
# gradient vs FP64 central finite differences
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1, 2])
def test_gradient_matches_finite_differences(mode):
    m, mu = S.tiny_scene()
    s = S.sensor_tiny(40.0)
    prm = O.Params(normalise=mode)
    alpha, gain = 0.05, 1.0
    fwd = O.render(m, mu, alpha, gain, s, prm, seed=0, frame=0, fan=False)
    tgt = O.render(m, mu * np.array([1.2, 0.85], np.float32), 0.06, 1.2, s, prm, seed=0, frame=0,
                   fan=False)["polar"]
    _, In = O.loss_from_hits(m, mu, alpha, gain, s, prm, 0, 0, fwd, tgt)
    n = In.size
    N, _, _ = O.normalise(s, In, mode)
    G = 2.0 * (N - tgt.ravel()) / n
    g = O.grad(m, mu, alpha, gain, s, prm, 0, 0, G, In, fwd)
    theta = np.array([alpha, gain] + list(mu.astype(np.float64)))

    def central(h):
        fd = np.zeros_like(theta)
        for k in range(theta.size):
            tp, tm = theta.copy(), theta.copy()
            tp[k] += h
            tm[k] -= h
            lp, _ = O.loss_from_hits(m, tp[2:], tp[0], tp[1], s, prm, 0, 0, fwd, tgt)
            lm, _ = O.loss_from_hits(m, tm[2:], tm[0], tm[1], s, prm, 0, 0, fwd, tgt)
            fd[k] = (lp - lm) / (2 * h)
        return fd

    fd1, fd2 = central(1e-4), central(5e-5)
    assert np.all(np.abs(g) > 0)
    # central differences with step 1e-4 carry an O(h^2) truncation error; the
    # exp(-2 alpha r) factor makes it largest for alpha (~1e-5 relative)
    assert np.allclose(g, fd1, rtol=1e-4, atol=1e-12), (g, fd1)
    # Richardson extrapolation removes the h^2 term: the analytic gradient must
    # then agree to near the rounding level of the differences
    rich = (4.0 * fd2 - fd1) / 3.0
    assert np.allclose(g, rich, rtol=2e-7, atol=1e-13), (g, rich)


def test_ray_subset_matches_full_render(tiny):
    m, mu = tiny
    s = S.sensor_tiny(40.0)
    full = O.render(m, mu, 0.05, 1.0, s, O.Params(), fan=False)
    ids = np.array([0, 5, 77, 500, 1023])
    sub = O.render(m, mu, 0.05, 1.0, s, O.Params(), ray_ids=ids)
    for k in ("tri", "t", "dn"):
        assert np.array_equal(sub["hits"][k], full["hits"][k][ids])
    assert np.array_equal(sub["key"], full["key"][ids])
