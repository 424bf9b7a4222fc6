"""GPU parity of the DVL (Sec. III-A-3) through the C ABI against the FP64
oracle: beam ranges, validity flags, least-squares velocities, ping periods
and the measurement schedule.

Tolerances: ranges within 1e-5 relative (the ray-cast bar), excluding beams
whose oracle hit is an edge, tie or grazing hit and beams within 1e-4 m of
the valid window's ends (a rounding may flip those); velocities within
2e-5 (|v| + 1) (FP32 noise draws and a Cramer solve of a system with
condition number 6); periods within 1e-5 relative; schedules compared on
vehicles whose periods are all at least 1e-3 steps away from a whole number
of steps (elsewhere FP32 and FP64 may round the step count apart)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import DvlParams, Sonar, SonarError  # noqa: E402

OP = O.DvlParams()   # the same defaults on both sides


@pytest.fixture(scope="module")
def son():
    s = Sonar(0)
    yield s
    s.close()


def ambiguous_beams(recs, t, P):
    """[n, 4] bool: beams whose oracle hit is an edge, tie or grazing hit, or
    whose range lies within 1e-4 m of the valid window's ends."""
    amb = np.zeros(t.shape, bool)
    for p, h in enumerate(recs):
        hit = h["tri"] >= 0
        bary = np.minimum(np.minimum(h["u"], h["v"]), 1.0 - h["u"] - h["v"])
        with np.errstate(invalid="ignore"):      # a miss has t = t2 = inf
            tie = h["t2"] - h["t"] < 1e-6 * h["t"]
        amb[p] = hit & ((bary < 1e-6) | tie | (np.abs(h["dn"]) < 1e-6))
    amb |= (np.abs(t - P.r_min) < 1e-4) | (np.abs(t - P.r_max) < 1e-4)
    return amb


def compare(got, tv, poses, vels, seed, P=OP):
    n = poses.shape[0]
    R = poses[:, 3:].astype(np.float64).reshape(n, 3, 3)
    t, recs = O.dvl_ranges(tv, poses[:, :3].astype(np.float64), R, P.tilt)
    vel, flags, period = O.dvl_measure(R, vels.astype(np.float64), t, P, seed)
    amb = ambiguous_beams(recs, t, P)
    gr = got["ranges"].double().cpu().numpy()
    ok = ~amb
    both_inf = np.isinf(gr) & np.isinf(t)
    fin = ok & ~both_inf
    assert np.all(np.isfinite(gr[fin]) == np.isfinite(t[fin]))
    f2 = fin & np.isfinite(t)
    assert np.allclose(gr[f2], t[f2], rtol=1e-5, atol=0)
    clean = ~amb.any(axis=1)
    gf = got["flags"].cpu().numpy()
    assert np.array_equal(gf[clean], flags[clean])
    gv = got["vel"].double().cpu().numpy()
    same = clean & (gf == flags)
    scale = np.abs(vels).max() + 1.0
    assert np.allclose(gv[same], vel[same], rtol=0, atol=2e-5 * scale)
    gp = got["period"].double().cpu().numpy()
    assert np.allclose(gp[same], period[same], rtol=1e-5)
    return period, flags, clean, t


def test_flat_seabed_closed_form(son):
    h = 7.0
    mesh = S.quad(-h, 60.0)
    sid = son.upload_mesh(mesh)
    n = 64
    rng = np.random.default_rng(2)
    poses = np.zeros((n, 12), np.float32)
    poses[:, :2] = rng.uniform(-5, 5, (n, 2))
    poses[:, 3:] = np.eye(3, dtype=np.float32).ravel()
    v = rng.normal(size=(n, 3)).astype(np.float32)
    out = son.dvl(sid, torch.tensor(poses, device=son.device), torch.tensor(v, device=son.device),
                  DvlParams(sigma_b=0.0), seed=1)
    torch.cuda.synchronize()
    assert np.allclose(out["ranges"].cpu().numpy(), h / math.cos(math.radians(30.0)), rtol=2e-6)
    assert np.all(out["flags"].cpu().numpy() == 31)
    assert np.allclose(out["vel"].cpu().numpy(), v, atol=2e-6)          # level: sensor frame = world frame
    son.release(sid)


def test_matches_oracle_on_a_small_seabed(son):
    """Full parity on a 128^2-cell seabed with piles and boxes: 48 vehicles of
    64 steps, altitudes 0.2-70 m (dropouts included)."""
    mesh, mu, hfn = S.single_frame_scene(n_cells=128, n_piles=12, n_boxes=6)
    sid = son.upload_mesh(mesh)
    tv = O.tri_verts(mesh)
    poses, vels = S.dvl_trajectories(hfn, 48, 64, 0.05, seed=5, alt_lo=0.2, alt_hi=70.0)
    P = poses.reshape(-1, 12)
    V = vels.reshape(-1, 3)
    out = son.dvl(sid, torch.tensor(P, device=son.device), torch.tensor(V, device=son.device), DvlParams(), seed=77)
    torch.cuda.synchronize()
    period, flags, clean, t = compare(out, tv, P, V, 77)
    fl = out["flags"].cpu().numpy()
    assert (fl & 16).any() and (~fl & 16).any()          # valid and dropped measurements both occur
    assert ((fl & 15) == 15).any() and (np.isin(fl & 15, [7, 11, 13, 14])).any()
    # the schedule, on vehicles where no period sits near a whole number of steps
    dt = 0.05
    gper = out["period"].view(48, 64)
    emit = son.dvl_schedule(gper, dt).cpu().numpy()
    want = O.dvl_schedule(period.reshape(48, 64), dt)
    q = period.reshape(48, 64) / dt
    far = (np.abs(q - np.round(q)) > 1e-3).all(axis=1) & clean.reshape(48, 64).all(axis=1)
    assert far.sum() > 10
    assert np.array_equal(emit[far], want[far])
    st, bits = son.check()
    assert st == 0 and bits == 0
    son.release(sid)


def test_sampled_parity_on_the_bench_scene(son):
    """The bench's scene (2.1M triangles): 64 poses sampled from its vehicles."""
    mesh, mu, hfn = S.single_frame_scene()
    sid = son.upload_mesh(mesh)
    tv = O.tri_verts(mesh)
    poses, vels = S.dvl_trajectories(hfn, 512, 32, 0.05, seed=3)
    P = poses.reshape(-1, 12)
    V = vels.reshape(-1, 3)
    out = son.dvl(sid, torch.tensor(P, device=son.device), torch.tensor(V, device=son.device), DvlParams(), seed=9)
    torch.cuda.synchronize()
    idx = np.random.default_rng(4).choice(P.shape[0], 64, replace=False)
    sub = {k: v[torch.tensor(idx, device=son.device)] for k, v in out.items()}
    # the sampled poses keep their global indices (they index the noise stream):
    # compare through an oracle call on all of them, then select
    n = P.shape[0]
    R = P[idx, 3:].astype(np.float64).reshape(-1, 3, 3)
    t, recs = O.dvl_ranges(tv, P[idx, :3].astype(np.float64), R, OP.tilt)
    full_t = np.full((n, 4), np.inf)
    full_t[idx] = t
    vel, flags, period = O.dvl_measure(P[:, 3:].astype(np.float64).reshape(n, 3, 3), V.astype(np.float64),
                                       full_t, OP, 9)
    amb = ambiguous_beams(recs, t, OP)
    clean = ~amb.any(axis=1)
    gr = sub["ranges"].double().cpu().numpy()
    fin = ~amb & np.isfinite(t)
    assert np.allclose(gr[fin], t[fin], rtol=1e-5)
    gf = sub["flags"].cpu().numpy()
    assert np.array_equal(gf[clean], flags[idx][clean])
    same = clean & (gf == flags[idx])
    assert np.allclose(sub["vel"].double().cpu().numpy()[same], vel[idx][same], atol=2e-5 * (np.abs(V).max() + 1))
    son.release(sid)


def test_schedule_of_given_periods(son):
    per = torch.tensor([[0.105] * 30, [0.01] * 30, [0.5] * 30], device=son.device)
    emit = son.dvl_schedule(per, 0.05).cpu().numpy()
    assert list(np.nonzero(emit[0])[0]) == list(range(0, 30, 3))
    assert emit[1].all()
    assert list(np.nonzero(emit[2])[0]) == [0, 10, 20]


def test_argument_errors(son, tiny):
    sid = son.upload_mesh(tiny[0])
    p = torch.zeros(4, 12, device=son.device)
    v = torch.zeros(4, 3, device=son.device)
    for bad in (DvlParams(tilt=0.0), DvlParams(min_beams=2), DvlParams(r_min=5.0, r_max=4.0),
                DvlParams(sigma_b=-1.0), DvlParams(t_lost=0.0)):
        with pytest.raises(SonarError):
            son.dvl(sid, p, v, bad)
    with pytest.raises(SonarError):
        son.dvl_schedule(torch.zeros(2, 3, device=son.device), 0.0)
    son.release(sid)
