"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on
the same seeded inputs.  Small configurations here; the full-size
single-frame workload is in test_gpu_fullsize.py."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S
from tests._parity import assert_bins_close, excluded_bins, gpu_hits, hit_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import NO_KEY, RenderParams, Sonar, SonarError, hits_numpy  # noqa: E402


@pytest.fixture(scope="module")
def son():
    s = Sonar(0)
    yield s
    s.close()


@pytest.fixture(scope="module")
def tiny_sid(son, tiny):
    mesh, mu = tiny
    return son.upload_mesh(mesh)


def oparams(p: RenderParams) -> O.Params:
    return O.Params(p.sigma_sa, p.sigma_sm, p.sigma_phi, p.normalise, p.two_sided, p.clip_tmax)


def full_check(son, sid, mesh, mu, alpha, gain, spec, prm, seed=0, frame=0, fan=True):
    theta = son.theta(alpha, gain, mu)
    out = son.render(sid, spec, theta, prm, seed, frame, hits=True, binned=True, fan=fan)
    torch.cuda.synchronize()
    st, bits = son.check()
    assert st == 0 and bits == 0
    ref = O.render(mesh, mu, alpha, gain, spec, oparams(prm), seed=seed, frame=frame, fan=False)
    h = hits_numpy(out["hits"])
    hit_parity(ref, h)
    mask = excluded_bins(spec, ref, h)
    P = out["binned"].double().cpu().numpy()
    In = out["noised"].double().cpu().numpy()
    N = out["polar"].double().cpu().numpy()
    assert_bins_close(P, ref["P"], mask, what="binned P")
    assert_bins_close(In, ref["noised"], mask, what="noised I~")
    # normalisation: rows whose maximum sits on an excluded bin are skipped
    if prm.normalise == 1:
        rows_ok = ~mask[np.arange(mask.shape[0]), ref["argmax"]] & ~mask[np.arange(mask.shape[0]),
                                                                           In.argmax(axis=1)]
        m2 = mask | ~rows_ok[:, None]
    else:
        m2 = mask if prm.normalise == 0 else (mask if not mask.ravel()[ref["argmax"][0]] else np.ones_like(mask))
    assert_bins_close(N, ref["polar"], m2, what="normalised N")
    # the GPU's own normalisation is exact to FP32 rounding: N = I~ / rowmax(I~)
    if prm.normalise == 1:
        m = In.max(axis=1, keepdims=True)
        exp = np.where(m > 0, In / np.where(m > 0, m, 1), In)
        assert np.allclose(N, exp, rtol=2e-7, atol=0)
    if fan and spec.fan_w:
        F = out["fan"].double().cpu().numpy()
        # resampler alone: oracle fan of the GPU's own polar image
        fr, flag = O.fan_image(spec, N, spec.fan_w, spec.fan_h)
        bad = ~flag & ~np.isclose(F, fr, rtol=1e-4, atol=1e-5)
        assert not bad.any(), f"fan: {bad.sum()} pixels differ"
    return out, ref


@pytest.mark.parametrize("clip", [1, 0])
@pytest.mark.parametrize("pitch", [40.0, 28.0, 20.0])
def test_tiny_parity(son, tiny, tiny_sid, pitch, clip):
    mesh, mu = tiny
    spec = S.sensor_tiny(pitch)
    out, ref = full_check(son, tiny_sid, mesh, mu, 0.05, 1.0, spec, RenderParams(clip_tmax=clip))
    if pitch == 20.0:
        # the configuration as written: every return lies beyond r_max, so the image is noise only
        assert (ref["key"] < 0).all()
        assert float(out["binned"].abs().max()) == 0.0
        # a cast bounded at r_max finds nothing; an unbounded one records the far returns
        tri = hits_numpy(out["hits"])["tri"]
        assert (tri == 0xFFFFFFFF).all() if clip else (tri != 0xFFFFFFFF).mean() > 0.5
    elif pitch == 28.0:
        # returns on both sides of r_max: the bounded cast misses exactly the far ones
        h = hits_numpy(out["hits"])
        rmax = np.float32(spec.r_max)
        assert (ref["key"] >= 0).sum() > 200
        if clip:
            assert ((ref["hits"]["tri"] < 0) & ~ref["flags"]["limit"]).sum() > 200
            assert (h["r"][h["tri"] != 0xFFFFFFFF] < rmax).all()
        else:
            assert ((ref["hits"]["tri"] >= 0) & ~(ref["hits"]["t"] < rmax)).sum() > 200
    else:
        assert (ref["key"] >= 0).sum() > 900


@pytest.mark.parametrize("normalise", [0, 2])
def test_normalise_modes(son, tiny, tiny_sid, normalise):
    mesh, mu = tiny
    full_check(son, tiny_sid, mesh, mu, 0.05, 1.0, S.sensor_tiny(40.0), RenderParams(normalise=normalise))


def test_one_sided_and_unbounded(son, tiny, tiny_sid):
    mesh, mu = tiny
    full_check(son, tiny_sid, mesh, mu, 0.05, 1.0, S.sensor_tiny(40.0), RenderParams(two_sided=0, clip_tmax=0))


@pytest.mark.parametrize("clip", [1, 0])
@pytest.mark.parametrize("seed,n", [(1, 1), (2, 5), (3, 300), (4, 2000)])
def test_random_soups(son, seed, n, clip):
    mesh = S.random_soup(n, seed)
    spec = S.SensorSpec(np.zeros(3, np.float32), S.pose_matrix(0.1, math.radians(15)), 48, 24, 200, 48,
                        math.radians(100.0), math.radians(30.0), 0.5, 20.0, 160, 90)
    sid = son.upload_mesh(mesh)
    mu = np.array([0.2, 0.5, 0.7, 0.9], np.float32)
    full_check(son, sid, mesh, mu, 0.03, 1.7, spec, RenderParams(clip_tmax=clip))


@pytest.mark.parametrize("nb,naz", [(100, 37), (64, 200), (37, 37)])
def test_uneven_beam_and_azimuth_counts(son, tiny, tiny_sid, nb, naz):
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    spec.n_beams, spec.n_az_bins, spec.n_elev, spec.n_range_bins = nb, naz, 11, 97
    full_check(son, tiny_sid, mesh, mu, 0.05, 1.0, spec, RenderParams())


@pytest.mark.parametrize("octant", [(1, 1, 1), (-1, 1, 1), (1, -1, -1), (-1, -1, -1)])
def test_ray_octants(son, octant):
    """Every ray of the sensor in one octant of directions, including all
    components positive and all negative (the cases where a box slot left
    empty in a 4-wide node sits at +inf along every axis that the ray runs
    up), against a soup of triangles ahead of it; a larger soup so that the
    tree has empty slots at several levels."""
    sx, sy, sz = octant
    yaw = math.atan2(-sx, sy)                       # forward along (sx, sy) in the x-y plane
    pitch_down = -sz * math.radians(35.0)
    fwd = np.array([sx, sy, 0.0]) / math.sqrt(2.0)
    c = 6.0 * (fwd * math.cos(math.radians(35.0)) + np.array([0.0, 0.0, sz * math.sin(math.radians(35.0))]))
    mesh = S.random_soup(1500, 40 + sx + 2 * sy + 4 * sz, center=tuple(c), spread=3.0)
    spec = S.SensorSpec(np.zeros(3, np.float32), S.pose_matrix(yaw, pitch_down), 40, 16, 120, 40,
                        math.radians(60.0), math.radians(20.0), 0.5, 15.0, 120, 68)
    d = O.ray_dirs(spec)
    assert (np.sign(d) == np.array(octant)).all()     # the sensor's rays really lie in the octant
    sid = son.upload_mesh(mesh)
    mu = np.array([0.2, 0.5, 0.7, 0.9], np.float32)
    out, ref = full_check(son, sid, mesh, mu, 0.03, 1.7, spec, RenderParams())
    assert (ref["hits"]["tri"] >= 0).mean() > 0.3


def test_empty_scene(son):
    mesh = S.Mesh(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.int32))
    sid = son.upload_mesh(mesh)
    spec = S.sensor_tiny(40.0)
    out, ref = full_check(son, sid, mesh, np.array([0.5], np.float32), 0.05, 1.0, spec, RenderParams())
    h = hits_numpy(out["hits"])
    assert (h["tri"] == 0xFFFFFFFF).all() and (h["key"] == NO_KEY).all()


def test_accumulate_modes_and_determinism(son, tiny, tiny_sid):
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    spec.n_elev = 64      # several rays per bin
    theta = son.theta(0.05, 1.0, mu)
    a = son.render(tiny_sid, spec, theta, RenderParams(accumulate=0), binned=True)
    b = son.render(tiny_sid, spec, theta, RenderParams(accumulate=0), binned=True)
    c = son.render(tiny_sid, spec, theta, RenderParams(accumulate=1), binned=True)
    assert torch.equal(a["binned"], b["binned"]) and torch.equal(a["polar"], b["polar"])
    assert torch.allclose(a["binned"], c["binned"], rtol=1e-5, atol=1e-7)


def test_fan_resample_entry_point(son, tiny, tiny_sid):
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    theta = son.theta(0.05, 1.0, mu)
    out = son.render(tiny_sid, spec, theta, RenderParams(), fan=True)
    F = son.fan_resample(spec, out["polar"], spec.fan_w, spec.fan_h)
    assert torch.equal(F, out["fan"])
    # closed form: a field linear in range is reproduced inside the fan
    H = float(np.float32(spec.hfov))
    rmin, rmax = float(np.float32(spec.r_min)), float(np.float32(spec.r_max))
    rc = rmin + (np.arange(spec.n_range_bins) + 0.5) * (rmax - rmin) / spec.n_range_bins
    pol = torch.tensor(np.repeat(rc[:, None], spec.n_az_bins, 1), dtype=torch.float32, device=son.device)
    F = son.fan_resample(spec, pol, 300, 200).double().cpu().numpy()
    fr, flag = O.fan_image(spec, pol.double().cpu().numpy(), 300, 200)
    assert np.allclose(F[~flag], fr[~flag], rtol=1e-5, atol=1e-5)


def test_backward_matches_oracle_and_recompute(son, tiny, tiny_sid):
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    for mode in (0, 1, 2):
        prm = RenderParams(normalise=mode)
        theta = son.theta(0.05, 1.0, mu)
        out = son.render(tiny_sid, spec, theta, prm, 3, 7, hits=True)
        # upstream gradient and the noised image fed to both sides come from the oracle/seeded inputs
        ref = O.render(mesh, mu, 0.05, 1.0, spec, oparams(prm), seed=3, frame=7, fan=False)
        In32 = ref["noised"].astype(np.float32)
        G = np.random.default_rng(mode).normal(size=In32.shape).astype(np.float32)
        d_in = torch.tensor(In32, device=son.device)
        d_g = torch.tensor(G, device=son.device)
        g_st = son.backward(tiny_sid, spec, theta, prm, 3, 7, d_g, d_in, out["hits"])
        g_rc = son.backward(tiny_sid, spec, theta, prm, 3, 7, d_g, d_in, None)
        assert torch.equal(g_st, g_rc)
        want = O.grad(mesh, mu, 0.05, 1.0, spec, oparams(prm), 3, 7, G.astype(np.float64),
                      In32.astype(np.float64), ref)
        got = g_st.double().cpu().numpy()
        scale = np.abs(want).max()
        assert np.allclose(got, want, rtol=1e-3, atol=1e-4 * scale), (mode, got, want)


def test_autograd_function(son, tiny, tiny_sid):
    from paper_2503_01074_gb300.autograd import sonar_render
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    prm = RenderParams()
    theta = son.theta(0.05, 1.0, mu).requires_grad_(True)
    target = son.render(tiny_sid, spec, son.theta(0.06, 1.2, mu * np.array([1.2, 0.8], np.float32)), prm)["polar"]
    losses = []
    opt = torch.optim.Adam([theta], lr=0.01)
    for it in range(8):
        opt.zero_grad()
        N = sonar_render(theta, son, tiny_sid, spec, prm, 0, 0, save_hits=(it % 2 == 0))
        loss = torch.mean((N - target) ** 2)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < losses[0]
    assert torch.isfinite(theta.grad).all()


def test_argument_errors(son, tiny, tiny_sid):
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    theta = son.theta(0.05, 1.0, mu)
    with pytest.raises(SonarError, match="n_mat"):
        son.render(tiny_sid, spec, theta[:3], RenderParams())
    bad = S.sensor_tiny(40.0)
    bad.r_max = bad.r_min
    with pytest.raises(SonarError, match="r_min"):
        son.render(tiny_sid, bad, theta, RenderParams())
    with pytest.raises(SonarError, match="sigma_phi"):
        son.render(tiny_sid, spec, theta, RenderParams(sigma_phi=0.0))
    with pytest.raises(SonarError, match="scene"):
        son.render(12345, spec, theta, RenderParams())
    v = mesh.verts.copy()
    v[5, 1] = np.nan
    with pytest.raises(SonarError, match="finite"):
        son.upload(v, mesh.tris, mesh.mat)
    t = mesh.tris.copy()
    t[3, 2] = len(v) + 4
    with pytest.raises(SonarError, match="index"):
        son.upload(mesh.verts, t, mesh.mat)
    st, bits = son.check()
    assert st == 0 and bits == 0


def test_trace_stats(son, tiny, tiny_sid):
    spec = S.sensor_tiny(40.0)
    st = son.trace_stats(tiny_sid, spec)
    info = son.scene_info(tiny_sid)
    assert st["rays"] == spec.n_rays
    assert 0 < st["nodes_touched"] <= info["n_pairs"] and 0 < st["tris_touched"] <= info["n_tris"]
    assert st["visits"] >= st["nodes_touched"] and st["tests"] >= st["tris_touched"]


def test_philox_stream_bitwise(son):
    """The kernels' Philox4x32-10 against the oracle's (itself pinned to a
    library implementation), word for word: random counters, the extremes and
    the counters of a frame's bins (bin, frame lo, 0, frame hi)."""
    rng = np.random.default_rng(8)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    frame = (5 << 32) | 77
    ctr[2:2050, 0] = np.arange(2048, dtype=np.uint32)
    ctr[2:2050, 1] = frame & 0xFFFFFFFF
    ctr[2:2050, 2] = 0
    ctr[2:2050, 3] = frame >> 32
    d_ctr = torch.tensor(ctr.view(np.int32), device=son.device)
    for seed in (0, 1, 0x0123456789ABCDEF):
        got = son.philox(d_ctr, seed).cpu().numpy().view(np.uint32)
        want = O.philox(ctr, np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32))
        assert np.array_equal(got, want), seed
    unaligned = torch.zeros(20, dtype=torch.int32, device=son.device)[1:17].view(4, 4)
    with pytest.raises(SonarError):
        son.philox(unaligned, 0)
    st, bits = son.check()
    assert st == 0 and bits == 0


def test_l2_read_probe_reads_every_byte(son):
    # a buffer of ones with a ragged length: the block sums add up to the
    # number of floats times the passes, exactly (every partial sum is an
    # integer below 2^24)
    n = (1 << 20) + 12
    buf = torch.ones(n, dtype=torch.float32, device=son.device)
    for passes, blocks in ((1, 1), (3, 608), (2, 37)):
        sums = son.probe_l2_read(buf, passes, blocks)
        torch.cuda.synchronize()
        assert sums.double().sum().item() == n * passes
    for bad in ((buf[:3], 1, 4), (buf, 0, 4), (buf, 1, 0), (buf, 1, 70000), (buf[1:5], 1, 4)):
        with pytest.raises(SonarError):
            son.probe_l2_read(*bad)
    st, bits = son.check()
    assert st == 0 and bits == 0


def batch_items(son, tiny, tiny_sid):
    mesh, mu = tiny
    soup = S.random_soup(500, 9)
    sid2 = son.upload_mesh(soup)
    items = []
    rng = np.random.default_rng(0)
    for k in range(7):
        spec = S.sensor_tiny(float(rng.uniform(25, 50)))
        spec = spec.replace_pose((rng.uniform(-1, 1), rng.uniform(-1, 1), 0.0),
                                 S.pose_matrix(rng.uniform(-0.3, 0.3), math.radians(rng.uniform(25, 50))))
        spec.n_beams, spec.n_elev = [(128, 8), (64, 16), (96, 5)][k % 3]
        spec.n_az_bins = [128, 64, 40][k % 3]
        spec.n_range_bins = [256, 100, 333][k % 3]
        spec.fan_w, spec.fan_h = [(200, 120), (0, 0), (64, 48)][k % 3]
        items.append((tiny_sid if k % 2 == 0 else sid2, spec, 11 + k, 100 + k))
    return items


def test_batch_equals_single_renders(son, tiny, tiny_sid):
    mesh, mu = tiny
    items = batch_items(son, tiny, tiny_sid)
    theta = son.theta(0.05, 1.0, np.concatenate([mu, [0.4, 0.6]]).astype(np.float32))
    b = son.batch(items)
    prm = RenderParams()
    for rep in range(2):          # first call captures the graph, second replays it
        b.render(theta, prm)
        torch.cuda.synchronize()
        for k, (sid, spec, seed, frame) in enumerate(items):
            single = son.render(sid, spec, theta, prm, seed, frame, hits=True, fan=True)
            v = b.view(k)
            assert torch.equal(v["polar"], single["polar"]), k
            assert torch.equal(v["noised"], single["noised"]), k
            assert torch.equal(v["hits"], single["hits"]), k
            if spec.fan_w:
                assert torch.equal(v["fan"], single["fan"]), k
    # the first replay builds the exact-ray and fan tables; the second, with no
    # update in between, is the forward without the two table kernels
    assert b.info()["graphs"] == 2
    k_full, k_lean = None, b.kernels()["forward"]
    # new poses through the update path: the full forward again (same graph),
    # then the lean one
    new = [(sid, spec.replace_pose(spec.pos + np.float32(0.3), spec.rot), seed + 1, frame + 1)
           for sid, spec, seed, frame in items]
    b.update(new)
    for rep in range(2):
        b.render(theta, prm)
        torch.cuda.synchronize()
        if rep == 0:
            k_full = b.kernels()["forward"]
        for k, (sid, spec, seed, frame) in enumerate(new):
            single = son.render(sid, spec, theta, prm, seed, frame, hits=True, fan=True)
            assert torch.equal(b.view(k)["polar"], single["polar"]), k
            if spec.fan_w:   # the fan tables were kept (same geometry): still the single render's fan
                assert torch.equal(b.view(k)["fan"], single["fan"]), k
    assert b.info()["graphs"] == 2
    assert k_lean == k_full - 2           # no sin/cos table and no fan table kernel
    b.close()


def test_batch_shared_fan_tables(son, tiny, tiny_sid):
    """Frames with one fan geometry share a coordinate table (11 frames: two
    runs of users); a frame whose geometry changes leaves it, and when the
    owner's changes the others stop matching it.  Every fan stays bitwise equal
    to a single render's."""
    mesh, mu = tiny
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    base = S.sensor_tiny(40.0)
    base.fan_w, base.fan_h = 160, 96
    items = [(tiny_sid, base.replace_pose((0.2 * k, 0.1 * k, 0.0), S.pose_matrix(0.05 * k, math.radians(40.0))),
              5, k) for k in range(11)]
    b = son.batch(items)

    def check(its):
        b.render(theta, prm, fan=True)
        torch.cuda.synchronize()
        for k, (sid, spec, seed, frame) in enumerate(its):
            one = son.render(sid, spec, theta, prm, seed, frame, fan=True)
            v = b.view(k)
            assert torch.equal(one["polar"], v["polar"]), k
            assert torch.equal(one["fan"], v["fan"]), k
            assert float(v["fan"].abs().sum()) > 0.0, k

    check(items)
    moved = list(items)
    sid, spec, seed, frame = moved[3]
    s3 = spec.replace_pose(spec.pos, spec.rot)
    s3.hfov = spec.hfov * 0.9
    moved[3] = (sid, s3, seed, frame)
    b.update(moved)
    check(moved)
    sid, spec, seed, frame = moved[0]
    s0 = spec.replace_pose(spec.pos, spec.rot)
    s0.r_max = spec.r_max * 1.1
    moved[0] = (sid, s0, seed, frame)
    b.update(moved)
    check(moved)
    b.update(items)
    check(items)
    assert b.info()["graphs"] == 1
    b.close()


def test_batch_fans_after_renders_without_fans(son, tiny, tiny_sid):
    """A batch rendered without fans and then with them, no update between: the
    shared fan coordinate table is built by the first forward that writes
    fans (the replays without the table kernels wait for it), so every fan
    equals a single render's."""
    mesh, mu = tiny
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    base = S.sensor_tiny(40.0)
    base.fan_w, base.fan_h = 160, 96
    items = [(tiny_sid, base.replace_pose((0.2 * k, 0.1 * k, 0.0), S.pose_matrix(0.05 * k, math.radians(40.0))),
              5, k) for k in range(4)]
    b = son.batch(items)
    b.render(theta, prm, fan=False)
    b.render(theta, prm, fan=False)
    for rep in range(2):
        b.render(theta, prm, fan=True)
        torch.cuda.synchronize()
        for k, (sid, spec, seed, frame) in enumerate(items):
            one = son.render(sid, spec, theta, prm, seed, frame, fan=True)
            assert torch.equal(one["fan"], b.view(k)["fan"]), (rep, k)
            assert float(one["fan"].abs().sum()) > 0.0
    st, bits = son.check()
    assert st == 0 and bits == 0
    b.close()

def test_batch_backward_equals_sum_of_singles(son, tiny, tiny_sid):
    mesh, mu = tiny
    items = batch_items(son, tiny, tiny_sid)
    theta = son.theta(0.05, 1.0, np.concatenate([mu, [0.4, 0.6]]).astype(np.float32))
    prm = RenderParams()
    b = son.batch(items)
    b.render(theta, prm)
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(2)).to(son.device)
    d_b = b.backward(theta, prm, G, hits=True)
    # kernels per replay: the row terms, the gather and the final sum (stored hits)
    k = b.kernels()
    assert 4 <= k["forward"] <= 7 and k["adjoint"] == 3, k
    d_r = b.backward(theta, prm, G, hits=False)
    assert b.kernels()["adjoint"] == 5       # + the sin/cos tables and the ray cast (recomputed hits)
    torch.cuda.synchronize()
    assert torch.equal(d_b, d_r)
    total = torch.zeros_like(theta, dtype=torch.float64)
    for k, (sid, spec, seed, frame) in enumerate(items):
        v = b.view(k)
        p0 = b.layout[k][0]
        g = G[p0:p0 + spec.n_range_bins * spec.n_az_bins].view(spec.n_range_bins, spec.n_az_bins)
        total += son.backward(sid, spec, theta, prm, seed, frame, g, v["noised"], v["hits"]).double()
    assert torch.allclose(d_b.double(), total, rtol=1e-5, atol=1e-6 * float(total.abs().max()))
    b.close()


def test_autotune_keeps_results(son, tiny, tiny_sid):
    mesh, mu = tiny
    items = batch_items(son, tiny, tiny_sid)
    theta = son.theta(0.05, 1.0, np.concatenate([mu, [0.4, 0.6]]).astype(np.float32))
    prm = RenderParams()
    b = son.batch(items)
    b.autotune(theta, prm)
    rows = son.tune_get()
    assert len(rows) >= 3
    # both stages chose a measured candidate (a stage whose every candidate
    # failed would leave the derived defaults, 0)
    assert all(r[4] > 0 and r[5] > 0 for r in rows.tolist()), rows
    b.render(theta, prm)
    torch.cuda.synchronize()
    for k, (sid, spec, seed, frame) in enumerate(items):
        single = son.render(sid, spec, theta, prm, seed, frame)
        # elevation-lane mapping keeps the canonical fold order: any tile shape gives the same bits
        assert torch.equal(b.view(k)["polar"], single["polar"]), k
    # the tuner timed the adjoint on its own scratch: the tuned batch's adjoint
    # still equals the sum of the single-frame adjoints
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(3)).to(son.device)
    d_b = b.backward(theta, prm, G, hits=True)
    total = torch.zeros_like(theta, dtype=torch.float64)
    for k, (sid, spec, seed, frame) in enumerate(items):
        v = b.view(k)
        p0 = b.layout[k][0]
        g = G[p0:p0 + spec.n_range_bins * spec.n_az_bins].view(spec.n_range_bins, spec.n_az_bins)
        total += son.backward(sid, spec, theta, prm, seed, frame, g, v["noised"], v["hits"]).double()
    torch.cuda.synchronize()
    assert torch.allclose(d_b.double(), total, rtol=1e-5, atol=1e-6 * float(total.abs().max()))
    st, bits = son.check()
    assert st == 0 and bits == 0
    b.close()


def test_batch_without_hit_buffers(son, tiny, tiny_sid):
    # the batch keeps its own hit-record scratch when the caller passes none,
    # through graph capture and through the autotuner's re-planning
    mesh, mu = tiny
    items = batch_items(son, tiny, tiny_sid)
    theta = son.theta(0.05, 1.0, np.concatenate([mu, [0.4, 0.6]]).astype(np.float32))
    prm = RenderParams()
    b = son.batch(items)
    b.autotune(theta, prm, hits=False)
    b.render(theta, prm, hits=False)
    torch.cuda.synchronize()
    ref = b.polar.clone()
    b.render(theta, prm, hits=True)
    torch.cuda.synchronize()
    assert torch.equal(ref, b.polar)
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(4)).to(son.device)
    assert torch.equal(b.backward(theta, prm, G, hits=False), b.backward(theta, prm, G, hits=True))
    st, bits = son.check()
    assert st == 0 and bits == 0
    b.close()


@pytest.mark.parametrize("normalise", [0, 1, 2])
def test_batch_step_equals_separate_calls(son, tiny, tiny_sid, normalise):
    """sonar_render_batch_step runs the adjoint as a branch beside the
    normalisation and fan in one graph: its images, records and gradient
    equal a forward call followed by an adjoint call, bit for bit, through
    graph replays and with the records in the batch's own scratch."""
    mesh, mu = tiny
    items = batch_items(son, tiny, tiny_sid)
    theta = son.theta(0.05, 1.0, np.concatenate([mu, [0.4, 0.6]]).astype(np.float32))
    prm = RenderParams(normalise=normalise)
    ref = son.batch(items)
    stp = son.batch(items)
    G = torch.randn(ref.n_polar, generator=torch.Generator().manual_seed(5)).to(son.device)
    for hits in (True, False):
        ref.render(theta, prm, hits=True, fan=True)
        d_ref = ref.backward(theta, prm, G, hits=True).clone()
        for rep in range(2):          # capture, then replay
            d = stp.step(theta, prm, G, hits=hits).clone()
            torch.cuda.synchronize()
            assert torch.equal(d, d_ref), (hits, rep)
            assert torch.equal(stp.polar, ref.polar) and torch.equal(stp.noised, ref.noised)
            assert torch.equal(stp.fan, ref.fan)
            if hits:
                assert torch.equal(stp.hits, ref.hits)
    t = stp.timings()
    assert all(t[k] > 0 for k in ("trace", "bin_noise", "normalise_fan", "adjoint_gather"))
    st, bits = son.check()
    assert st == 0 and bits == 0
    ref.close()
    stp.close()


def test_batch_update_moves_items_between_scenes(son, tiny, tiny_sid):
    """An update may move items to another scene: the ray-cast block map,
    which carries each block's scene, follows, and every item again equals
    its single render bit for bit (graph replayed, not recaptured)."""
    mesh, mu = tiny
    items = batch_items(son, tiny, tiny_sid)
    sids = sorted({sid for sid, _, _, _ in items})
    assert len(sids) == 2
    theta = son.theta(0.05, 1.0, np.concatenate([mu, [0.4, 0.6]]).astype(np.float32))
    prm = RenderParams()
    b = son.batch(items)
    b.render(theta, prm)
    graphs = b.info()["graphs"]
    moved = [(sids[1] if sid == sids[0] else sids[0], spec, seed + 3, frame + 3) for sid, spec, seed, frame in items]
    b.update(moved)
    b.render(theta, prm)
    torch.cuda.synchronize()
    for k, (sid, spec, seed, frame) in enumerate(moved):
        single = son.render(sid, spec, theta, prm, seed, frame, hits=True, fan=True)
        v = b.view(k)
        assert torch.equal(v["hits"], single["hits"]), k
        assert torch.equal(v["polar"], single["polar"]), k
    assert b.info()["graphs"] == graphs
    st, bits = son.check()
    assert st == 0 and bits == 0
    b.close()


def test_single_calls_rebuild_exact_ray_tables_on_geometry_change(son, tiny, tiny_sid):
    """Single-sensor calls keep the context's exact-ray tables while the angular
    geometry is unchanged and rebuild them when it changes: alternating two
    fields of view (and a beam count) gives each frame the same bits as its
    first render, and the oracle's hits."""
    mesh, mu = tiny
    theta = son.theta(0.05, 1.0, mu)
    prm = RenderParams()
    a = S.sensor_tiny(40.0)
    b = S.sensor_tiny(40.0)
    b.hfov, b.vfov = b.hfov * 0.8, b.vfov * 1.2
    c = S.sensor_tiny(40.0)
    c.n_beams = a.n_beams + 8
    first = {}
    for rep in range(2):
        for name, spec in (("a", a), ("b", b), ("c", c)):
            o = son.render(tiny_sid, spec, theta, prm, 3, 1, hits=True, fan=False)
            torch.cuda.synchronize()
            if rep == 0:
                first[name] = (o["hits"].clone(), o["polar"].clone())
                ref = O.render(mesh, mu, 0.05, 1.0, spec, oparams(prm), seed=3, frame=1, fan=False)
                hit_parity(ref, hits_numpy(o["hits"]))
            else:
                assert torch.equal(o["hits"], first[name][0]), name
                assert torch.equal(o["polar"], first[name][1]), name
    st, bits = son.check()
    assert st == 0 and bits == 0
