"""Full-size parity on the single-frame workload (2,100,512 triangles, 512 x 64
rays, 1000 x 512 bins, 1024 x 576 fan) in the launch configuration bench.py
times: a batch of 64 poses, autotuned, graph-replayed.

One whole frame is compared with the oracle's brute force over all 32,768
rays (about half a minute of FP64 work on 16 host cores): hit triangles,
ranges and bin keys of every ray; the binned image P, the noised image I~ and
the range-normalised image N bin by bin; the fan; and the gradient with
respect to (alpha, gain, mu) in the row and whole-image normalisation modes.
Other frames are checked on
  - sampled rays, one by one (hit triangle, range, bin, incidence);
  - complete azimuth columns: every ray of the beams that fall into a column,
    so the column's binned and noised values can be compared bin by bin;
and by properties that hold at any size (the polar total equals the sum of
the binned scores; N = I~ / row max; single render = batch frame).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S
from tests._parity import assert_bins_close, excluded_bins, gpu_hits, hit_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import RenderParams, Sonar, hits_numpy  # noqa: E402

ALPHA, GAIN, B = 0.04, 1.5, 64


@pytest.fixture(scope="module")
def setup():
    mesh, mu, hfn = S.single_frame_scene()
    base = S.sensor_single(hfn)
    poses = S.trajectory(base, hfn, B, radius=20.0, seed=0)
    son = Sonar(0)
    sid = son.upload_mesh(mesh)
    theta = son.theta(ALPHA, GAIN, mu)
    prm = RenderParams()
    items = [(sid, p, k, k) for k, p in enumerate(poses)]
    batch = son.batch(items)
    batch.autotune(theta, prm)
    batch.render(theta, prm, hits=True, fan=True, binned=True)
    torch.cuda.synchronize()
    st, bits = son.check()
    assert st == 0 and bits == 0
    yield dict(mesh=mesh, mu=mu, poses=poses, son=son, sid=sid, theta=theta, prm=prm, batch=batch,
               tv=O.tri_verts(mesh))
    batch.close()
    son.close()


def column_rays(spec, cols):
    ids = []
    for c in cols:
        for i in range(spec.n_beams):
            if ((2 * i + 1) * spec.n_az_bins) // (2 * spec.n_beams) == c:
                ids.extend(range(i * spec.n_elev, (i + 1) * spec.n_elev))
    return np.array(ids, np.int64)


@pytest.mark.parametrize("frame", [0, 21, 63])
def test_sampled_rays_and_complete_columns(setup, frame):
    d = setup
    spec = d["poses"][frame]
    v = d["batch"].view(frame)
    h = hits_numpy(v["hits"])
    rng = np.random.default_rng(frame)
    cols = [0, int(rng.integers(1, spec.n_az_bins - 1)), spec.n_az_bins - 1]
    ids = np.unique(np.concatenate([column_rays(spec, cols), rng.choice(spec.n_rays, 128, replace=False)]))
    ref = O.render(d["mesh"], d["mu"], ALPHA, GAIN, spec, O.Params(), seed=frame, frame=frame,
                   ray_ids=ids, tv=d["tv"])
    hit_parity(ref, h, ids)
    assert (ref["key"] >= 0).sum() > 0.4 * len(ids)      # the test is not vacuous
    # column-complete comparison of P and I~
    nb = spec.n_range_bins * spec.n_az_bins
    P = np.zeros(nb)
    O.lib().oracle_accumulate(len(ids), ref["key"], ref["score"], nb, P)
    In = O.noise(spec, P.reshape(spec.n_range_bins, spec.n_az_bins), frame, frame, O.Params())
    sub = {"flags": ref["flags"], "key": ref["key"]}
    hsub = h[ids]
    mask = excluded_bins(spec, sub, hsub)
    colmask = np.ones((spec.n_range_bins, spec.n_az_bins), bool)
    colmask[:, cols] = False
    gP = v["binned"].double().cpu().numpy()
    gI = v["noised"].double().cpu().numpy()
    assert_bins_close(gP, P.reshape(gP.shape), mask | colmask, what="binned columns")
    assert_bins_close(gI, In, mask | colmask, what="noised columns")
    # whole-image properties
    N = v["polar"].double().cpu().numpy()
    m = gI.max(axis=1, keepdims=True)
    assert np.allclose(N, np.where(m > 0, gI / np.where(m > 0, m, 1), gI), rtol=2e-7, atol=0)
    _, key, r, cs = gpu_hits(h)
    tri = h["tri"]
    mat = d["mesh"].mat[tri[key >= 0]]
    s = d["mu"][mat].astype(np.float64) * cs[key >= 0] * np.exp(-2 * ALPHA * r[key >= 0]) * GAIN
    assert np.isclose(gP.sum(), s.sum(), rtol=1e-5)


def test_whole_frame_against_oracle(setup):
    """Frame 0 of the bench's batch against the oracle's full render."""
    d = setup
    spec = d["poses"][0]
    v = d["batch"].view(0)
    h = hits_numpy(v["hits"])
    ref = O.render(d["mesh"], d["mu"], ALPHA, GAIN, spec, O.Params(), seed=0, frame=0, tv=d["tv"])
    excl = hit_parity(ref, h)
    assert (ref["key"] >= 0).mean() > 0.5 and excl.mean() < 0.05          # not vacuous
    mask = excluded_bins(spec, ref, h)
    gP = v["binned"].double().cpu().numpy()
    gI = v["noised"].double().cpu().numpy()
    gN = v["polar"].double().cpu().numpy()
    assert_bins_close(gP, ref["P"], mask, what="binned image")
    assert_bins_close(gI, ref["noised"], mask, what="noised image")
    # range-wise normalisation (the default mode): rows whose maximum lies in
    # a compared bin
    nr, naz = spec.n_range_bins, spec.n_az_bins
    am = ref["argmax"]
    good_row = ~mask[np.arange(nr), am]
    assert good_row.mean() > 0.9
    rowmask = mask | ~good_row[:, None]
    assert_bins_close(gN, ref["polar"], rowmask, what="normalised image")
    # the fan: against the oracle's fan of the GPU's own N (the resampler
    # alone), and against the oracle's own fan wherever every bin a pixel
    # blends was compared above
    gF = v["fan"].double().cpu().numpy()
    fr, flag = O.fan_image(spec, gN, spec.fan_w, spec.fan_h)
    assert np.allclose(gF[~flag], fr[~flag], rtol=1e-4, atol=1e-5)
    probe, _ = O.fan_image(spec, np.where(rowmask, np.nan, 0.0), spec.fan_w, spec.fan_h)
    ok = ~flag & np.isfinite(probe)
    assert ok.mean() > 0.3 and (gF[ok] != 0).mean() > 0.5
    bad = ok & ~np.isclose(gF, ref["fan"], rtol=1e-4, atol=1e-5)
    assert not bad.any(), f"fan: {bad.sum()} of {ok.sum()} pixels out of tolerance"
    # gradient in modes 1 and 2 through the batch adjoint: both sides take
    # the oracle's I~ in FP32 and the same upstream gradient, which is zero on
    # every bin a flagged ray may reach and on rows (mode 1) whose maximum is
    # such a bin, so that rays the two sides may bin differently add nothing
    b = d["batch"]
    In32 = ref["noised"].astype(np.float32)
    G = np.random.default_rng(11).normal(size=(nr, naz)).astype(np.float32) * 1e-3
    G[rowmask] = 0.0
    saved = b.noised.clone()
    try:
        b.noised[:nr * naz] = torch.tensor(In32.ravel(), device=d["son"].device)
        Gd = torch.zeros(b.n_polar, device=d["son"].device)
        Gd[:nr * naz] = torch.tensor(G.ravel(), device=d["son"].device)
        for mode in (1, 2):
            if mode == 2:
                gmax = int(np.argmax(In32.ravel()))
                assert not mask.ravel()[gmax]
            prm = RenderParams(normalise=mode)
            got = b.backward(d["theta"], prm, Gd, hits=True).double().cpu().numpy()
            want = O.grad(d["mesh"], d["mu"], ALPHA, GAIN, spec, O.Params(normalise=mode), 0, 0,
                          G.astype(np.float64), In32.astype(np.float64), ref)
            scale = np.abs(want).max()
            assert scale > 0
            assert np.allclose(got, want, rtol=1e-3, atol=1e-4 * scale), (mode, got, want)
    finally:
        b.noised.copy_(saved)
        torch.cuda.synchronize()


def test_single_render_equals_batch_frame(setup):
    d = setup
    for frame in (0, 40):
        spec = d["poses"][frame]
        single = d["son"].render(d["sid"], spec, d["theta"], d["prm"], frame, frame, hits=True, fan=True)
        v = d["batch"].view(frame)
        for k in ("polar", "noised", "hits", "fan"):
            assert torch.equal(single[k], v[k]), (frame, k)


def test_fan_of_batch_frame(setup):
    d = setup
    spec = d["poses"][5]
    v = d["batch"].view(5)
    F = v["fan"].double().cpu().numpy()
    fr, flag = O.fan_image(spec, v["polar"].double().cpu().numpy(), spec.fan_w, spec.fan_h)
    bad = ~flag & ~np.isclose(F, fr, rtol=1e-4, atol=1e-5)
    assert not bad.any(), bad.sum()
    assert (F[~flag] != 0).mean() > 0.3
    # the fused normalisation + fan resamples I~ scaled by the row maxima: the
    # same bits as resampling the N it wrote
    again = d["son"].fan_resample(spec, v["polar"], spec.fan_w, spec.fan_h)
    torch.cuda.synchronize()
    assert torch.equal(again, v["fan"])


def test_adjoint_full_size_stored_equals_recomputed(setup):
    d = setup
    b = d["batch"]
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(3)).to(d["son"].device)
    g1 = b.backward(d["theta"], d["prm"], G, hits=True)
    g2 = b.backward(d["theta"], d["prm"], G, hits=False)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    assert torch.isfinite(g1).all() and float(g1.abs().sum()) > 0


def test_bounded_cast_gives_the_unbounded_images(setup):
    """The bench's batch with the cast bounded at r_max (the default) and
    unbounded: the binned, noised and normalised images, the fans and the
    gradient are the same bits; the hit records agree on every ray whose
    unbounded return lies inside r_max, and the other rays are misses in the
    bounded cast (about a tenth of this workload's rays reach the seabed
    beyond r_max)."""
    d = setup
    b = d["batch"]
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(5)).to(d["son"].device)
    out = {}
    for clip in (0, 1):
        prm = RenderParams(clip_tmax=clip)
        b.render(d["theta"], prm, hits=True, fan=True, binned=True)
        g = b.backward(d["theta"], prm, G, hits=True)
        torch.cuda.synchronize()
        out[clip] = [t.clone() for t in (b.binned, b.noised, b.polar, b.fan, g)] + [hits_numpy(b.hits)]
    for a, c in zip(out[0][:5], out[1][:5]):
        assert torch.equal(a, c)
    h0, h1 = out[0][5], out[1][5]
    rmax = np.float32(d["poses"][0].r_max)
    far = (h0["tri"] != 0xFFFFFFFF) & (h0["r"] >= rmax)
    assert 0.02 < far.mean() < 0.5
    assert (h1["tri"][far] == 0xFFFFFFFF).all()
    assert np.array_equal(h0[~far], h1[~far])
    st, bits = d["son"].check()
    assert st == 0 and bits == 0
