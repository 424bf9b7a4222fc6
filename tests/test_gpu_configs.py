"""Full-size parity for the remaining workload configurations, each in a
batched graph-replayed launch like the bench's:

  differentiable  single-frame scene with 64 materials: the adjoint against the
                  oracle on complete azimuth columns (mode 0, so the gradient of
                  an upstream image that is zero outside those columns involves
                  only their rays), stored = recomputed, and a 32-iteration fit;
  heterogeneous   4 seabed scenes (512^2 .. 1024^2 cells) and 128 sensors of
                  three shapes in one batch: sampled rays and complete columns
                  against the oracle, and batch frames = single renders;
  large           a 4096^2-cell (33.6M-triangle) seabed, 1024 x 256 rays,
                  4000 range bins, 0.1-60 m: sampled rays and a complete column
                  against the oracle, the adjoint with recomputed hits;
  large, 1024     the large scene with 1024 materials: the adjoint on a
  materials       complete column against the oracle, zero gradient for absent
                  materials, stored = recomputed, and a short fit;
  dense rays      3000 x 460 rays into 350 x 220 bins: sampled rays and the
                  polar total against the scores.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S
from tests._parity import assert_bins_close, excluded_bins, gpu_hits, hit_parity
from tests._scene_cache import cached

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import RenderParams, Sonar, hits_numpy  # noqa: E402


@pytest.fixture(scope="module")
def son():
    s = Sonar(0)
    yield s
    s.close()


def column_rays(spec, cols):
    ids = []
    for c in cols:
        for i in range(spec.n_beams):
            if ((2 * i + 1) * spec.n_az_bins) // (2 * spec.n_beams) == c:
                ids.extend(range(i * spec.n_elev, (i + 1) * spec.n_elev))
    return np.array(ids, np.int64)


def check_frame(mesh, mu, alpha, gain, spec, view, seed, frame, cols, n_random, tv, prm=O.Params()):
    """Sampled-ray and complete-column parity of one rendered frame."""
    h = hits_numpy(view["hits"])
    rng = np.random.default_rng(seed + 17)
    ids = np.unique(np.concatenate([column_rays(spec, cols),
                                    rng.choice(spec.n_rays, n_random, replace=False)]))
    ref = O.render(mesh, mu, alpha, gain, spec, prm, seed=seed, frame=frame, ray_ids=ids, tv=tv)
    hit_parity(ref, h, ids)
    nb = spec.n_range_bins * spec.n_az_bins
    P = np.zeros(nb)
    O.lib().oracle_accumulate(len(ids), ref["key"], ref["score"], nb, P)
    In = O.noise(spec, P.reshape(spec.n_range_bins, spec.n_az_bins), seed, frame, prm)
    mask = excluded_bins(spec, {"flags": ref["flags"], "key": ref["key"]}, h[ids])
    colmask = np.ones((spec.n_range_bins, spec.n_az_bins), bool)
    colmask[:, cols] = False
    if "binned" in view:
        assert_bins_close(view["binned"].double().cpu().numpy(), P.reshape(spec.n_range_bins, -1),
                          mask | colmask, what="binned columns")
    assert_bins_close(view["noised"].double().cpu().numpy(), In, mask | colmask, what="noised columns")
    return ref, ids


# ---------------------------------------------------------------------------
# differentiable configuration (64 materials)
# ---------------------------------------------------------------------------

def test_differentiable_64_materials(son):
    mesh, mu, hfn = S.single_frame_scene(n_mat=64, mu_lo=0.05, mu_hi=0.95)
    base = S.sensor_single(hfn)
    poses = S.trajectory(base, hfn, 4, radius=20.0, seed=3)
    sid = son.upload_mesh(mesh)
    tv = O.tri_verts(mesh)
    prm0 = RenderParams(normalise=0)
    theta = son.theta(0.04, 1.5, mu)
    b = son.batch([(sid, p, k, k) for k, p in enumerate(poses)])
    b.render(theta, prm0, binned=True)
    torch.cuda.synchronize()
    spec = poses[1]
    cols = [100, 301]
    ref, ids = check_frame(mesh, mu, 0.04, 1.5, spec, b.view(1), 1, 1, cols, 0, tv, O.Params(normalise=0))
    # upstream gradient: nonzero only on the two columns of frame 1
    G = torch.zeros(b.n_polar, device=son.device)
    g1 = np.zeros((spec.n_range_bins, spec.n_az_bins), np.float32)
    g1[:, cols] = np.random.default_rng(4).normal(size=(spec.n_range_bins, 2)).astype(np.float32)
    p0 = b.layout[1][0]
    G[p0:p0 + g1.size] = torch.tensor(g1.ravel(), device=son.device)
    d_st = b.backward(theta, prm0, G, hits=True)
    d_rc = b.backward(theta, prm0, G, hits=False)
    torch.cuda.synchronize()
    assert torch.equal(d_st, d_rc)
    # oracle gradient from the oracle's own hits of those columns (rays with a
    # binned return elsewhere meet G = 0 and add nothing)
    col_only = np.isin(ref["ray_ids"], column_rays(spec, cols))
    sub = {"hits": {k: v[col_only] for k, v in ref["hits"].items() if k != "threads"},
           "key": ref["key"][col_only]}
    unused = np.zeros(g1.shape)   # mode 0: the noised image does not enter the gradient
    want = O.grad(mesh, mu, 0.04, 1.5, spec, O.Params(normalise=0), 1, 1, g1.astype(np.float64), unused, sub)
    got = d_st.double().cpu().numpy()
    scale = np.abs(want).max()
    assert np.allclose(got, want, rtol=1e-3, atol=2e-4 * scale)
    # a short fit lowers the loss
    from paper_2503_01074_gb300.autograd import sonar_render
    prm = RenderParams()
    target = son.render(sid, spec, son.theta(0.06, 1.2, mu * np.random.default_rng(5).uniform(0.8, 1.2, 64)
                                             .astype(np.float32)), prm, 1, 1)["polar"]
    th = theta.clone().requires_grad_(True)
    opt = torch.optim.Adam([th], lr=0.02)
    losses = []
    for it in range(32):
        opt.zero_grad()
        loss = torch.mean((sonar_render(th, son, sid, spec, prm, 1, 1, save_hits=it % 2 == 0) - target) ** 2)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.9 * losses[0], losses
    b.close()


# ---------------------------------------------------------------------------
# heterogeneous batch: 4 scenes, 128 sensors of three shapes
# ---------------------------------------------------------------------------

def test_heterogeneous_batch(son):
    scenes, mu, sensors = S.batched_workload()
    sids = [son.upload_mesh(m) for m, _ in scenes]
    items = [(sids[si], spec, 500 + k, k) for k, (si, spec) in enumerate(sensors)]
    theta = son.theta(0.04, 1.5, mu)
    prm = RenderParams()
    b = son.batch(items)
    b.autotune(theta, prm)
    b.render(theta, prm, binned=True)
    torch.cuda.synchronize()
    st, bits = son.check()
    assert st == 0 and bits == 0
    tvs = {}
    picked = {}
    for k, (si, spec) in enumerate(sensors):
        picked.setdefault((spec.n_beams, si % 2), k)
    assert len({spec.n_beams for _, spec in sensors}) == 3
    for key, k in sorted(picked.items())[:6]:
        si, spec = sensors[k]
        mesh = scenes[si][0]
        tv = tvs.setdefault(si, O.tri_verts(mesh))
        check_frame(mesh, mu, 0.04, 1.5, spec, b.view(k), 500 + k, k, [spec.n_az_bins // 3], 64, tv)
        single = son.render(sids[si], spec, theta, prm, 500 + k, k, hits=True, fan=True)
        v = b.view(k)
        for name in ("polar", "noised", "hits", "fan"):
            assert torch.equal(single[name], v[name]), (k, name)
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(9)).to(son.device)
    assert torch.equal(b.backward(theta, prm, G, hits=True), b.backward(theta, prm, G, hits=False))
    b.close()


# ---------------------------------------------------------------------------
# large scene: 33.6M triangles, 262,144 rays a frame, 4000 range bins
# ---------------------------------------------------------------------------

def test_large_scene(son):
    mesh, mu = cached("large", S.large_scene)
    hfn = S.height_function(400.0, 4.0, 7)
    base = S.sensor_single(hfn, n_beams=1024, n_elev=256, n_range_bins=4000, r_min=0.1, r_max=60.0,
                           fan_w=0, fan_h=0)
    poses = S.trajectory(base, hfn, 4, radius=60.0, seed=7)
    sid = son.upload_mesh(mesh)
    info = son.scene_info(sid)
    assert info["n_tris"] == mesh.n_tris > 33_000_000
    theta = son.theta(0.04, 1.5, mu)
    prm = RenderParams()
    b = son.batch([(sid, p, 900 + k, k) for k, p in enumerate(poses)])
    b.render(theta, prm, binned=True, fan=False)
    torch.cuda.synchronize()
    tv = O.tri_verts(mesh)
    check_frame(mesh, mu, 0.04, 1.5, poses[2], b.view(2), 902, 2, [640], 48, tv)
    G = torch.randn(b.n_polar, generator=torch.Generator().manual_seed(2)).to(son.device)
    d_rc = b.backward(theta, prm, G, hits=False)
    d_st = b.backward(theta, prm, G, hits=True)
    torch.cuda.synchronize()
    assert torch.equal(d_rc, d_st) and torch.isfinite(d_rc).all()
    st, bits = son.check()
    assert st == 0 and bits == 0
    b.close()
    son.release(sid)


# ---------------------------------------------------------------------------
# large scene with 1024 materials: per-material gradient at that scale
# ---------------------------------------------------------------------------

def test_large_scene_1024_materials(son):
    mesh, mu = cached("large1024", S.large_scene, n_mat=1024)
    assert mu.size == 1024 and int(mesh.mat.max()) < 1024
    hfn = S.height_function(400.0, 4.0, 7)
    base = S.sensor_single(hfn, n_beams=1024, n_elev=256, n_range_bins=4000, r_min=0.1, r_max=60.0,
                           fan_w=0, fan_h=0)
    poses = S.trajectory(base, hfn, 4, radius=60.0, seed=11)
    sid = son.upload_mesh(mesh)
    theta = son.theta(0.04, 1.5, mu)
    prm0 = RenderParams(normalise=0)
    b = son.batch([(sid, p, 40 + k, k) for k, p in enumerate(poses)])
    b.render(theta, prm0, binned=True, fan=False)
    torch.cuda.synchronize()
    spec = poses[1]
    cols = [300]
    tv = O.tri_verts(mesh)
    ref, ids = check_frame(mesh, mu, 0.04, 1.5, spec, b.view(1), 41, 1, cols, 0, tv, O.Params(normalise=0))
    # upstream gradient on that column of frame 1 only
    G = torch.zeros(b.n_polar, device=son.device)
    g1 = np.zeros((spec.n_range_bins, spec.n_az_bins), np.float32)
    g1[:, cols] = np.random.default_rng(8).normal(size=(spec.n_range_bins, len(cols))).astype(np.float32)
    p0 = b.layout[1][0]
    G[p0:p0 + g1.size] = torch.tensor(g1.ravel(), device=son.device)
    d_st = b.backward(theta, prm0, G, hits=True)
    d_rc = b.backward(theta, prm0, G, hits=False)
    torch.cuda.synchronize()
    assert torch.equal(d_st, d_rc)
    want = O.grad(mesh, mu, 0.04, 1.5, spec, O.Params(normalise=0), 41, 1, g1.astype(np.float64),
                  np.zeros(g1.shape), {"hits": {k: v for k, v in ref["hits"].items() if k != "threads"},
                                       "key": ref["key"]})
    got = d_st.double().cpu().numpy()
    scale = np.abs(want).max()
    assert np.allclose(got, want, rtol=1e-3, atol=2e-4 * scale)
    # materials no binned return of that column hits get exactly zero
    hit_mats = set(mesh.mat[ref["hits"]["tri"][(ref["key"] != 0xFFFFFFFF) & (ref["hits"]["tri"] >= 0)]].tolist())
    absent = [m for m in range(1024) if m not in hit_mats]
    assert len(absent) > 900 and np.all(got[2 + np.array(absent)] == 0.0)
    # a short fit of the 1024 reflectivities through autograd lowers the loss
    from paper_2503_01074_gb300.autograd import sonar_render
    prm = RenderParams()
    mu_t = (mu * np.random.default_rng(12).uniform(0.7, 1.3, 1024)).astype(np.float32)
    target = son.render(sid, spec, son.theta(0.04, 1.5, mu_t), prm, 41, 1)["polar"]
    mu_p = theta[2:].clone().requires_grad_(True)      # alpha and gain match the target: fit mu only
    opt = torch.optim.Adam([mu_p], lr=0.005)
    losses = []
    for it in range(16):
        opt.zero_grad()
        th = torch.cat([theta[:2], mu_p])
        loss = torch.mean((sonar_render(th, son, sid, spec, prm, 41, 1, save_hits=it % 2 == 0) - target) ** 2)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.8 * losses[0], losses
    st, bits = son.check()
    assert st == 0 and bits == 0
    b.close()
    son.release(sid)


# ---------------------------------------------------------------------------
# dense rays: 3000 x 460 rays into 350 x 220 bins
# ---------------------------------------------------------------------------

def test_dense_rays(son):
    mesh, mu, hfn = S.single_frame_scene()
    spec = S.sensor_single(hfn, n_beams=3000, n_elev=460, n_range_bins=350, n_az_bins=220,
                           fan_w=440, fan_h=248)
    sid = son.upload_mesh(mesh)
    theta = son.theta(0.04, 1.5, mu)
    prm = RenderParams()
    b = son.batch([(sid, spec, 3, 3)])
    b.render(theta, prm, binned=True)
    torch.cuda.synchronize()
    v = b.view(0)
    tv = O.tri_verts(mesh)
    check_frame(mesh, mu, 0.04, 1.5, spec, v, 3, 3, [0], 96, tv)
    h = hits_numpy(v["hits"])
    _, key, r, cs = gpu_hits(h)
    s = mu[mesh.mat[h["tri"][key >= 0]]].astype(np.float64) * cs[key >= 0] * np.exp(-0.08 * r[key >= 0]) * 1.5
    assert np.isclose(v["binned"].double().sum().item(), s.sum(), rtol=1e-5)
    single = son.render(sid, spec, theta, prm, 3, 3, fan=True)
    assert torch.equal(single["polar"], v["polar"]) and torch.equal(single["fan"], v["fan"])
    b.close()
