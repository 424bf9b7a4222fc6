"""The ray cast over the 4-wide and over the 8-wide tree.

Both trees are built per scene from the same binary hierarchy (Sec. III-A-2:
the geometry is queried by ray casting).  A ray's closest hit does not depend
on how its boxes are grouped or in which order they are tested, so every
ray-cast variant (registers capped or not, 4-wide or 8-wide tree) must give
bitwise the same hit records, and with them the same images, fans and
gradients.  Single-sensor calls walk the 8-wide tree for launches of at most
one wave, so the oracle parity tests of the single path cover it; here a
batch is pinned to each variant by a tuning row and compared with the single
path, with the other variants and with the oracle.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S

from tests._parity import hit_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import RenderParams, Sonar, SonarError, hits_numpy  # noqa: E402

CAP, WIDE = 8, 16
VARIANTS = (0, CAP, WIDE, CAP | WIDE)


@pytest.fixture(scope="module")
def son():
    s = Sonar(0)
    yield s
    s.close()


def shape(spec):
    return [spec.n_beams, spec.n_elev, spec.n_range_bins, spec.n_az_bins]


def render_variants(son, items, theta, prm, G=None):
    """Renders (and differentiates, if G is given) the batch under each
    variant; returns {variant: (hits, polar, noised, fan, dtheta)}."""
    out = {}
    for v in VARIANTS:
        son.tune_set([shape(spec) + [4, 8, 128, v] for _, spec, _, _ in items])
        b = son.batch(items)
        b.render(theta, prm, hits=True, fan=True)
        d = b.backward(theta, prm, G, hits=True).clone() if G is not None else None
        torch.cuda.synchronize()
        out[v] = (b.hits.clone(), b.polar.clone(), b.noised.clone(),
                  b.fan.clone() if b.fan is not None else None, d)
        b.close()
    return out


def soup_case(seed, n):
    mesh = S.random_soup(n, seed)
    spec = S.SensorSpec(np.zeros(3, np.float32), S.pose_matrix(0.1, math.radians(15)), 48, 24, 200, 48,
                        math.radians(100.0), math.radians(30.0), 0.5, 20.0, 160, 90)
    return mesh, spec


@pytest.mark.parametrize("seed,n", [(3, 300), (4, 2000), (5, 20000)])
def test_variants_bitwise_and_against_oracle(son, seed, n):
    mesh, spec = soup_case(seed, n)
    sid = son.upload_mesh(mesh)
    mu = np.array([0.2, 0.5, 0.7, 0.9], np.float32)
    theta = son.theta(0.03, 1.7, mu)
    prm = RenderParams()
    items = [(sid, spec.replace_pose(spec.pos + np.float32(0.2 * k), spec.rot), 7 + k, k) for k in range(3)]
    G = torch.randn(3 * spec.n_range_bins * spec.n_az_bins, generator=torch.Generator().manual_seed(seed))
    res = render_variants(son, items, theta, prm, G.to(son.device))
    ref = res[0]
    for v in VARIANTS[1:]:
        for a, b in zip(ref, res[v]):
            if a is not None:
                assert torch.equal(a, b), v
    # the single path (8-wide for this small launch) gives the same records
    nray = spec.n_rays
    for k, (s_, sp, seed_, frame) in enumerate(items):
        single = son.render(s_, sp, theta, prm, seed_, frame, hits=True, fan=True)
        assert torch.equal(single["hits"], ref[0][k * nray:(k + 1) * nray]), k
    # and the oracle's hits, frame 0 (8-wide batch)
    p = prm
    oref = O.render(mesh, mu, 0.03, 1.7, items[0][1], O.Params(p.sigma_sa, p.sigma_sm, p.sigma_phi, p.normalise,
                                                                 p.two_sided, p.clip_tmax), seed=7, frame=0, fan=False)
    hit_parity(oref, hits_numpy(res[WIDE][0][:nray]))
    st, bits = son.check()
    assert st == 0 and bits == 0


def test_variants_bitwise_full_size(son):
    """One pose of the 2.1M-triangle seabed and 32,768 rays per frame: the four
    variants' records, images and fans are identical."""
    mesh, mu, hfn = S.single_frame_scene()
    sid = son.upload_mesh(mesh)
    poses = S.trajectory(S.sensor_single(hfn), hfn, 2, radius=20.0, seed=5)
    items = [(sid, p, 3, k) for k, p in enumerate(poses)]
    theta = son.theta(0.04, 1.5, mu)
    res = render_variants(son, items, theta, RenderParams())
    for v in VARIANTS[1:]:
        for a, b in zip(res[0][:4], res[v][:4]):
            assert torch.equal(a, b), v
    h = hits_numpy(res[0][0])
    assert (h["tri"] != 0xFFFFFFFF).mean() > 0.5     # most rays hit the seabed
    st, bits = son.check()
    assert st == 0 and bits == 0


def test_stats_walk_the_tuned_tree(son):
    """The counter mode walks the tree of the shape's tuning row: the 8-wide
    walk makes fewer node visits, the same triangle tests up to the visiting
    order, and touches no more 8-wide nodes than the 4-wide tree has."""
    mesh, spec = soup_case(6, 20000)
    sid = son.upload_mesh(mesh)
    info = son.scene_info(sid)
    got = {}
    for v in (CAP, CAP | WIDE):
        son.tune_set([shape(spec) + [4, 8, 128, v]])
        got[v] = son.trace_stats(sid, spec)
    s4, s8 = got[CAP], got[CAP | WIDE]
    assert s8["visits"] < s4["visits"]
    assert 0 < s8["nodes_touched"] < s4["nodes_touched"] <= info["n_pairs"]
    assert s4["rays"] == s8["rays"] == spec.n_rays
    # the device bytes count both trees: 128 B per 4-wide node, 256 B per 8-wide one, 52 B per triangle
    assert info["bytes"] > 128 * info["n_pairs"] + 52 * info["n_tris"]


def test_tune_rows_reject_unknown_variant_bits(son):
    row = [48, 24, 200, 48, 4, 8, 128]
    son.tune_set([row + [CAP | WIDE]])
    with pytest.raises(SonarError, match="tune row"):
        son.tune_set([row + [4]])
    with pytest.raises(SonarError, match="tune row"):
        son.tune_set([row + [32]])
