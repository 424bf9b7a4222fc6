"""GPU parity of the underwater image formation (Eq. 1) through the C ABI,
element by element against the FP64 oracle.

Tolerance: the kernel rounds beta * d to FP32 and evaluates exp with a few
ulp of error, so each transmission factor is within about 2 eps of the exact
one (e^-x (x + 2) eps <= 2 eps); with the FMA and the products, |I - I_ref| <=
about 4 eps max(J, B_inf), eps = 2^-24.  Tested at 1e-6 absolute (values <= 1)
plus 1e-6 relative."""
import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2503_01074_gb300.sonar import RenderParams, Sonar, SonarError, hits_numpy  # noqa: E402

RTOL, ATOL = 1e-6, 1e-6


@pytest.fixture(scope="module")
def son():
    s = Sonar(0)
    yield s
    s.close()


@pytest.fixture(scope="module")
def tiny_sid(son, tiny):
    return son.upload_mesh(tiny[0])


def close(got, want):
    got = got.double().cpu().numpy()
    assert got.shape == want.shape
    assert np.allclose(got, want, rtol=RTOL, atol=ATOL), np.abs(got - want).max()


def coef_sets(rng):
    yield np.concatenate([rng.uniform(0.02, 0.8, 6), rng.uniform(0.0, 1.0, 3)])
    yield np.array([0.0, 0.3, 0.0, 0.1, 0.0, 0.0, 0.2, 0.5, 0.9])      # zero coefficients
    yield np.array([0.4, 0.4, 0.4, 0.4, 0.4, 0.4, 0.3, 0.3, 0.3])       # attn = bs


@pytest.mark.parametrize("n", [1, 3, 4, 1001, 65536 + 7])
def test_matches_oracle_ragged_and_special_depths(son, n):
    rng = np.random.default_rng(n)
    J = rng.random((n, 3), dtype=np.float32)
    d = rng.uniform(0.0, 60.0, n).astype(np.float32)
    d[:: 7] = 0.0
    d[3:: 11] = np.inf
    d[5:: 13] = 1e4
    Jg = torch.tensor(J, device=son.device)
    dg = torch.tensor(d, device=son.device)
    for coef in coef_sets(rng):
        close(son.uw_image(Jg, dg, coef), O.uw_image(J, d, coef))


def test_unaligned_views_and_in_place(son):
    rng = np.random.default_rng(3)
    n = 4099
    J = rng.random((n + 1, 3), dtype=np.float32)
    d = rng.uniform(0.0, 30.0, n + 1).astype(np.float32)
    coef = np.concatenate([rng.uniform(0.02, 0.5, 6), rng.uniform(0, 1, 3)])
    Jg = torch.tensor(J, device=son.device)
    dg = torch.tensor(d, device=son.device)
    # one pixel in: 12- and 4-byte offsets take the scalar path
    close(son.uw_image(Jg[1:], dg[1:], coef), O.uw_image(J[1:], d[1:], coef))
    # in place on an aligned buffer (the vectorised path)
    want = O.uw_image(J[:n - 3], d[:n - 3], coef)
    buf = Jg[: n - 3].clone()
    out = son.uw_image(buf, dg[: n - 3], coef, out=buf)
    assert out.data_ptr() == buf.data_ptr()
    close(buf, want)


def test_depth_from_the_ray_caster(son, tiny, tiny_sid):
    """J: a seeded texture; d: the ranges our own ray caster returns for a
    128 x 8-ray sensor looking at the tiny scene (misses give +inf)."""
    mesh, mu = tiny
    spec = S.sensor_tiny(40.0)
    out = son.render(tiny_sid, spec, son.theta(0.05, 1.0, mu), RenderParams(), 0, 0, hits=True)
    h = hits_numpy(out["hits"])
    depth = np.where(h["tri"] != 0xFFFFFFFF, h["r"], np.inf).astype(np.float32)
    depth = depth.reshape(spec.n_beams, spec.n_elev).T.copy()
    assert np.isfinite(depth).sum() > depth.size // 2
    J = S.camera_rgb(spec.n_elev, spec.n_beams, 5)
    coef = [0.35, 0.12, 0.08, 0.30, 0.15, 0.10, 0.05, 0.25, 0.35]
    I = son.uw_image(torch.tensor(J, device=son.device), torch.tensor(depth, device=son.device), coef)
    close(I, O.uw_image(J, depth, coef))


def test_full_size_batch(son):
    """The bench's launch: 64 frames of 1920 x 1080 in one call; sampled
    pixels against the oracle, a frame whole."""
    H, W, F = 1080, 1920, 64
    J1 = S.camera_rgb(H, W, 9)
    d1 = S.camera_seabed_depth(H, W)
    Jg = torch.tensor(J1, device=son.device).expand(F, H, W, 3).contiguous()
    scale = torch.linspace(0.5, 1.5, F, device=son.device).view(F, 1, 1)
    dg = (torch.tensor(d1, device=son.device) * scale).contiguous()
    coef = [0.35, 0.12, 0.08, 0.30, 0.15, 0.10, 0.05, 0.25, 0.35]
    I = son.uw_image(Jg, dg, coef)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    idx = torch.tensor(rng.integers(0, F * H * W, 200_000), device=son.device)
    Jf = Jg.view(-1, 3)[idx].cpu().numpy()
    df = dg.view(-1)[idx].cpu().numpy()
    close(I.view(-1, 3)[idx], O.uw_image(Jf, df, coef))
    close(I[F - 1], O.uw_image(Jg[F - 1].cpu().numpy(), dg[F - 1].cpu().numpy(), coef))


def test_argument_errors(son):
    J = torch.zeros(4, 3, device=son.device)
    d = torch.zeros(4, device=son.device)
    good = [0.1] * 9
    for bad in ([-0.1] + [0.1] * 8, [0.1] * 3 + [float("nan")] + [0.1] * 5, [0.1] * 8 + [float("inf")]):
        with pytest.raises(SonarError):
            son.uw_image(J, d, bad)
    # an empty image is a no-op
    son.uw_image(torch.zeros(0, 3, device=son.device), torch.zeros(0, device=son.device), good)
    st, bits = son.check()
    assert st == 0 and bits == 0
