"""Pins for the oracle's underwater image formation (Sec. III-A-1, Eq. 1)
against properties the model fixes, not against a retyped formula: the
identity at zero depth or zero coefficients, the half-value depths of the
attenuation and backscatter terms, the limit at great depth, the fixed point
J = B_inf, composition of two layers of water, monotonic approach to the
veiling light, and channel independence.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O


def rand_coef(rng):
    return np.concatenate([rng.uniform(0.02, 0.8, 3), rng.uniform(0.02, 0.8, 3), rng.uniform(0.0, 1.0, 3)])


def test_zero_depth_and_zero_coefficients_give_the_in_air_image():
    rng = np.random.default_rng(1)
    J = rng.random((500, 3), dtype=np.float32)
    assert np.array_equal(O.uw_image(J, np.zeros(500, np.float32), rand_coef(rng)), J.astype(np.float64))
    coef = np.concatenate([np.zeros(6), rng.uniform(0, 1, 3)])
    d = rng.uniform(0, 50, 500).astype(np.float32)
    d[:10] = np.inf
    assert np.array_equal(O.uw_image(J, d, coef), J.astype(np.float64))


def test_half_value_depths_fix_the_exponent_scales():
    # B_inf = 0: the signal halves at d = ln 2 / beta_attn; J = 0: the veiling
    # light reaches half of B_inf at d = ln 2 / beta_bs (beta_attn set apart)
    for beta in (0.05, 0.3, 1.7):
        d = np.array([math.log(2.0) / beta], np.float32)
        J = np.array([[0.8, 0.6, 0.4]], np.float32)
        I = O.uw_image(J, d, [beta] * 3 + [9.0] * 3 + [0.0] * 3)
        assert np.allclose(I, J * np.exp(-beta * float(d[0])), rtol=1e-14)
        assert np.allclose(I, J / 2.0, rtol=1e-6)          # d is ln 2 / beta rounded to FP32
        B = np.array([0.2, 0.5, 0.9])
        I = O.uw_image(np.zeros((1, 3), np.float32), d, [5.0] * 3 + [beta] * 3 + list(B))
        assert np.allclose(I[0], B / 2.0, rtol=1e-6)


def test_great_depth_gives_the_veiling_light():
    rng = np.random.default_rng(2)
    coef = rand_coef(rng)
    J = rng.random((64, 3), dtype=np.float32)
    for d in (1e4, np.inf):
        I = O.uw_image(J, np.full(64, d, np.float32), coef)
        assert np.allclose(I, np.broadcast_to(coef[6:], I.shape), rtol=0, atol=1e-12)


def test_object_at_the_veiling_light_is_invisible():
    # J = B_inf and beta_attn = beta_bs: the image equals B_inf at every depth
    rng = np.random.default_rng(3)
    B = rng.uniform(0.1, 0.9, 3)
    beta = rng.uniform(0.05, 0.5, 3)
    J = np.tile(B.astype(np.float32), (100, 1))
    d = rng.uniform(0, 80, 100).astype(np.float32)
    I = O.uw_image(J, d, np.concatenate([beta, beta, B]))
    assert np.allclose(I, J.astype(np.float64), rtol=0, atol=1e-7)


def test_two_layers_compose_into_one():
    # with beta_attn = beta_bs the model is an affine contraction towards
    # B_inf; imaging through d1 and then through d2 equals imaging through d1 + d2
    rng = np.random.default_rng(4)
    beta = rng.uniform(0.02, 0.6, 3)
    coef = np.concatenate([beta, beta, rng.uniform(0, 1, 3)])
    J = rng.random((300, 3), dtype=np.float32)
    d1 = rng.uniform(0, 20, 300).astype(np.float32)
    d2 = rng.uniform(0, 20, 300).astype(np.float32)
    once = O.uw_image(J, d1, coef)
    twice = O.uw_image(once.astype(np.float32), d2, coef)
    direct = O.uw_image(J, (d1.astype(np.float64) + d2).astype(np.float32), coef)
    assert np.allclose(twice, direct, rtol=0, atol=2e-6)
    # ... which a swap of the two terms would break
    swapped = J * (1 - np.exp(-beta * d1[:, None])) + coef[6:] * np.exp(-beta * d1[:, None])
    assert not np.allclose(once, swapped, atol=1e-3)


def test_monotonic_approach_to_the_veiling_light():
    rng = np.random.default_rng(5)
    coef = rand_coef(rng)
    J = rng.random((1, 3), dtype=np.float32)
    d = np.linspace(0, 30, 301).astype(np.float32)
    I = O.uw_image(np.repeat(J, d.size, 0), d, coef)
    gap = np.abs(I - coef[6:])
    beta_a, beta_b = coef[:3], coef[3:6]
    for c in range(3):
        if beta_a[c] == beta_b[c]:
            assert np.all(np.diff(gap[:, c]) <= 1e-15)
    # with equal coefficients the distance to B_inf shrinks monotonically
    coef2 = np.concatenate([coef[:3], coef[:3], coef[6:]])
    I2 = O.uw_image(np.repeat(J, d.size, 0), d, coef2)
    assert np.all(np.diff(np.abs(I2 - coef[6:]), axis=0) <= 1e-15)


def test_channels_are_independent():
    rng = np.random.default_rng(6)
    coef = rand_coef(rng)
    J = rng.random((200, 3), dtype=np.float32)
    d = rng.uniform(0, 40, 200).astype(np.float32)
    perm = [2, 0, 1]
    I = O.uw_image(J, d, coef)
    coef_p = np.concatenate([coef[:3][perm], coef[3:6][perm], coef[6:][perm]])
    Ip = O.uw_image(np.ascontiguousarray(J[:, perm]), d, coef_p)
    assert np.array_equal(Ip, I[:, perm])


@pytest.mark.parametrize("shape", [(7, 5), (1, 1), (0,)])
def test_shapes(shape):
    rng = np.random.default_rng(7)
    J = rng.random(shape + (3,), dtype=np.float32)
    d = rng.uniform(0, 10, shape).astype(np.float32)
    I = O.uw_image(J, d, rand_coef(rng))
    assert I.shape == J.shape
