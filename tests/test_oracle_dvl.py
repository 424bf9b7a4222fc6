"""Pins for the oracle's DVL model (Sec. III-A-3) against things other than
itself: the Janus geometry (angles between beams), a flat seabed's closed-form
ranges, exact velocity recovery from noise-free beams (four or three), the
range window and dropout, the least-squares error covariance sigma^2 (B^T B)^-1,
and the schedule of a constant period.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_01074_gb300 import scenes as S


def rot(yaw, pitch, roll):
    cy, sy, cp, sp, cr, sr = (math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch),
                              math.cos(roll), math.sin(roll))
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    Ry = np.array([[cr, 0, sr], [0, 1, 0], [-sr, 0, cr]])
    return Rz @ Rx @ Ry


def test_janus_geometry():
    P = O.DvlParams()
    b = O.dvl_beams(np.eye(3)[None], P.tilt)[0]
    assert np.allclose(np.linalg.norm(b, axis=1), 1.0)
    down = np.array([0.0, 0.0, -1.0])
    assert np.allclose(np.degrees(np.arccos(b @ down)), 30.0)
    # opposite beams are 2 tilt apart, neighbours are 90 degrees apart around the axis
    assert np.isclose(np.degrees(np.arccos(b[0] @ b[2])), 60.0)
    assert np.isclose(np.degrees(np.arccos(b[1] @ b[3])), 60.0)
    hz = b[:, :2] / np.linalg.norm(b[:, :2], axis=1, keepdims=True)
    assert np.allclose(hz[0] @ hz[1], 0.0) and np.allclose(hz[1] @ hz[2], 0.0)
    assert np.allclose(np.degrees(np.arctan2(hz[0, 1], hz[0, 0])), 45.0)
    # a pose rotates the beams rigidly
    R = rot(0.3, -0.2, 0.1)
    assert np.allclose(O.dvl_beams(R[None], P.tilt)[0], b @ R.T)


@pytest.mark.parametrize("pitch", [0.0, 12.0])
def test_flat_seabed_ranges(pitch):
    h = 6.0
    mesh = S.quad(-h, 40.0)
    tv = O.tri_verts(mesh)
    P = O.DvlParams()
    R = rot(0.4, math.radians(pitch), 0.0)
    t, _ = O.dvl_ranges(tv, [[0.3, -0.7, 0.0]], R[None], P.tilt)
    d = O.dvl_beams(R[None], P.tilt)[0]
    assert np.allclose(t[0], h / -d[:, 2], rtol=1e-12)
    if pitch == 0.0:
        assert np.allclose(t[0], h / math.cos(P.tilt), rtol=1e-12)


def test_noise_free_velocity_is_exact_with_four_or_three_beams():
    rng = np.random.default_rng(1)
    P = O.DvlParams(sigma_b=0.0)
    n = 200
    R = np.stack([rot(*rng.uniform(-0.5, 0.5, 3)) for _ in range(n)])
    v = rng.normal(size=(n, 3))
    t = rng.uniform(1.0, 40.0, (n, 4))
    t[n // 2:, 1] = np.inf                 # the second half has three beams
    vel, flags, _ = O.dvl_measure(R, v, t, P, seed=3)
    vs = np.einsum("nji,nj->ni", R, v)     # R^T v
    assert np.allclose(vel, vs, rtol=0, atol=1e-12)
    assert np.all(flags[: n // 2] == 0b11111) and np.all(flags[n // 2:] == 0b11101)


def test_range_window_and_dropout():
    P = O.DvlParams(sigma_b=0.0)
    R = np.eye(3)[None].repeat(5, 0)
    v = np.ones((5, 3))
    t = np.array([[P.r_min, P.r_max, 10.0, 10.0],                       # bounds included
                  [P.r_min * 0.999, P.r_max * 1.001, 10.0, 10.0],       # two out: dropout
                  [np.inf, 10.0, 10.0, 10.0],                           # three beams
                  [np.inf] * 4,                                         # nothing below
                  [0.0, 10.0, 10.0, 10.0]])                             # too close
    vel, flags, period = O.dvl_measure(R, v, t, P, seed=0)
    assert list(flags) == [0b11111, 0b01100, 0b11110, 0, 0b11110]
    assert np.all(vel[[1, 3]] == 0.0)
    assert np.allclose(period[[1, 3]], P.t_lost)
    assert np.isclose(period[0], P.t0 + P.t1 * P.r_max)
    assert np.isclose(period[2], P.t0 + P.t1 * 10.0)


def test_least_squares_error_covariance():
    # with all beams valid the fitted velocity's error is (B^T B)^-1 B^T sigma w:
    # zero mean, covariance sigma^2 (B^T B)^-1, B the beam matrix of the reading
    P = O.DvlParams(sigma_b=0.1)
    n = 40000
    R = np.eye(3)[None].repeat(n, 0)
    v = np.tile([0.4, -0.3, 0.05], (n, 1))
    t = np.full((n, 4), 10.0)
    vel, flags, _ = O.dvl_measure(R, v, t, P, seed=11)
    err = vel - v
    tau = P.tilt
    B = np.array([[math.sin(tau) * math.cos(a), math.sin(tau) * math.sin(a), -math.cos(tau)]
                  for a in np.radians([45, 135, 225, 315])])
    cov = P.sigma_b ** 2 * np.linalg.inv(B.T @ B)
    assert np.all(np.abs(err.mean(0)) < 4 * np.sqrt(np.diag(cov) / n))
    emp = np.cov(err.T)
    assert np.allclose(np.diag(emp), np.diag(cov), rtol=0.05)
    assert np.allclose(emp, cov, atol=0.05 * cov.max())


def test_schedule_of_a_constant_period():
    dt = 0.05
    for T, every in ((0.105, 3), (0.1, 2), (0.01, 1), (0.5, 10)):
        emit = O.dvl_schedule(np.full((3, 40), T), dt)
        assert np.array_equal(np.nonzero(emit[0])[0], np.arange(0, 40, every)), T
    # the period read at each measurement sets the next one
    per = np.array([[0.12, 9.0, 9.0, 0.04, 0.2, 9.0, 9.0, 9.0, 0.01, 0.01]])
    assert list(np.nonzero(O.dvl_schedule(per, 0.05)[0])[0]) == [0, 3, 4, 8, 9]
