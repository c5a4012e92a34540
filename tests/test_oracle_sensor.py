"""Pins of the oracle's paper sensor mode and uncertainty bridge.

Sec. IV-A sensor: 128 rays over the 180-degree front field of view, minimum
range 0.1 m, ranges given to two decimal places.  Expected values are
analytic wall distances rounded by hand, the minimum range itself, the
geometry of a front arc, and the variance of rounded Gaussian noise
(sigma^2 + q^2/12 for a rounding step q).  Sec. III-G, Eq. 21-22 bridge:
alpha = min(1, t / T_bridge), U = alpha U_new + (1 - alpha) U_old, pinned at
its end points, its midpoint and its monotonicity.
"""
import math

import numpy as np
import pytest

from tests.test_oracle_step import bordered, one_env


def test_two_decimal_ranges_of_analytic_distances(orc):
    # 64 x 64 at 0.1 m, border walls; beams at 0, 90, 180, 270 degrees
    b = one_env(orc, bordered(64, 64), 4, 0.1, (1.234, 2.071, 0.0), r_max=10.0, sigma=0.0,
                decimals=2)
    o = b.step(np.zeros((1, 2), np.float32))
    exact = [6.3 - 1.234, 6.3 - 2.071, 1.234 - 0.1, 2.071 - 0.1]   # 5.066 4.229 1.134 1.971
    np.testing.assert_allclose(o["z_true"][0], exact, atol=2e-6)
    np.testing.assert_array_equal(o["z"][0], np.float32([5.07, 4.23, 1.13, 1.97]))


def test_zero_decimals_gives_whole_metres(orc):
    b = one_env(orc, bordered(64, 64), 4, 0.1, (1.234, 2.071, 0.0), r_max=10.0, sigma=0.0,
                decimals=0)
    o = b.step(np.zeros((1, 2), np.float32))
    np.testing.assert_array_equal(o["z"][0], np.float32([5.0, 4.0, 1.0, 2.0]))


def test_minimum_range_clips_returned_beams(orc):
    # wall cell column 0 covers x in [0, 0.1); the robot at x = 0.15 sees it
    # 0.05 m behind (beam 2), below r_min = 0.1
    b = one_env(orc, bordered(64, 64), 4, 0.1, (0.15, 3.2, 0.0), r_max=10.0, sigma=0.0,
                r_min=0.1)
    o = b.step(np.zeros((1, 2), np.float32))
    assert o["z_true"][0, 2] == pytest.approx(0.05, abs=2e-6)
    assert o["z"][0, 2] == np.float32(0.1) and o["hit"][0, 2] == 1
    np.testing.assert_allclose(o["z"][0, [0, 1, 3]], [6.3 - 0.15, 6.3 - 3.2, 3.2 - 0.1], atol=2e-6)


def test_no_return_reports_unrounded_r_max(orc):
    occ = np.zeros((64, 64), np.uint8)
    b = one_env(orc, occ, 16, 0.1, (3.2, 3.2, 0.3), r_max=2.345, sigma=0.01, decimals=1)
    o = b.step(np.zeros((1, 2), np.float32))
    assert not o["hit"].any()
    np.testing.assert_array_equal(o["z"][0], np.float32(2.345))


def test_front_arc_of_128_beams(orc):
    # A wall only at x < 0.3 m (no border walls).  Facing +x, the robot at
    # the centre sees nothing.  Facing -x, beam b (at heading - pi/2 +
    # b*pi/127) returns iff it reaches the wall face x = 0.3 before leaving
    # the 6.4 m map through y = 0 or y = 6.4; then its range is analytic.
    occ = np.zeros((64, 64), np.uint8)
    occ[:, :3] = 1
    fwd = one_env(orc, occ, 128, 0.1, (3.2, 3.2, 0.0), r_max=10.0, sigma=0.0, fov=math.pi)
    o = fwd.step(np.zeros((1, 2), np.float32))
    assert not o["hit"].any()
    th = float(np.float32(math.pi - 1e-3))
    back = one_env(orc, occ, 128, 0.1, (3.2, 3.2, th), r_max=10.0, sigma=0.0, fov=math.pi)
    o = back.step(np.zeros((1, 2), np.float32))
    ang = th - math.pi / 2 + np.arange(128) * math.pi / 127
    dx, dy = np.cos(ang), np.sin(ang)
    t_wall = np.where(dx < 0, (3.2 - 0.3) / np.maximum(-dx, 1e-12), np.inf)
    t_side = 3.2 / np.maximum(np.abs(dy), 1e-12)
    clear = np.abs(t_wall - t_side) > 0.05          # away from the corner case
    expect_hit = t_wall < t_side
    np.testing.assert_array_equal(o["hit"][0][clear], expect_hit[clear])
    assert expect_hit.sum() > 60
    for bb in np.nonzero(expect_hit & clear)[0]:
        assert o["z"][0, bb] == pytest.approx(t_wall[bb], abs=1e-4), bb


def test_rounded_noise_has_the_rounding_variance(orc):
    b = one_env(orc, bordered(96, 96), 360, 0.1, (4.81, 4.77, 0.0), r_max=10.0, sigma=0.01,
                decimals=2)
    err = []
    for _ in range(30):
        o = b.step(np.zeros((1, 2), np.float32))
        z = o["z"][0].astype(np.float64)
        np.testing.assert_allclose(z * 100, np.rint(z * 100), atol=1e-3)
        err.append(z - o["z_true"][0])
    err = np.concatenate(err)
    assert abs(err.mean()) < 1e-3
    # a rounding done before the noise would give 0.0100 (4 % lower)
    assert err.std() == pytest.approx(math.sqrt(0.01 ** 2 + 0.01 ** 2 / 12), rel=0.02)


def test_bridge_end_points_midpoint_and_monotone(orc):
    u_old = np.float32([0.3, 1.2, 0.0, 0.7])
    u_new = np.float32([0.9, 0.2, 2.0, 0.7])
    np.testing.assert_array_equal(orc.bridge_u(u_old, u_new, 0, 1000), u_old)
    np.testing.assert_array_equal(orc.bridge_u(u_old, u_new, 1000, 1000), u_new)
    np.testing.assert_array_equal(orc.bridge_u(u_old, u_new, 7000, 1000), u_new)
    np.testing.assert_allclose(orc.bridge_u(u_old, u_new, 500, 1000), (u_old + u_new) / 2,
                               rtol=1e-7, atol=1e-7)
    seq = np.stack([orc.bridge_u(u_old, u_new, t, 64) for t in range(0, 70)])
    d = np.diff(seq, axis=0) * np.sign(u_new - u_old)
    assert np.all(d >= 0)
    # equal inputs stay equal up to the fp32 rounding of the two products
    assert np.abs(seq[:, 3] - np.float32(0.7)).max() <= 2 * np.spacing(np.float32(0.7))
