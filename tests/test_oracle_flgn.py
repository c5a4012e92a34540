"""Pins of the oracle's fixed-lag window Gauss-Newton (Sec. III-D, Eq. 5-6).

* Consistent data (odometry = the exact relative motions of a trajectory,
  pose factors = the true poses): Gauss-Newton from a perturbed start
  returns the trajectory.
* A straight line with the heading pinned: the newest pose's marginal
  variance is the closed form 1/w_prior + (L-1)/w_odo per axis, and a pose
  factor on the newest pose combines with it as information adds.
* A window of one pose: prior and pose factor informations add.
* Rotating the whole problem by phi rotates the solution and the covariance
  (R Sigma R^T on x, y).
"""
import math

import numpy as np
import pytest


def trajectory(rng, L):
    x = np.zeros((L, 3))
    x[0] = [rng.uniform(1, 5), rng.uniform(1, 5), rng.uniform(-3, 3)]
    for i in range(1, L):
        th = x[i - 1, 2]
        v, w = rng.uniform(0.02, 0.06), rng.uniform(-0.2, 0.2)
        x[i] = [x[i - 1, 0] + v * math.cos(th), x[i - 1, 1] + v * math.sin(th),
                math.remainder(th + w, 2 * math.pi)]
    return x


def odometry(x):
    u = []
    for i in range(len(x) - 1):
        c, s = math.cos(x[i, 2]), math.sin(x[i, 2])
        dx, dy = x[i + 1, 0] - x[i, 0], x[i + 1, 1] - x[i, 1]
        u.append([c * dx + s * dy, -s * dx + c * dy,
                  math.remainder(x[i + 1, 2] - x[i, 2], 2 * math.pi)])
    return np.array(u)


@pytest.mark.parametrize("seed", range(4))
def test_consistent_data_is_recovered(orc, seed):
    rng = np.random.default_rng(seed)
    L = 8
    xt = trajectory(rng, L)
    wm = np.zeros((L, 3))
    wm[::3] = 1e4
    x0 = xt + rng.normal(0, [0.05, 0.05, 0.05], size=xt.shape)
    x, cov, rc = orc.fixed_lag_gn(x0, odometry(xt), xt, wm, xt[0], [1e4] * 3, [1e4] * 3, iters=6)
    assert rc == 0
    d = x - xt
    d[:, 2] = np.remainder(d[:, 2] + math.pi, 2 * math.pi) - math.pi
    assert np.abs(d).max() < 1e-9
    assert np.all(np.linalg.eigvalsh(cov) > 0)


def test_straight_line_variance_closed_form(orc):
    L = 6
    xt = np.array([[1.0 + 0.05 * i, 2.0, 0.0] for i in range(L)])
    wp, wo, big = 400.0, 2500.0, 1e12
    wm = np.zeros((L, 3))
    x, cov, rc = orc.fixed_lag_gn(xt, odometry(xt), xt, wm, xt[0], [wp, wp, big],
                                  [wo, wo, big], iters=2)
    chain = 1 / wp + (L - 1) / wo
    assert cov[0, 0] == pytest.approx(chain, rel=1e-6)
    assert cov[1, 1] == pytest.approx(chain, rel=1e-6)
    wm[-1] = [900.0, 100.0, 0.0]
    x, cov, rc = orc.fixed_lag_gn(xt, odometry(xt), xt, wm, xt[0], [wp, wp, big],
                                  [wo, wo, big], iters=2)
    assert cov[0, 0] == pytest.approx(1 / (1 / chain + 900.0), rel=1e-6)
    assert cov[1, 1] == pytest.approx(1 / (1 / chain + 100.0), rel=1e-6)


def test_single_pose_window(orc):
    z = [1.0, 2.0, 0.5]
    x, cov, rc = orc.fixed_lag_gn([[1.1, 1.9, 0.4]], np.zeros((0, 3)), [z], [[300.0, 200.0, 50.0]],
                                  [1.0, 2.0, 0.5], [100.0, 100.0, 50.0], [1.0] * 3, iters=3)
    np.testing.assert_allclose(np.diag(cov), [1 / 400.0, 1 / 300.0, 1 / 100.0], rtol=1e-12)
    np.testing.assert_allclose(x[0], z, atol=1e-12)


def test_rotating_the_problem_rotates_the_solution(orc):
    rng = np.random.default_rng(9)
    L = 7
    xt = trajectory(rng, L)
    u = odometry(xt) + rng.normal(0, 0.005, size=(L - 1, 3))
    meas = xt + rng.normal(0, 0.01, size=xt.shape)
    wm = np.zeros((L, 3))
    wm[2] = [2e3, 5e3, 1e3]
    wm[-1] = [8e3, 1e3, 4e3]
    args = dict(odo_info=[3e3, 1e3, 5e3], iters=5)
    phi = 0.7
    R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])

    def rot(p):
        p = np.array(p, np.float64).copy()
        p[..., :2] = p[..., :2] @ R.T
        p[..., 2] = np.remainder(p[..., 2] + phi + math.pi, 2 * math.pi) - math.pi
        return p
    # pose-factor information is diagonal in the world frame: rotate it as a
    # matrix only when it is isotropic in x, y
    wm_r = wm.copy()
    wm_r[:, 0] = wm_r[:, 1] = wm[:, :2].mean(axis=1)
    x1, c1, _ = orc.fixed_lag_gn(xt, u, meas, wm_r, xt[0], [1e3] * 3, **args)
    x2, c2, _ = orc.fixed_lag_gn(rot(xt), u, rot(meas), wm_r, rot(xt[0]), [1e3] * 3, **args)
    np.testing.assert_allclose(x2[:, :2], x1[:, :2] @ R.T, atol=1e-9)
    R3 = np.eye(3)
    R3[:2, :2] = R
    np.testing.assert_allclose(c2, R3 @ c1 @ R3.T, rtol=1e-7, atol=1e-14)
