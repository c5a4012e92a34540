"""Pins of the oracle's in-step pose uncertainty (Sec. III-D, Eq. 5-6).

Reading: the scan-match information of the soft expected-range model,
A = sum_b J_b J_b^T / sigma_r^2 (J_b at the robot's pose, on the map before
the scan is integrated), fused with the previous covariance propagated by
one step of odometry noise Q: Sigma_t = ((Sigma_{t-1} + Q)^-1 + A)^-1,
U_t = det(Sigma_t)^(1/3) / det(Q)^(1/3).

Pinned by: the closed form on an all-unknown map (no information:
Sigma = Sigma_0 + Q, U = 2 for a prior equal to Q); a corridor whose map is
constant along x, where x decouples exactly and Sigma_xx grows by Q_xx every
step while y and theta stay constrained; the fusion step recomputed with
numpy's inverse from soft Jacobians of the (separately pinned) soft-range
oracle; a closed room being less uncertain than the corridor; reset.
"""
import numpy as np
import pytest

from paper_2603_25834_gb300 import synth

Q1 = float(np.float32(0.01)) ** 2     # the noise parameters are fp32 configuration values
UQ = dict(u_mode=1, uq_samples=64, uq_range_sigma=0.01, uq_odo=(0.01, 0.01, 0.01),
          uq_prior=(0.01, 0.01, 0.01))


def corridor_world(W=256, H=64, j1=26, j2=37):
    occ = np.ones((H, W), np.uint8)
    occ[j1:j2 + 1, :] = 0                      # free rows j1..j2, walls elsewhere
    return occ


def make(orc, occ, pose, **p):
    spawn = np.tile(np.asarray(pose, np.float32), (1, 2, 1))
    inp = synth.custom_2d([occ], [90], 0.05, spawn)
    return orc.OracleBatch2D(inp, r_max=6.0, sigma=0.0, **UQ, **p)


def test_unknown_map_has_no_scan_information(orc):
    occ = corridor_world()
    b = make(orc, occ, (6.4, 1.6, 0.0))
    o = b.step(np.zeros((1, 2), np.float32))                # first scan: map all unknown
    np.testing.assert_allclose(b.sigma[0], [2e-4, 0, 0, 2e-4, 0, 2e-4], rtol=1e-6, atol=1e-18)
    assert o["obs"][0, -1] == pytest.approx(2.0, rel=1e-6)


def test_corridor_leaves_x_unconstrained(orc):
    occ = corridor_world()
    b = make(orc, occ, (6.4, 1.6, 0.0))
    # the belief is the corridor itself, free -3584 inside, occupied +3584
    # outside, restored before every step (a scan's update may end a grazing
    # beam one cell early, which would break the x-symmetry of the map)
    corridor = np.where(occ.reshape(-1) > 0, 3584, -3584).astype(np.int16)
    b.sigma[0] = [1e-4, 0, 0, 1e-4, 0, 1e-4]
    for t in range(12):
        b.belief[:] = corridor
        prev = b.sigma[0].copy()
        b.step(np.float32([[0.3, 0.0]]))                   # drive along the corridor
        s = b.sigma[0]
        assert s[0] == pytest.approx(prev[0] + Q1, rel=1e-9)
        assert abs(s[1]) < 1e-18 and abs(s[2]) < 1e-18
        assert s[3] < 1e-5 and s[5] < 1e-4


def test_fusion_step_matches_numpy(orc):
    inp = synth.paper_scale(E=1, W=128, B=90, seed=21)
    b = orc.OracleBatch2D(inp, r_max=6.0, sigma=0.01, **UQ)
    acts = synth.random_actions(6, 1, 2)
    for s in range(5):
        b.step(acts[s])
    L_before = b.belief.astype(np.float64) * (1.0 / 1024.0)
    S0 = b.sigma[0].copy()
    o = b.step(acts[5])
    assert b.done[0] == 0
    pose = np.array([b.x[0], b.y[0], b.th[0]], np.float64)
    r32 = float(np.float32(0.05))                        # res and ds are fp32 configuration values
    cfg = orc.soft_cfg(128, 128, 90, K=64, res=r32, ds=r32)
    _, gp, _ = orc.soft_ranges(cfg, L_before.astype(np.float32).reshape(1, 128, 128), [pose],
                               grad_pose=True)
    J = np.zeros((90, 3))
    for bb in range(90):
        gr = np.zeros((1, 90)); gr[0, bb] = 1.0
        _, g1, _ = orc.soft_ranges(cfg, L_before.astype(np.float32).reshape(1, 128, 128), [pose],
                                   gr=gr, grad_pose=True)
        J[bb] = g1[0]
    A = J.T @ J / 0.01 ** 2
    P = np.array([[S0[0], S0[1], S0[2]], [S0[1], S0[3], S0[4]], [S0[2], S0[4], S0[5]]]) + \
        np.diag([Q1, Q1, Q1])
    Sn = np.linalg.inv(np.linalg.inv(P) + A)
    np.testing.assert_allclose(b.sigma[0], [Sn[0, 0], Sn[0, 1], Sn[0, 2], Sn[1, 1], Sn[1, 2],
                                            Sn[2, 2]], rtol=1e-7, atol=1e-15)
    U = np.cbrt(np.linalg.det(Sn)) / np.cbrt(Q1 ** 3)
    assert o["obs"][0, -1] == pytest.approx(U, rel=1e-6)


def test_rotating_world_and_robot_rotates_the_covariance(orc):
    # belief = a world's own occupancy (+-3584); the same world rotated by
    # +90 degrees about the map centre with the robot rotated with it gives
    # Sigma' = R Sigma R^T, R = rot(90 deg) on (x, y), identity on theta
    inp = synth.paper_scale(E=1, W=96, B=90, seed=8)
    occ = inp.gt.reshape(96, 96)
    occ_r = np.empty_like(occ)
    for j in range(96):
        for i in range(96):
            occ_r[i, 95 - j] = occ[j, i]
    x, y, th = (float(v) for v in inp.spawn[0, 0])
    c = 96 * 0.05 / 2
    pose_r = (c - (y - c), c + (x - c), th + np.pi / 2)
    sig = []
    for grid, pose in ((occ, (x, y, th)), (occ_r, pose_r)):
        spawn = np.tile(np.asarray(pose, np.float32), (1, 2, 1))
        b = orc.OracleBatch2D(synth.custom_2d([grid], [90], 0.05, spawn), r_max=6.0, sigma=0.0,
                              **UQ)
        b.belief[:] = np.where(grid.reshape(-1) > 0, 3584, -3584).astype(np.int16)
        b.sigma[0] = [1e-4, 0, 0, 1e-4, 0, 1e-4]
        b.step(np.zeros((1, 2), np.float32))
        S = b.sigma[0]
        sig.append(np.array([[S[0], S[1], S[2]], [S[1], S[3], S[4]], [S[2], S[4], S[5]]]))
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    np.testing.assert_allclose(sig[1], R @ sig[0] @ R.T, rtol=2e-4, atol=1e-12)
    assert not np.allclose(sig[0], sig[1], rtol=1e-2)      # the rotation is not trivial


def test_reset_restarts_from_the_prior(orc):
    b = make(orc, corridor_world(), (6.4, 1.6, 0.0))
    for _ in range(3):
        b.step(np.float32([[0.3, 0.0]]))
    b.done[0] = 1
    o = b.step(np.zeros((1, 2), np.float32))
    np.testing.assert_allclose(b.sigma[0], [2e-4, 0, 0, 2e-4, 0, 2e-4], rtol=1e-6, atol=1e-18)
    assert o["obs"][0, -1] == pytest.approx(2.0, rel=1e-6)
