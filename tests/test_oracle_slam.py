"""Pins of the oracle's SLAM backbone in the step (u_mode 2; Sec. III-D).

* Window bookkeeping: the pose count grows by one per step up to L, then
  the window slides; a reset restarts it at one pose.
* Straight motion along x with no returned beam (no scan information): x
  decouples from the heading, so the newest pose's variance along x is the
  chain closed form 1/prior_info + (n-1) sigma_odo^2 for a window of n
  poses, and stays there at n = L once it slides and the oldest pose is
  re-anchored.
* The first step of an episode integrates its scan with weight 1, so the
  weighted and the unweighted update give the same map after one step; the
  weights of later steps are the steps' normalised match scores.
"""
import numpy as np
import pytest

from paper_2603_25834_gb300 import synth

SIG2 = float(np.float32(0.01)) ** 2


def empty_world(L=6, **p):
    occ = np.zeros((80, 200), np.uint8)
    spawn = np.tile(np.float32([1.0, 2.0, 0.0]), (1, 2, 1))
    inp = synth.custom_2d([occ], [32], 0.05, spawn)
    import oracle
    return oracle.OracleBatch2D(inp, r_max=1.0, sigma=0.0, u_mode=2, slam_window=L, **p)


def test_window_counts_slide_and_reset(orc):
    b = empty_world(L=4)
    counts = []
    for s in range(7):
        b.step(np.float32([[0.2, 0.0]]))
        counts.append(int(b.win_n[0]))
    assert counts == [1, 2, 3, 4, 4, 4, 4]
    b.done[0] = 1
    b.step(np.float32([[0.2, 0.0]]))
    assert b.win_n[0] == 1


def test_straight_motion_without_scans_is_dead_reckoning(orc):
    L = 6
    b = empty_world(L=L, slam_prior_info=(1.0 / SIG2,) * 3)
    for s in range(10):
        b.step(np.float32([[0.3, 0.0]]))
        n = int(b.win_n[0])
        assert b.slam_match[0].tolist() == [0.0, 0.0, 0.0]
        prior_var = 1.0 / float(np.float32(1.0 / SIG2))      # fp32 configuration value
        assert b.sigma[0, 0] == pytest.approx(prior_var + (n - 1) * SIG2, rel=1e-9)
        assert abs(b.sigma[0, 1]) < 1e-15 and abs(b.sigma[0, 2]) < 1e-15
    assert n == L


def test_first_scan_has_full_weight(orc):
    inp = synth.paper_scale(E=2, W=128, B=90, seed=33)
    acts = synth.random_actions(5, 2, 4)
    import oracle
    w = oracle.OracleBatch2D(inp, r_max=6.0, sigma=0.01, u_mode=2, slam_weighted=1)
    u = oracle.OracleBatch2D(inp, r_max=6.0, sigma=0.01, u_mode=2, slam_weighted=0)
    w.step(acts[0])
    u.step(acts[0])
    assert np.array_equal(w.belief, u.belief) and np.all(w.slam_upd_w == 1.0)
    for s in range(1, 5):
        w.step(acts[s])
        np.testing.assert_array_equal(w.slam_upd_w, w.slam_match[:, 0])
        assert np.all(w.slam_upd_w < 1.0)


def test_aligned_scan_is_integrated_at_the_optimised_pose(orc):
    """Sec. III-D: the scan enters the occupancy grid after the window
    optimisation has aligned it.  Each step's per-cell counts must equal an exact-rational
    recount of that step's measured ranges walked from the window's newest
    optimised pose -- not from the simulator's true pose, from which the
    recount differs whenever the two poses differ."""
    from tests.test_oracle_step import bordered, recount_at
    occ = bordered(48, 40)
    occ[10:14, 20:30] = 1
    occ[25:36, 8:11] = 1
    occ[28:31, 30:44] = 1
    spawn = np.tile(np.float32([1.21, 1.03, 0.3]), (1, 2, 1))
    inp = synth.custom_2d([occ], [40], 0.05, spawn)
    import oracle
    b = oracle.OracleBatch2D(inp, r_max=1.5, sigma=0.02, u_mode=2, slam_window=4)
    acts = synth.random_actions(10, 1, 21, v_max=0.3)
    discriminated = 0
    for s in range(10):
        o = b.step(acts[s], counts=True)
        if b.done[0]:
            break
        n = int(b.win_n[0])
        est = b.win_x[0, n - 1]
        h, m = recount_at(orc, b, o, est)
        np.testing.assert_array_equal(o["cnt_h"], h, err_msg="hits step %d" % s)
        np.testing.assert_array_equal(o["cnt_m"], m, err_msg="misses step %d" % s)
        assert o["ray_cells"][0] == int((h + m).sum())
        ht, mt = recount_at(orc, b, o, (b.x[0], b.y[0], b.th[0]))
        if not (np.array_equal(ht, h) and np.array_equal(mt, m)):
            discriminated += 1
    assert discriminated >= 3
