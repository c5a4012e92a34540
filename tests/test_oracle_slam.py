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


# ---- scan-to-map Gauss-Newton correction of the match (slam_gn_iters) ------------
def _corr_world(seed=71, W=128):
    """A world-like int16 belief (+-3 nats on occupied / free cells) and a
    known pose on the 1 mm / 1 mrad lattice."""
    inp = synth.paper_scale(E=1, W=W, B=8, seed=seed)
    L = synth.logodds_maps(inp)[0]
    belief = np.rint(L * 1024.0).astype(np.int16)
    true = np.round(inp.spawn[0, 0].astype(np.float64), 3).astype(np.float32)
    return inp.res, belief, true


def _ranges_at(orc, belief, res, B, pose, K=64):
    cfg = orc.soft_cfg(belief.shape[1], belief.shape[0], B, K=K, res=res, ds=res)
    L = (belief.astype(np.float64) / 1024.0).astype(np.float32)[None]
    r, _, _ = orc.soft_ranges(cfg, L, np.asarray(pose, np.float32)[None])
    return r[0].astype(np.float32)


def test_correction_recovers_a_known_pose(orc):
    """Ranges of the soft model at a known pose (itself on the lattice): from
    a match 3 cm / 2 cm / 8 mrad off, the Gauss-Newton steps reach it and the
    lattice rounding returns it exactly; each step brings the pose closer (a
    wrong sign or a dropped Jacobian term diverges, and the search box then
    keeps the match)."""
    res, belief, true = _corr_world()
    B = 180
    z = _ranges_at(orc, belief, res, B, true)
    start = (true.astype(np.float64) + [0.03, -0.02, 0.008]).astype(np.float32)
    out = orc.slam_correct(belief, res, 0.0, z, start, iters=6)
    np.testing.assert_array_equal(out, true)
    errs = [np.abs(orc.slam_correct(belief, res, 0.0, z, start, iters=k).astype(np.float64) - true).max()
            for k in (1, 2, 3)]
    assert errs[0] < 0.03 and errs[1] < errs[0] and errs[2] <= errs[1]


def test_correction_keeps_the_match_outside_the_search_box(orc):
    """An iterate that leaves the matcher's box (here +-(0 + 1) cells) abandons
    the correction: the match comes back unchanged (not rounded)."""
    res, belief, true = _corr_world()
    z = _ranges_at(orc, belief, res, 180, true)
    start = (true.astype(np.float64) + [0.08, 0.0, 0.0]).astype(np.float32)
    out = orc.slam_correct(belief, res, 0.0, z, start, iters=3, n_xy=0)
    np.testing.assert_array_equal(out, start)


def test_correction_on_an_unknown_map_only_rounds(orc):
    """All cells unknown: every sample has p = 1/2 at zero gradient, so J = 0,
    the steps are zero and the match is returned on the lattice."""
    res, belief, true = _corr_world()
    z = np.full(90, 1.7, np.float32)
    start = np.float32([2.34567, 3.45678, 0.123456])
    out = orc.slam_correct(np.zeros_like(belief), res, 0.0, z, start, iters=3)
    np.testing.assert_array_equal(out, np.round(start.astype(np.float64), 3).astype(np.float32))


def test_corrected_match_is_the_window_measurement(orc):
    """In the step: the correction runs on the map before this scan, from the
    correlative match, with this scan's measured ranges (a direct call on a
    copy of that map gives the same pose); its result is the window's newest
    pose measurement; an episode's first scan keeps the match; an accepted
    correction is on the lattice and inside the matcher's search box, and
    most corrections are accepted."""
    import oracle
    inp = synth.paper_scale(E=3, W=128, B=180, seed=34)
    acts = synth.random_actions(8, 3, 5)
    b = oracle.OracleBatch2D(inp, r_max=6.0, sigma=0.01, u_mode=2, slam_gn_iters=2)
    accepted = total = 0
    for s in range(8):
        before = b.belief.copy()
        o = b.step(acts[s])
        for e in range(3):
            n = int(b.win_n[e])
            np.testing.assert_array_equal(b.win_meas[e, n - 1], b.slam_gn_pose[e])
            if n == 1:
                np.testing.assert_array_equal(b.slam_gn_pose[e], b.slam_pose[e])
                continue
            m0, W, H = int(b.map_off[e]), int(b.map_w[e]), int(b.map_h[e])
            direct = orc.slam_correct(before[m0:m0 + W * H].reshape(H, W), inp.res, 0.0,
                                      o["z"][e, :int(b.n_beams[e])], b.slam_pose[e], iters=2)
            np.testing.assert_array_equal(b.slam_gn_pose[e], direct)
            total += 1
            if np.array_equal(b.slam_gn_pose[e], b.slam_pose[e]):
                continue
            accepted += 1
            v = b.slam_gn_pose[e].astype(np.float64) * 1000.0
            assert np.all(np.abs(v - np.rint(v)) < 1e-2)
            d = np.abs(b.slam_gn_pose[e].astype(np.float64) - b.slam_pose[e])
            assert d[0] <= 6 * inp.res + 1e-3 and d[1] <= 6 * inp.res + 1e-3 and d[2] <= 0.06 + 1e-3
    assert accepted >= total // 2, (accepted, total)
