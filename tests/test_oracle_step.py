"""Pins of the oracle's environment step against closed forms and hand cases.

Sec. IV-A sensor (ranges to the first obstacle, N(0, sigma^2) noise),
Sec. III-D log-odds grid update, Table I map entropy, Sec. III-E reward
(Eq. 7-17) and Eq. 3 observation.  Expected values are analytic distances,
N*ln2, hand-computed reward branches, or an exact-rational recount of the
traversed cells; none comes from the oracle itself.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2603_25834_gb300 import synth
from tests.test_oracle_walk import brute_path

LN2 = math.log(2.0)


def bordered(W, H):
    o = np.zeros((H, W), np.uint8)
    o[0, :] = o[-1, :] = o[:, 0] = o[:, -1] = 1
    return o


def one_env(orc, occ, beams, res, pose, K=2, **p):
    spawn = np.tile(np.asarray(pose, np.float32), (1, K, 1))
    inp = synth.custom_2d([occ], [beams], res, spawn)
    return orc.OracleBatch2D(inp, **p)


def test_axis_aligned_ranges_are_analytic(orc):
    # 64 x 64 at 0.1 m, border walls only; robot at (1.23, 2.07), heading 0;
    # beams at 0, 90, 180, 270 degrees.  Walls: cells 0 and 63 on each axis.
    b = one_env(orc, bordered(64, 64), 4, 0.1, (1.23, 2.07, 0.0), r_max=10.0, sigma=0.0)
    o = b.step(np.zeros((1, 2), np.float32))
    expect = [6.3 - 1.23, 6.3 - 2.07, 1.23 - 0.1, 2.07 - 0.1]
    np.testing.assert_allclose(o["z"][0], expect, atol=2e-6)
    np.testing.assert_array_equal(o["z"][0], o["z_true"][0])
    assert o["hit"][0].tolist() == [1, 1, 1, 1]


def test_empty_map_gives_max_range(orc):
    occ = np.zeros((40, 40), np.uint8)
    b = one_env(orc, occ, 64, 0.1, (2.0, 2.0, 0.3), r_max=1.5, sigma=0.01)
    o = b.step(np.zeros((1, 2), np.float32))
    assert np.all(o["z"][0] == np.float32(1.5)) and not o["hit"].any()
    # rays that leave a small map also report r_max and no hit
    b = one_env(orc, np.zeros((6, 6), np.uint8), 32, 0.1, (0.3, 0.3, 0.0), r_max=5.0)
    o = b.step(np.zeros((1, 2), np.float32))
    assert np.all(o["z"][0] == np.float32(5.0)) and not o["hit"].any()
    # the belief then holds misses only
    assert b.belief.max() <= 0 and b.belief.min() < 0


def test_all_unknown_map_entropy_is_n_ln2(orc):
    # plain fp64 summation of n terms: relative error below n * 2^-53
    for n in (1, 7, 4096, 65536):
        assert orc.map_entropy(np.zeros(n, np.int16), 1 / 1024) == pytest.approx(
            n * LN2, rel=max(1e-15, n * 2.0 ** -53))
    # h is symmetric in L and maximal at L = 0
    for l in (0.1, 1.0, 3.5):
        assert orc.cell_entropy(l) == pytest.approx(orc.cell_entropy(-l), rel=1e-14)
        assert orc.cell_entropy(l) < LN2
    # closed form at p = sigma(3.5)
    p = 1 / (1 + math.exp(-3.5))
    assert orc.cell_entropy(3.5) == pytest.approx(-p * math.log(p) - (1 - p) * math.log(1 - p),
                                                  rel=1e-14)


def test_entropy_reward_is_information_gain(orc):
    inp = synth.plain_1env()
    b = orc.OracleBatch2D(inp, r_max=5.0)
    N = int(inp.map_off[-1])
    o = b.step(np.zeros((1, 2), np.float32))
    # first step from the all-unknown map: dH = N ln2 - H_after
    L = b.belief.astype(np.float64) / 1024
    p = 1 / (1 + np.exp(-L))
    H_after = float(np.sum(-p * np.log(p) - (1 - p) * np.log(1 - p)))
    assert o["terms"][0, 0] == pytest.approx(N * LN2 - H_after, rel=1e-9)
    assert o["terms"][0, 0] > 0


def test_update_hand_case_and_clamp(orc):
    # 10 x 10 at 0.1 m, wall column i = 6; robot at the centre of cell (2, 3)
    # looking along +x with one beam: cells 2..5 miss, cell 6 hit.
    occ = np.zeros((10, 10), np.uint8)
    occ[:, 6] = 1
    b = one_env(orc, occ, 1, 0.1, (0.25, 0.35, 0.0), r_max=5.0, sigma=0.0)
    o = b.step(np.zeros((1, 2), np.float32), counts=True)
    L = b.env_belief(0)
    assert L[3, 2:7].tolist() == [-410, -410, -410, -410, 870]
    assert np.count_nonzero(L) == 5
    assert o["cnt_h"].sum() == 1 and o["cnt_m"].sum() == 4
    assert o["ray_cells"][0] == 5 and o["gt_cells"][0] == 5
    assert o["z"][0, 0] == pytest.approx(0.35, abs=1e-6)
    for _ in range(8):
        b.step(np.zeros((1, 2), np.float32))
    L = b.env_belief(0)
    # nine scans: +870*9 and -410*9 saturate at +-3584
    assert L[3, 2:7].tolist() == [-3584, -3584, -3584, -3584, 3584]


def test_many_beams_through_one_cell_sum_then_clamp(orc):
    # 8 beams all start in the robot cell: one step gives it 8 misses at once.
    occ = bordered(20, 20)
    b = one_env(orc, occ, 8, 0.1, (1.05, 1.05, 0.0), r_max=5.0, sigma=0.0)
    o = b.step(np.zeros((1, 2), np.float32), counts=True)
    rc = 10 * 20 + 10
    assert o["cnt_m"][rc] == 8 and o["cnt_h"][rc] == 0
    assert b.belief[rc] == -3280
    b.step(np.zeros((1, 2), np.float32))
    assert b.belief[rc] == -3584


def recount(orc, b, o, e=0):
    """Exact-rational recount of one step's per-cell hit/miss counts."""
    return recount_at(orc, b, o, (b.x[e], b.y[e], b.th[e]), e)


def recount_at(orc, b, o, pose, e=0):
    """Exact-rational recount of env e's per-cell hit/miss counts for the
    step's measured ranges walked from `pose` (x, y, th)."""
    W, H, B = int(b.map_w[e]), int(b.map_h[e]), int(b.n_beams[e])
    res = np.float32(b.inp.res)
    s, c = orc.sincosf(float(pose[2]))
    cb, sb = orc.beam_dirs(B, b.p["fov"])
    h = np.zeros(W * H, np.int64)
    m = np.zeros(W * H, np.int64)
    for k in range(B):
        Px, Py, Dx, Dy = orc.ray_setup(float(pose[0]), float(pose[1]), c, s, float(cb[k]),
                                       float(sb[k]), float(res))
        z = np.float32(o["z"][e, k])
        Tz = int(np.rint(np.float32(np.float32(z / res) * np.float32(65536.0))))
        cells, left = brute_path(Px, Py, Dx, Dy, Tz, W, H)
        for n, cell in enumerate(cells):
            if n == len(cells) - 1 and not left and o["hit"][e, k]:
                h[cell] += 1
            else:
                m[cell] += 1
    return h, m


def test_counts_and_map_match_exact_recount(orc):
    occ = bordered(16, 16)
    occ[5:9, 9:11] = 1
    occ[11, 3:7] = 1
    b = one_env(orc, occ, 24, 0.1, (0.62, 0.71, 0.4), r_max=1.2, sigma=0.01)
    acts = synth.random_actions(4, 1, 11, v_max=0.3)
    for s in range(4):
        L0 = b.belief.copy()
        o = b.step(acts[s], counts=True)
        if b.done[0]:
            break
        h, m = recount(orc, b, o)
        np.testing.assert_array_equal(o["cnt_h"], h)
        np.testing.assert_array_equal(o["cnt_m"], m)
        exp = np.clip(L0.astype(np.int64) + 870 * h - 410 * m, -3584, 3584)
        np.testing.assert_array_equal(b.belief, exp)
        # untouched cells are unchanged; |L| never exceeds the clamp
        assert np.all(b.belief[(h + m) == 0] == L0[(h + m) == 0])
        assert np.abs(b.belief).max() <= 3584
        assert o["ray_cells"][0] == int((h + m).sum())


def test_noise_statistics(orc):
    inp = synth.plain_1env()
    b = orc.OracleBatch2D(inp, r_max=5.0, sigma=0.01)
    d = []
    for s in range(60):
        o = b.step(np.zeros((1, 2), np.float32))
        hit = o["hit"][0].astype(bool)
        zt = o["z_true"][0][hit]
        ok = (zt > 0.05) & (zt < 4.95)
        d.append((o["z"][0][hit] - zt)[ok])
    d = np.concatenate(d).astype(np.float64)
    assert d.size > 3000
    assert abs(d.mean()) < 0.0015
    assert abs(d.std() - 0.01) < 0.001


def test_motion_closed_forms(orc):
    occ = bordered(200, 200)
    # straight line
    b = one_env(orc, occ, 4, 0.1, (5.0, 5.0, 0.5), r_max=2.0)
    for _ in range(20):
        b.step(np.array([[0.4, 0.0]], np.float32))
    assert b.x[0] == pytest.approx(5.0 + 20 * 0.04 * math.cos(0.5), abs=2e-5)
    assert b.y[0] == pytest.approx(5.0 + 20 * 0.04 * math.sin(0.5), abs=2e-5)
    assert b.th[0] == np.float32(0.5)
    # pure rotation with heading wrap to [-pi, pi)
    b = one_env(orc, occ, 4, 0.1, (5.0, 5.0, 3.0), r_max=2.0)
    for _ in range(5):
        b.step(np.array([[0.0, 1.0]], np.float32))
    assert b.x[0] == np.float32(5.0) and b.y[0] == np.float32(5.0)
    assert b.th[0] == pytest.approx(3.5 - 2 * math.pi, abs=1e-6)
    # clamps on v and w (Eq. 4 bounds, v_max = 0.5)
    b = one_env(orc, occ, 4, 0.1, (5.0, 5.0, 0.0), r_max=2.0)
    b.step(np.array([[9.0, -9.0]], np.float32))
    assert b.x[0] == pytest.approx(5.05, abs=1e-6) and b.th[0] == pytest.approx(-0.1, abs=1e-7)
    b.step(np.array([[-3.0, 0.0]], np.float32))
    assert b.x[0] == pytest.approx(5.05, abs=1e-6)
    # constant (v, w) arc: Euler tracks the exact circle to O(dt)
    b = one_env(orc, occ, 4, 0.1, (5.0, 5.0, 0.0), r_max=2.0)
    v, w, n = 0.5, 0.8, 30
    for _ in range(n):
        b.step(np.array([[v, w]], np.float32))
    T = n * 0.1
    xe = 5.0 + v / w * math.sin(w * T)
    ye = 5.0 + v / w * (1 - math.cos(w * T))
    assert math.hypot(b.x[0] - xe, b.y[0] - ye) < 0.5 * v * w * T * 0.1 + 1e-4


def test_reward_branches_hand_computed(orc):
    # 32 x 32 at 0.1 m, border walls; robot static at (1.6, 1.6), 4 beams:
    # every range is 1.5 m.  With d_crash = 1, d_full = 2: alpha_hug = 0.5.
    p = dict(r_max=5.0, sigma=0.0, d_crash=1.0, d_full=2.0, lam_col=10.0, lam_explore=1.0,
             lam_abs=0.1, lam_delta=1.0, kappa=0.05, u_hi=1.0, t_episode=2048)
    b = one_env(orc, bordered(32, 32), 4, 0.1, (1.6, 1.6, 0.0), **p)
    z = np.zeros((1, 2), np.float32)
    T = orc.TERM_NAMES.index
    # step 1: U 0 -> 0.3.  c = 1, I = 1, new cell (1), R_explore* = 0.5,
    # R_abs = 0, R_delta = -0.3 (negative: not scaled).  R = 0.2.
    o = b.step(z, u=np.array([0.3], np.float32))
    t = o["terms"][0]
    assert t[T("alpha_hug")] == pytest.approx(0.5, abs=1e-6)
    assert t[T("dcells")] == 1.0 and t[T("I")] == 1.0
    assert t[T("r_explore")] == pytest.approx(0.5, abs=1e-6)
    assert t[T("r_abs")] == 0.0
    assert t[T("r_delta")] == pytest.approx(-0.3, abs=1e-7)
    assert t[T("R")] == pytest.approx(0.2, abs=2e-6)
    assert o["reward_comp"][0] == pytest.approx(0.2, abs=2e-6)
    # step 2: U 0.3 -> 0.2.  c = 0.49, iota = 1, I = 1; revisit after 1 step:
    # dcells = 0.5/2048.  R_abs = 0.03 e^0.3, R_delta = 0.1 e^0.3 > 0 -> x0.5.
    o = b.step(z, u=np.array([0.2], np.float32))
    t = o["terms"][0]
    e03 = 1.3498588075760032
    assert t[T("dcells")] == pytest.approx(0.5 / 2048, rel=1e-12)
    assert t[T("I")] == pytest.approx(1.0, abs=1e-7)
    assert t[T("r_abs")] == pytest.approx(0.03 * e03, rel=1e-6)
    assert t[T("r_delta")] == pytest.approx(0.05 * e03, rel=2e-6)
    assert t[T("R")] == pytest.approx(0.5 * 0.5 / 2048 - 0.03 * e03 + 0.05 * e03, rel=2e-6)
    # step 3: U 0.2 -> 0.2: iota = 0 and R_delta = 0; c = 0.64 so I = 0.64.
    o = b.step(z, u=np.array([0.2], np.float32))
    t = o["terms"][0]
    assert t[T("I")] == pytest.approx(0.64, rel=1e-6)
    assert t[T("r_delta")] == 0.0
    # step 4: U 0.2 -> 1.7 then 5: U_prev >= U_hi gives c = 0, so I = iota.
    b.step(z, u=np.array([1.7], np.float32))
    o = b.step(z, u=np.array([1.69], np.float32))
    t = o["terms"][0]
    iota = min(max(np.float32(1.7) - np.float32(1.69), 0) / 0.05, 1.0)
    assert t[T("I")] == pytest.approx(iota, rel=1e-5)
    assert t[T("collision")] == 0.0


def test_collision_terminates_and_resets(orc):
    # robot 0.12 m from the wall: true d_min < d_crash = 0.15 -> R = -lam_col
    occ = bordered(32, 32)
    spawn = np.array([[[1.6, 1.6, 0.0], [0.22, 1.6, 0.0]]], np.float32)
    inp = synth.custom_2d([occ], [16], 0.1, spawn)
    b = orc.OracleBatch2D(inp, r_max=5.0, sigma=0.0, lam_col=7.0)
    b.x[0], b.y[0] = np.float32(0.22), np.float32(1.6)
    o = b.step(np.zeros((1, 2), np.float32))
    assert o["terms"][0, orc.TERM_NAMES.index("collision")] == 1.0
    assert o["reward_comp"][0] == -7.0 and b.done[0] == 1
    assert b.belief.min() < 0
    # the next step resets: spawn[1 % 2] = (0.22, 1.6) again, map cleared first
    o2 = b.step(np.zeros((1, 2), np.float32))
    assert b.ep[0] == 1 and b.t[0] == 1
    # after a reset the first step sees the all-unknown map again
    N = 32 * 32
    assert o2["terms"][0, 0] == pytest.approx(N * LN2 - o2["terms"][0, 11], abs=1e-9)


def test_episode_truncation(orc):
    b = one_env(orc, bordered(32, 32), 4, 0.1, (1.6, 1.6, 0.0), r_max=5.0, t_episode=3)
    z = np.zeros((1, 2), np.float32)
    for k in range(3):
        b.step(z)
    assert b.done[0] == 1
    b.step(z)
    assert b.t[0] == 1 and b.ep[0] == 1


def test_observation_layout_and_padding(orc):
    inp = synth.custom_2d([bordered(20, 20), bordered(24, 16)], [6, 3], 0.1,
                          np.array([[[1.0, 1.0, 0.2]] * 2, [[1.2, 0.8, -0.4]] * 2], np.float32))
    b = orc.OracleBatch2D(inp, r_max=5.0)
    o = b.step(np.zeros((2, 2), np.float32), u=np.array([0.25, 0.5], np.float32))
    assert o["obs"].shape == (2, 8)
    np.testing.assert_array_equal(o["obs"][0, :6], o["z"][0, :6])
    np.testing.assert_array_equal(o["obs"][1, :3], o["z"][1, :3])
    assert np.all(o["obs"][1, 3:6] == np.float32(5.0))
    assert o["obs"][0, 6] == np.float32(0.2) and o["obs"][0, 7] == np.float32(0.25)
    assert o["obs"][1, 6] == np.float32(-0.4) and o["obs"][1, 7] == np.float32(0.5)


def test_threads_over_envs_change_no_result(orc):
    """The CPU baseline spreads the step's independent envs over threads:
    every output and state must equal the serial step's (the fixed-lag mode
    included, whose scan matcher keeps its scores per call)."""
    inp = synth.uneven(E=12, sides=(64, 96), beams=(45, 90), seed=31)
    acts = synth.random_actions(4, 12, 5)
    u = synth.random_uncertainty(4, 12, 6)
    runs = []
    for th in (1, 4):
        orc.set_threads(th)
        try:
            for mode in (0, 2):
                ob = orc.OracleBatch2D(inp, r_max=4.0, sigma=0.01, u_mode=mode)
                outs = [ob.step(acts[s], u[s], counts=True) for s in range(4)]
                runs.append((th, mode, ob.belief.copy(), ob.x.copy(), outs[-1]))
        finally:
            orc.set_threads(1)
    for (t1, m1, b1, x1, o1), (t4, m4, b4, x4, o4) in zip(runs[:2], runs[2:]):
        assert m1 == m4
        np.testing.assert_array_equal(b1, b4)
        np.testing.assert_array_equal(x1, x4)
        for k in ("z", "terms", "obs", "cnt_h", "cnt_m", "ray_cells"):
            np.testing.assert_array_equal(o1[k], o4[k])


def test_nonfinite_actions_take_the_clamp_bounds(orc):
    """Host-side fault injection: Eq. 4 bounds the action, and the clamp takes
    a NaN to the non-NaN bound (C99 fmax/fmin return the other operand):
    v = NaN -> 0, w = NaN -> -w_max; +-Inf -> the nearer bound."""
    occ = bordered(200, 200)
    b = one_env(orc, occ, 4, 0.1, (5.0, 5.0, 0.0), r_max=2.0)
    b.step(np.array([[np.nan, 0.0]], np.float32))
    assert b.x[0] == np.float32(5.0) and b.y[0] == np.float32(5.0) and b.th[0] == 0.0
    b.step(np.array([[0.0, np.nan]], np.float32))
    assert b.x[0] == np.float32(5.0) and b.th[0] == pytest.approx(-0.1, abs=1e-7)
    b = one_env(orc, occ, 4, 0.1, (5.0, 5.0, 0.0), r_max=2.0)
    b.step(np.array([[np.inf, np.inf]], np.float32))
    assert b.x[0] == pytest.approx(5.05, abs=1e-6) and b.th[0] == pytest.approx(0.1, abs=1e-7)
    b.step(np.array([[-np.inf, -np.inf]], np.float32))
    assert b.x[0] == pytest.approx(5.05, abs=1e-6) and b.th[0] == pytest.approx(0.0, abs=1e-7)
    assert np.all(np.isfinite(b.belief)) and int(np.abs(b.belief).max()) <= 3584
