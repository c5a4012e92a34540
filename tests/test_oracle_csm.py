"""Pins of the oracle's correlative scan matching (Sec. III-D).

* A scan constructed so that, from the true pose, every endpoint lands in an
  occupied cell: the matcher started from a pose offset by whole steps
  finds the true offset exactly, with the full score (evidence 224 per beam,
  so score_norm = 224/255).
* A pure-Python brute force of the score definition on a tiny map (every
  candidate's score, the best index with its tie rule, the second best
  outside the separation, the margin).
* A corridor constant along x: candidates that differ only along x tie, so
  the second best equals the best and the margin is 0.
* An empty map and a scan without returns: all zero.
"""
import math

import numpy as np
import pytest


def beam_table(B, fov=0.0):
    a = (2 * math.pi * np.arange(B)) / B if fov <= 0 else \
        -0.5 * fov + (np.arange(B) * fov) / (B - 1)
    return np.cos(a).astype(np.float32), np.sin(a).astype(np.float32)


def endpoint_cells(orc, pose, z, cb, sb, res, k_off=0, dth=0.01):
    """Cells of the endpoints from pose, in fp32 as the definition states."""
    f = np.float32
    th = f(f(pose[2]) + f(f(k_off) * f(dth)))
    s, c = orc.sincosf(float(th))
    s, c = f(s), f(c)
    dx = f(c * cb) - f(s * sb)
    dy = f(s * cb) + f(c * sb)
    ex = f(pose[0]) + f(z * dx)
    ey = f(pose[1]) + f(z * dy)
    return np.floor(ex / f(res)).astype(int), np.floor(ey / f(res)).astype(int)


def test_recovers_a_whole_step_offset(orc):
    rng = np.random.default_rng(3)
    W = H = 160
    res = np.float32(0.05)
    B = 90
    cb, sb = beam_table(B)
    true = np.float32([4.013, 3.987, 0.31])
    z = rng.uniform(0.6, 3.0, B).astype(np.float32)
    ci, cj = endpoint_cells(orc, true, z, cb, sb, res)
    L = np.zeros((H, W), np.int16)
    L[cj, ci] = 3584
    # predicted pose off by (+2, -1) cells and +2 rotation steps
    dth = np.float32(0.01)
    pred = np.float32([true[0] + np.float32(2) * res, true[1] - res, true[2] + np.float32(2) * dth])
    po, mt, sc = orc.csm(L, float(res), 10.0, 0.0, z, pred, n_xy=4, n_th=3, sep=1, dth=float(dth))
    side = 9
    i, j, k = -2, 1, -2
    assert sc[2] == ((k + 3) * side + (j + 4)) * side + (i + 4)
    assert sc[0] == 224 * B and mt[0] == np.float32(224 / 255)
    np.testing.assert_allclose(po, true, atol=2e-6)


def brute(L, res, r_max, z, cb, sb, pose, n, m, sep, dth, orc):
    H, W = L.shape
    side = 2 * n + 1
    scores = {}
    for k in range(-m, m + 1):
        ci, cj = endpoint_cells(orc, pose, z, cb, sb, res, k, dth)
        for j in range(-n, n + 1):
            for i in range(-n, n + 1):
                s = 0
                for b in range(len(z)):
                    if not z[b] < r_max:
                        continue
                    x, y = ci[b] + i, cj[b] + j
                    if 0 <= x < W and 0 <= y < H:
                        s += min(255, max(int(L[y, x]), 0) >> 4)
                scores[((k + m) * side + (j + n)) * side + (i + n)] = s
    best_q = min(q for q, v in scores.items() if v == max(scores.values()))
    best = scores[best_q]
    ib, jb, kb = best_q % side, (best_q // side) % side, best_q // (side * side)
    second = max([v for q, v in scores.items()
                  if max(abs(q % side - ib), abs((q // side) % side - jb),
                         abs(q // (side * side) - kb)) > sep] + [0])
    return best, second, best_q


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny(orc, seed):
    rng = np.random.default_rng(seed)
    L = rng.integers(-3584, 3585, size=(12, 10)).astype(np.int16)
    B = 7
    cb, sb = beam_table(B, fov=math.pi)
    z = rng.uniform(0.05, 0.4, B).astype(np.float32)
    z[2] = np.float32(0.5)                                  # a beam without return
    pose = np.float32([0.27, 0.31, rng.uniform(-3, 3)])
    res, r_max = 0.05, 0.5
    po, mt, sc = orc.csm(L, res, r_max, math.pi, z, pose, n_xy=2, n_th=2, sep=1, dth=0.05)
    best, second, q = brute(L, np.float32(res), np.float32(r_max), z, cb, sb, pose, 2, 2, 1,
                            np.float32(0.05), orc)
    assert (sc[0], sc[1], sc[2]) == (best, second, q)
    assert mt[0] == np.float32(best / (255 * 6))
    assert mt[1] == np.float32((best - second) / best if best else 0.0)


def test_corridor_is_ambiguous_along_x(orc):
    W, H = 200, 40
    L = np.full((H, W), -3584, np.int16)
    L[:10, :] = 3584
    L[30:, :] = 3584                                         # walls below y=0.5 and above y=1.5
    B = 64
    cb, sb = beam_table(B)
    pose = np.float32([5.0, 1.0, 0.0])
    # ranges to the walls for beams that see them within 2 m, none otherwise
    ang = 2 * np.pi * np.arange(B) / B
    with np.errstate(divide="ignore"):
        d = np.where(np.sin(ang) > 0, 0.5 / np.sin(ang), -0.5 / np.sin(ang))
    z = np.where(d < 2.0, d + 0.025, 10.0).astype(np.float32)
    po, mt, sc = orc.csm(L, 0.05, 10.0, 0.0, z, pose, n_xy=3, n_th=0, sep=1, dth=0.01)
    assert sc[0] > 0 and sc[1] == sc[0] and mt[1] == 0.0 and mt[2] == 0.0


def test_empty_map_and_no_returns(orc):
    L = np.zeros((50, 50), np.int16)
    z = np.full(16, 1.0, np.float32)
    po, mt, sc = orc.csm(L, 0.05, 5.0, 0.0, z, [1.2, 1.3, 0.1], n_xy=2, n_th=1)
    assert list(sc) == [0, 0, 0] and list(mt) == [0, 0, 0]
    np.testing.assert_allclose(po, [1.2 - 0.1, 1.3 - 0.1, 0.1 - 0.01], atol=1e-6)
    L[:] = 3584
    po, mt, sc = orc.csm(L, 0.05, 5.0, 0.0, np.full(16, 5.0, np.float32), [1.2, 1.3, 0.1])
    assert list(sc) == [0, 0, 0] and mt[0] == 0.0
