"""Pins of the oracle's soft expected-range raycaster and Gauss-Newton.

Closed forms (empty map -> K*ds, solid map -> ds, a wall -> the first sample
beyond it), central finite differences of the oracle's forward model in fp64
against its adjoint (pose and map), an invariance (a map constant along x
has zero x-gradient), a 90-degree rotation of map and pose, and Gauss-Newton
recovering a perturbed pose (Sec. III-D, Eq. 5-6).
"""
import math

import numpy as np
import pytest

from paper_2603_25834_gb300 import synth


def test_empty_and_solid_maps(orc):
    cfg = orc.soft_cfg(64, 64, 12)
    r, gp, gm = orc.soft_ranges(cfg, np.full((1, 64, 64), -40.0, np.float32), [[1.6, 1.6, 0.3]],
                                grad_pose=True, grad_map=True)
    np.testing.assert_allclose(r, 64 * 0.05, atol=1e-12)
    assert np.abs(gp).max() < 1e-12
    r, _, _ = orc.soft_ranges(cfg, np.full((1, 64, 64), 40.0, np.float32), [[1.6, 1.6, 0.3]])
    np.testing.assert_allclose(r, 0.05, atol=1e-12)


def test_wall_gives_first_sample_beyond_it(orc):
    # wall from cell column 40 on (x >= 2.0 m); beam 0 along +x from a point
    # 1 mm right of the centre of cell 10.
    L = np.full((1, 32, 64), -30.0, np.float32)
    L[:, :, 40:] = 30.0
    x0 = 10.5 * 0.05 + 0.001
    cfg = orc.soft_cfg(64, 32, 4)
    r, _, _ = orc.soft_ranges(cfg, L, [[x0, 16.5 * 0.05, 0.0]])
    # samples sit 1 mm right of cell centres; the first one inside the wall
    # band is 1 mm right of the centre of cell 40
    expect = (40.5 * 0.05 + 0.001) - x0
    assert r[0, 0] == pytest.approx(expect, abs=1e-9)
    # beam 2 (-x) reaches no wall within 64 samples... it leaves the map and
    # clamp-to-edge keeps the free value -> no return
    assert r[0, 2] == pytest.approx(3.2, abs=1e-9)


def textured_map(W, H, seed):
    rng = np.random.default_rng(seed)
    L = rng.normal(0.0, 1.2, size=(H, W))
    # a few solid blocks so that beams return
    for _ in range(6):
        i, j = rng.integers(4, W - 8), rng.integers(4, H - 8)
        L[j:j + 4, i:i + 4] = 3.0
    return L.astype(np.float32)[None]


def kink_free(cfg, pose, h_pos, h_th):
    """Beams whose samples stay clear of the bilinear kinks under +-h."""
    x, y, th = pose
    ok = []
    for b in range(cfg.B):
        phi = th + 2 * math.pi * b / cfg.B
        s = (np.arange(cfg.K) + 1) * cfg.ds
        u = (x + s * math.cos(phi)) / cfg.res - 0.5
        v = (y + s * math.sin(phi)) / cfg.res - 0.5
        margin = (h_pos + s * h_th) / cfg.res + 1e-9
        du = np.abs(u - np.round(u))
        dv = np.abs(v - np.round(v))
        ok.append(bool(np.all(du > margin) and np.all(dv > margin)))
    return np.array(ok)


def test_pose_adjoint_matches_central_differences(orc):
    W = H = 96
    L = textured_map(W, H, 3)
    cfg = orc.soft_cfg(W, H, 72)
    pose = np.array([2.41, 2.37, 0.43])
    h = 1e-5
    ok = kink_free(cfg, pose, h, h)
    assert ok.sum() > 20
    _, gp_all, _ = orc.soft_ranges(cfg, L, [pose], grad_pose=True)
    # per-beam gradients from one-hot upstream weights
    for b in np.nonzero(ok)[0][:24]:
        gr = np.zeros((1, cfg.B)); gr[0, b] = 1.0
        _, gp, _ = orc.soft_ranges(cfg, L, [pose], gr=gr, grad_pose=True)
        for d in range(3):
            e = np.zeros(3); e[d] = h
            rp, _, _ = orc.soft_ranges(cfg, L, [pose + e])
            rm, _, _ = orc.soft_ranges(cfg, L, [pose - e])
            fd = (rp[0, b] - rm[0, b]) / (2 * h)
            assert gp[0, d] == pytest.approx(fd, rel=1e-5, abs=1e-6), (b, d)


def test_map_adjoint_matches_central_differences(orc):
    W = H = 48
    L = textured_map(W, H, 5)
    cfg = orc.soft_cfg(W, H, 16, K=40)
    pose = np.array([1.21, 1.13, -0.7])
    rng = np.random.default_rng(2)
    gr = rng.normal(size=(1, cfg.B))
    _, _, gm = orc.soft_ranges(cfg, L, [pose], gr=gr, grad_map=True)
    cells = list(zip(*np.nonzero(np.abs(gm[0]) > 1e-4)))
    assert len(cells) > 30
    h = 1e-3
    for (j, i) in [cells[k] for k in rng.choice(len(cells), 25, replace=False)] + [(0, 0), (47, 47)]:
        Lp = L.copy(); Lp[0, j, i] += h
        Lm = L.copy(); Lm[0, j, i] -= h
        fp = (gr * orc.soft_ranges(cfg, Lp, [pose])[0]).sum()
        fm = (gr * orc.soft_ranges(cfg, Lm, [pose])[0]).sum()
        fd = (fp - fm) / np.float64(np.float32(L[0, j, i] + h) - np.float32(L[0, j, i] - h))
        assert gm[0, j, i] == pytest.approx(fd, rel=2e-4, abs=1e-7), (j, i)


def test_map_constant_along_x_has_zero_x_gradient(orc):
    W = H = 64
    L = np.repeat(np.linspace(-3, 3, H, dtype=np.float32)[:, None], W, axis=1)[None]
    cfg = orc.soft_cfg(W, H, 36)
    _, gp, _ = orc.soft_ranges(cfg, L, [[1.57, 1.13, 0.2]], grad_pose=True)
    assert abs(gp[0, 0]) < 1e-12
    assert abs(gp[0, 1]) > 1e-3


def test_rotating_map_and_pose_permutes_ranges(orc):
    W = H = 80
    L = textured_map(W, H, 9)
    cfg = orc.soft_cfg(W, H, 40)
    x, y, th = 1.93, 2.21, 0.37
    r, _, _ = orc.soft_ranges(cfg, L, [[x, y, th]])
    # rotate the grid by +90 degrees about its centre: new (i', j') = (W-1-j, i)
    Lr = np.empty_like(L[0])
    for j in range(H):
        for i in range(W):
            Lr[i, W - 1 - j] = L[0, j, i]
    c = W * 0.05 / 2
    xr, yr = c - (y - c), c + (x - c)
    rr, _, _ = orc.soft_ranges(cfg, Lr[None], [[xr, yr, th + math.pi / 2]])
    # beam b of the rotated robot points where beam b of the original did
    np.testing.assert_allclose(rr[0], r[0], atol=1e-9)


def test_gauss_newton_recovers_pose(orc):
    """Eq. 5: from N(0, 5 cm, 0.02 rad) perturbations, 5 GN steps on a
    world-like map bring most poses within 1 mm and cut the mean error."""
    inp = synth.paper_scale(E=4, W=128, B=90, seed=13)
    L = synth.logodds_maps(inp)
    cfg = orc.soft_cfg(128, 128, 90)
    rng_seed = 4
    errs0, errs = [], []
    for e in range(4):
        true = inp.spawn[e, :4].astype(np.float64)
        for t in true:
            z, _, _ = orc.soft_ranges(cfg, L[e:e + 1], [t])
            start = synth.perturb_poses(t[None], rng_seed)[0].astype(np.float64)
            rng_seed += 1
            pose, A = orc.gn(cfg, L[e:e + 1], [start], z.astype(np.float32), iters=5)
            errs0.append(np.abs(start - t))
            errs.append(np.abs(pose[0] - t))
            assert np.allclose(A[0], A[0].T) and np.all(np.linalg.eigvalsh(A[0]) > 0)
            # the true pose is a fixed point
            p2, _ = orc.gn(cfg, L[e:e + 1], [t], z.astype(np.float32), iters=5)
            assert np.abs(p2[0] - t).max() < 1e-5
    errs0, errs = np.array(errs0), np.array(errs)
    assert np.mean(np.all(errs < 1e-3, axis=1)) >= 0.75
    assert errs.mean() < errs0.mean() / 5
