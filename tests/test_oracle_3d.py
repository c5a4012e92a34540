"""Pins of the oracle's 3-D voxel variant.

* The 3-D traversal against an exact-rational classification of every voxel
  (entry key < exit key, ties ordered Z, then Y, then X) on small volumes,
  plus invariants (6-connected, |di|+|dj|+|dk|+1 voxels);
* a level beam (Dz = 0) visits exactly the 2-D oracle's cells in its layer;
* a beam pointing down at elevation el from height z_s hits the top of the
  floor layer at the analytic distance (z_s - res) / sin(-el);
* an all-unknown volume has entropy N ln 2; one step from it gains dH > 0.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2603_25834_gb300 import synth
from tests.test_oracle_walk import NEG_INF, POS_INF

TYPE = {2: 0, 1: 1, 0: 2}   # axis -> tie type: Z first (0), then Y (1), then X (2)


def axis_keys3(o, d, cell, c0, typ):
    if d == 0:
        return (NEG_INF, POS_INF) if cell == c0 else None
    if d > 0:
        if cell < c0:
            return None
        enter = NEG_INF if cell == c0 else ((Fr(cell) - o) / d, typ)
        return enter, ((Fr(cell + 1) - o) / d, typ)
    if cell > c0:
        return None
    enter = NEG_INF if cell == c0 else ((Fr(cell + 1) - o) / d, typ)
    return enter, ((Fr(cell) - o) / d, typ)


def brute_path3(P, D, T, dims):
    o = [Fr(p, 1 << 16) for p in P]
    d = [Fr(x, 1 << 30) for x in D]
    c0 = [math.floor(x) for x in o]
    Tf = Fr(T, 1 << 16)
    W, H, Dd = dims
    on = []
    for k in range(-1, Dd + 1):
        kz = axis_keys3(o[2], d[2], k, c0[2], TYPE[2])
        if kz is None:
            continue
        for j in range(-1, H + 1):
            ky = axis_keys3(o[1], d[1], j, c0[1], TYPE[1])
            if ky is None:
                continue
            for i in range(-1, W + 1):
                kx = axis_keys3(o[0], d[0], i, c0[0], TYPE[0])
                if kx is None:
                    continue
                enter = max(kx[0], ky[0], kz[0])
                exit_ = min(kx[1], ky[1], kz[1])
                if enter < exit_ and enter[0] <= Tf:
                    on.append((enter, i, j, k))
    on.sort()
    cells, left = [], False
    for _, i, j, k in on:
        if 0 <= i < W and 0 <= j < H and 0 <= k < Dd:
            assert not left
            cells.append((k * H + j) * W + i)
        else:
            left = True
    return cells, left


def random_rays3(rng, n, dims):
    W, H, Dd = dims
    out = []
    for _ in range(n):
        kind = rng.integers(0, 5)
        P = [int(rng.integers(0, s << 16)) for s in dims]
        if kind == 1:
            P = [p & ~0xFFFF for p in P]                 # origin on a voxel corner
        if kind == 2:                                    # axis-parallel
            ax = rng.integers(0, 3)
            D = [0, 0, 0]
            D[ax] = int(rng.choice([-1, 1])) * (1 << 30)
        elif kind == 3:                                  # exact diagonal through corners
            D = [int(rng.choice([-1, 1])) * 619925131 for _ in range(3)]
            P = [(p & ~0xFFFF) | 0x8000 for p in P]
        else:
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            D = [int(round(x * (1 << 30))) for x in v]
        T = int(rng.integers(0, sum(dims) << 16))
        out.append((P, D, T))
    return out


@pytest.mark.parametrize("dims", [(5, 4, 3), (6, 6, 2), (1, 7, 5)])
def test_walk3d_matches_exact_rational_brute_force(orc, dims):
    rng = np.random.default_rng(sum(dims))
    for P, D, T in random_rays3(rng, 80, dims):
        cells, en, ea, left = orc.walk3d(*P, *D, T, *dims)
        ref, ref_left = brute_path3(P, D, T, dims)
        assert list(cells) == ref, (P, D, T)
        assert left == ref_left
        ijk = [(int(c) % dims[0], (int(c) // dims[0]) % dims[1], int(c) // (dims[0] * dims[1]))
               for c in cells]
        for a, b in zip(ijk, ijk[1:]):
            assert sum(abs(x - y) for x, y in zip(a, b)) == 1
        if not left and cells.size:
            assert len(cells) == sum(abs(x - y) for x, y in zip(ijk[-1], ijk[0])) + 1


def test_level_beam_reduces_to_2d_walk(orc):
    rng = np.random.default_rng(1)
    W, H, Dd = 20, 17, 6
    for _ in range(60):
        P = [int(rng.integers(0, W << 16)), int(rng.integers(0, H << 16)),
             (int(rng.integers(0, Dd)) << 16) | 0x4000]
        a = rng.uniform(-math.pi, math.pi)
        D = [int(round(math.cos(a) * (1 << 30))), int(round(math.sin(a) * (1 << 30))), 0]
        T = int(rng.integers(0, 30 << 16))
        c3, _, _, l3 = orc.walk3d(*P, *D, T, W, H, Dd)
        c2, _, _, l2 = orc.walk2d(P[0], P[1], D[0], D[1], T, W, H)
        k = P[2] >> 16
        assert list(c3) == [k * W * H + c for c in c2] and l3 == l2


def test_floor_range_is_analytic(orc):
    # empty world except the floor layer; one ring pointing 15 degrees down
    W = H = 64
    Dd = 16
    occ = np.zeros((Dd, H, W), np.uint8)
    occ[0] = 1
    inp = synth.Batch3DInputs(np.array([W], np.int32), np.array([H], np.int32),
                              np.array([Dd], np.int32), np.array([8], np.int32), 0.1,
                              occ.reshape(-1), np.array([0, occ.size], np.int64),
                              np.array([[[3.2, 3.2, 0.0]] * 2], np.float32))
    el = -15.0 * math.pi / 180
    b = orc.OracleBatch3D(inp, n_rings=1, el_min=el, el_max=el, sensor_z=0.5, sigma=0.0, r_max=20.0)
    o = b.step(np.zeros((1, 2), np.float32), counts=True)
    expect = (0.5 - 0.1) / math.sin(-el)
    np.testing.assert_allclose(o["z"][0], expect, atol=2e-5)
    assert o["hit"][0].all()
    # the hits land in the floor layer, the misses above it
    assert o["cnt_h"][: W * H].sum() == 8 and o["cnt_h"][W * H:].sum() == 0


def test_entropy_and_update_invariants_3d(orc):
    inp = synth.voxel_batch(E=2, W=32, H=32, D=8, n_az=24, K=2)
    b = orc.OracleBatch3D(inp, n_rings=4, r_max=4.0, sigma=0.01)
    N = int(inp.map_off[1] - inp.map_off[0])
    o = b.step(np.zeros((2, 2), np.float32), counts=True)
    assert o["terms"][0, 0] == pytest.approx(N * math.log(2) - o["terms"][0, 11], abs=1e-8)
    assert o["terms"][:, 0].min() > 0
    assert np.abs(b.belief).max() <= 3584
    touched = (o["cnt_h"] + o["cnt_m"]) > 0
    assert np.all(b.belief[~touched] == 0)
    assert o["ray_cells"].sum() == int((o["cnt_h"] + o["cnt_m"]).sum())
