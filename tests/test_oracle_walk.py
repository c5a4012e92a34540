"""Pins of the oracle's exact grid traversal against exact-rational brute force.

The log-odds grid update of Sec. III-D touches "the cells the beam crosses";
the oracle walks them on a Q16 origin / Q30 direction with exact 128-bit
comparisons.  Here every cell of a small map (plus a ring of outside cells)
is classified with Python Fractions, with no walking at all:

  * a cell is on the path iff the key at which the ray enters it is below
    the key at which it leaves it, where a key is (ray parameter t, axis)
    with the horizontal-line (Y) crossing ordered before the vertical-line
    (X) crossing at equal t;
  * it is within range T iff its entry parameter is <= T.

Independently of that tie rule, the path must contain every cell whose open
interior the segment crosses, lie inside the cells whose closed square it
touches, and be a 4-connected staircase of |di|+|dj|+1 cells.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

NEG_INF = (Fr(-10 ** 9), -1)
POS_INF = (Fr(10 ** 9), 2)


def axis_keys(o, d, cell, c0, typ):
    """(enter_key, exit_key) of the ray along one axis for column/row `cell`."""
    if d == 0:
        return (NEG_INF, POS_INF) if cell == c0 else None
    if d > 0:
        if cell < c0:
            return None
        enter = NEG_INF if cell == c0 else ((Fr(cell) - o) / d, typ)
        exit_ = ((Fr(cell + 1) - o) / d, typ)
    else:
        if cell > c0:
            return None
        enter = NEG_INF if cell == c0 else ((Fr(cell + 1) - o) / d, typ)
        exit_ = ((Fr(cell) - o) / d, typ)
    return enter, exit_


def brute_path(Px, Py, Dx, Dy, T, W, H):
    ox, oy = Fr(Px, 1 << 16), Fr(Py, 1 << 16)
    dx, dy = Fr(Dx, 1 << 30), Fr(Dy, 1 << 30)
    Tf = Fr(T, 1 << 16)
    i0, j0 = math.floor(ox), math.floor(oy)
    on = []
    for j in range(-1, H + 1):
        ky = axis_keys(oy, dy, j, j0, 0)
        if ky is None:
            continue
        for i in range(-1, W + 1):
            kx = axis_keys(ox, dx, i, i0, 1)
            if kx is None:
                continue
            enter = max(kx[0], ky[0])
            exit_ = min(kx[1], ky[1])
            if enter < exit_ and enter[0] <= Tf:
                on.append((enter, i, j))
    on.sort()
    cells, left = [], False
    for _, i, j in on:
        if 0 <= i < W and 0 <= j < H:
            if left:
                raise AssertionError("path re-entered the map")
            cells.append(j * W + i)
        else:
            left = True
    return cells, left


def segment_cells(Px, Py, Dx, Dy, T, W, H, closed):
    ox, oy = Fr(Px, 1 << 16), Fr(Py, 1 << 16)
    dx, dy = Fr(Dx, 1 << 30), Fr(Dy, 1 << 30)
    Tf = Fr(T, 1 << 16)
    out = set()
    for j in range(H):
        for i in range(W):
            lo, hi = Fr(0), Tf
            ok = True
            for o, d, c in ((ox, dx, i), (oy, dy, j)):
                if d == 0:
                    inside = (c <= o <= c + 1) if closed else (c < o < c + 1)
                    if not inside:
                        ok = False
                    continue
                a, b = (Fr(c) - o) / d, (Fr(c + 1) - o) / d
                if a > b:
                    a, b = b, a
                lo, hi = max(lo, a), min(hi, b)
            if not ok:
                continue
            if (closed and lo <= hi) or (not closed and lo < hi):
                out.add(j * W + i)
    return out


def random_rays(rng, n, W, H):
    rays = []
    for _ in range(n):
        kind = rng.integers(0, 6)
        Px = int(rng.integers(0, W << 16))
        Py = int(rng.integers(0, H << 16))
        if kind == 1:                       # origin on a grid corner
            Px &= ~0xFFFF
            Py &= ~0xFFFF
        elif kind == 2:                     # origin on a vertical grid line
            Px &= ~0xFFFF
        if kind == 3:                       # axis-parallel
            Dx, Dy = [(1 << 30, 0), (-(1 << 30), 0), (0, 1 << 30), (0, -(1 << 30))][rng.integers(0, 4)]
        elif kind == 4:                     # exact diagonal: passes through corners
            Dx = int(rng.choice([-1, 1])) * 759250125
            Dy = int(rng.choice([-1, 1])) * 759250125
            Px = (Px & ~0xFFFF) | 0x8000
            Py = (Py & ~0xFFFF) | 0x8000
        else:
            a = rng.uniform(-math.pi, math.pi)
            Dx, Dy = int(round(math.cos(a) * (1 << 30))), int(round(math.sin(a) * (1 << 30)))
        T = int(rng.integers(0, (W + H) << 16))
        if rng.integers(0, 4) == 0:
            T = (T & ~0xFFFF) | 0x8000      # lands the endpoint on diagonal corners
        rays.append((Px, Py, Dx, Dy, T))
    return rays


@pytest.mark.parametrize("W,H", [(7, 5), (12, 12), (1, 9), (9, 1)])
def test_walk_matches_exact_rational_brute_force(orc, W, H):
    rng = np.random.default_rng(W * 100 + H)
    for (Px, Py, Dx, Dy, T) in random_rays(rng, 150, W, H):
        cells, en, ea, left = orc.walk2d(Px, Py, Dx, Dy, T, W, H)
        ref, ref_left = brute_path(Px, Py, Dx, Dy, T, W, H)
        assert list(cells) == ref, (Px, Py, Dx, Dy, T)
        assert left == ref_left


@pytest.mark.parametrize("W,H", [(10, 8), (16, 16)])
def test_walk_invariants(orc, W, H):
    rng = np.random.default_rng(7 + W)
    for (Px, Py, Dx, Dy, T) in random_rays(rng, 60, W, H):
        cells, en, ea, left = orc.walk2d(Px, Py, Dx, Dy, T, W, H)
        s = set(int(c) for c in cells)
        assert len(s) == len(cells)                       # each cell once
        inner = segment_cells(Px, Py, Dx, Dy, T, W, H, closed=False)
        outer = segment_cells(Px, Py, Dx, Dy, T, W, H, closed=True)
        if not left:
            assert inner <= s
        assert s <= outer
        ij = [(int(c) % W, int(c) // W) for c in cells]
        for a, b in zip(ij, ij[1:]):
            assert abs(a[0] - b[0]) + abs(a[1] - b[1]) == 1   # 4-connected
        if not left and cells.size:
            assert len(cells) == abs(ij[-1][0] - ij[0][0]) + abs(ij[-1][1] - ij[0][1]) + 1


def test_walk_entry_parameters_are_exact(orc):
    """The entry numerator/denominator of every cell is the crossing that entered it."""
    rng = np.random.default_rng(3)
    W = H = 12
    for (Px, Py, Dx, Dy, T) in random_rays(rng, 60, W, H):
        cells, en, ea, left = orc.walk2d(Px, Py, Dx, Dy, T, W, H)
        for k in range(1, len(cells)):
            t = Fr(int(en[k]) << 14, int(ea[k]))          # cells
            assert t <= Fr(T, 1 << 16)
            # the crossing point lies on the shared edge of the two cells
            px = Fr(Px, 1 << 16) + t * Fr(Dx, 1 << 30)
            py = Fr(Py, 1 << 16) + t * Fr(Dy, 1 << 30)
            i0, j0 = int(cells[k - 1]) % W, int(cells[k - 1]) // W
            i1, j1 = int(cells[k]) % W, int(cells[k]) // W
            if i1 != i0:
                assert px == max(i0, i1)
            else:
                assert py == max(j0, j1)


def test_axis_aligned_hand_cases(orc):
    # origin at the centre of cell (2, 3) of a 10 x 10 map, ray along +x,
    # endpoint 3.5 cells away: crossings at t = 0.5, 1.5, 2.5, 3.5 (<= T).
    Px, Py = (2 << 16) | 0x8000, (3 << 16) | 0x8000
    cells, en, ea, left = orc.walk2d(Px, Py, 1 << 30, 0, 7 << 15, 10, 10)
    assert list(cells) == [32, 33, 34, 35, 36] and not left
    # one Q16 unit shorter: the last crossing is no longer within range
    cells, *_ = orc.walk2d(Px, Py, 1 << 30, 0, (7 << 15) - 1, 10, 10)
    assert list(cells) == [32, 33, 34, 35]
    # ray along -y leaves the map after rows 3, 2, 1, 0
    cells, en, ea, left = orc.walk2d(Px, Py, 0, -(1 << 30), 20 << 16, 10, 10)
    assert list(cells) == [32, 22, 12, 2] and left
    # zero-length segment: just the origin cell
    cells, *_ = orc.walk2d(Px, Py, 1 << 30, 1 << 29, 0, 10, 10)
    assert list(cells) == [32]
    # origin outside the map: nothing
    cells, en, ea, left = orc.walk2d(-5, Py, 1 << 30, 0, 1 << 20, 10, 10)
    assert cells.size == 0 and left
