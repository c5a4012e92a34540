"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds none of the method's arithmetic: it only draws worlds
(ground-truth occupancy grids standing in for the Isaac Sim scenes of
Sec. IV-A), spawn poses, action sequences (Eq. 4) and uncertainty signals
(the scalar U_t of Eq. 3, which the fixed-lag SLAM backbone of Sec. III-D
would supply).  Everything is plain numpy driven by explicit seeds, so both
implementations receive bit-identical inputs.

Grid convention: cell (i, j) covers [i*res, (i+1)*res) x [j*res, (j+1)*res),
flat index j*W + i; a ground-truth cell is occupied iff its centre lies in
a closed rectangle or disc (3-D: a closed box or a vertical cylinder).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20260325


@dataclasses.dataclass
class World2D:
    W: int
    H: int
    res: float
    occ: np.ndarray          # uint8 [H, W]


def _raster_rects_discs(W, H, res, rects, discs):
    """Occupancy by cell centre, touching only each shape's bounding box."""
    occ = np.zeros((H, W), dtype=np.uint8)

    def box(x0, y0, hx, hy):
        i0 = max(int(np.floor((x0 - hx) / res)) - 1, 0)
        i1 = min(int(np.ceil((x0 + hx) / res)) + 1, W)
        j0 = max(int(np.floor((y0 - hy) / res)) - 1, 0)
        j1 = min(int(np.ceil((y0 + hy) / res)) + 1, H)
        cx = (np.arange(i0, i1, dtype=np.float64) + 0.5) * res
        cy = (np.arange(j0, j1, dtype=np.float64) + 0.5) * res
        return i0, i1, j0, j1, cx[None, :], cy[:, None]

    for (x0, y0, w, h) in rects:
        i0, i1, j0, j1, X, Y = box(x0, y0, w / 2, h / 2)
        if i1 > i0 and j1 > j0:
            occ[j0:j1, i0:i1] |= ((np.abs(X - x0) <= w / 2) & (np.abs(Y - y0) <= h / 2)).astype(np.uint8)
    for (x0, y0, r) in discs:
        i0, i1, j0, j1, X, Y = box(x0, y0, r, r)
        if i1 > i0 and j1 > j0:
            occ[j0:j1, i0:i1] |= (((X - x0) ** 2 + (Y - y0) ** 2) <= r * r).astype(np.uint8)
    return occ


def make_world_2d(W, H, res, rng, n_rect=(8, 8), rect_side=(0.3, 1.5),
                  n_disc=(0, 0), disc_r=(0.1, 0.6), border=True) -> World2D:
    """Border walls plus random axis-aligned rectangles and discs."""
    ext_x, ext_y = W * res, H * res
    nr = int(rng.integers(n_rect[0], n_rect[1] + 1))
    nd = int(rng.integers(n_disc[0], n_disc[1] + 1))
    rects = [(rng.uniform(0, ext_x), rng.uniform(0, ext_y),
              rng.uniform(*rect_side), rng.uniform(*rect_side)) for _ in range(nr)]
    discs = [(rng.uniform(0, ext_x), rng.uniform(0, ext_y), rng.uniform(*disc_r))
             for _ in range(nd)]
    occ = _raster_rects_discs(W, H, res, rects, discs)
    if border:
        occ[0, :] = 1
        occ[-1, :] = 1
        occ[:, 0] = 1
        occ[:, -1] = 1
    return World2D(W, H, res, occ)


def spawn_poses_2d(world: World2D, K, rng, clearance=0.3, max_tries=200000):
    """K free poses (x, y, theta) with no occupied cell centre within `clearance` m."""
    W, H, res, occ = world.W, world.H, world.res, world.occ
    r = int(np.ceil(clearance / res)) + 1
    out = []
    tries = 0
    while len(out) < K:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place spawn poses with the requested clearance")
        x = rng.uniform(clearance, W * res - clearance)
        y = rng.uniform(clearance, H * res - clearance)
        ci, cj = int(x / res), int(y / res)
        i0, i1 = max(ci - r, 0), min(ci + r + 1, W)
        j0, j1 = max(cj - r, 0), min(cj + r + 1, H)
        oy, ox = np.nonzero(occ[j0:j1, i0:i1])
        if ox.size:
            d2 = ((ox + i0 + 0.5) * res - x) ** 2 + ((oy + j0 + 0.5) * res - y) ** 2
            if d2.min() < clearance * clearance:
                continue
        th = rng.uniform(-math.pi, math.pi)
        out.append((x, y, th))
    return np.asarray(out, dtype=np.float32)


@dataclasses.dataclass
class Batch2DInputs:
    """Everything a 2-D batch needs, for both the CUDA path and the oracle."""
    map_w: np.ndarray        # int32 [E]
    map_h: np.ndarray        # int32 [E]
    n_beams: np.ndarray      # int32 [E]
    res: float
    gt: np.ndarray           # uint8 [sum W*H], env e at map_off[e]
    map_off: np.ndarray      # int64 [E+1]
    spawn: np.ndarray        # float32 [E, K, 3]

    @property
    def n_envs(self):
        return int(self.map_w.shape[0])


def _pack_batch(worlds, beams, res, K, rng_spawn):
    E = len(worlds)
    map_w = np.array([w.W for w in worlds], dtype=np.int32)
    map_h = np.array([w.H for w in worlds], dtype=np.int32)
    off = np.zeros(E + 1, dtype=np.int64)
    off[1:] = np.cumsum(map_w.astype(np.int64) * map_h)
    gt = np.concatenate([w.occ.reshape(-1) for w in worlds]).astype(np.uint8)
    spawn = np.stack([spawn_poses_2d(w, K, rng_spawn[e]) for e, w in enumerate(worlds)])
    return Batch2DInputs(map_w, map_h, np.asarray(beams, dtype=np.int32), res, gt, off, spawn)


def plain_1env(seed=BASE_SEED, K=16):
    """64x64 grid at 0.1 m, border + 8 random rectangles, 90 beams (single env)."""
    rng = np.random.default_rng(seed)
    w = make_world_2d(64, 64, 0.1, rng, n_rect=(8, 8), rect_side=(0.3, 1.5))
    return _pack_batch([w], [90], 0.1, K, [np.random.default_rng(seed + 10_000_000)])


def paper_scale(E=750, W=256, B=360, seed=BASE_SEED, K=16, envs=None):
    """E envs of WxW at 0.05 m with 20-40 rectangles and 5-15 discs, B beams.
    `envs` (default all): the indices of the envs to build, e.g. one rank's
    contiguous share; env e is the same world wherever it is built."""
    worlds, rs = [], []
    for e in (range(E) if envs is None else envs):
        rng = np.random.default_rng(seed + e)
        scale = (W / 256.0) ** 2
        worlds.append(make_world_2d(
            W, W, 0.05, rng,
            n_rect=(max(1, round(20 * scale)), max(1, round(40 * scale))), rect_side=(0.2, 2.0),
            n_disc=(max(0, round(5 * scale)), max(0, round(15 * scale))), disc_r=(0.1, 0.6)))
        rs.append(np.random.default_rng(seed + 10_000_000 + e))
    return _pack_batch(worlds, [B] * len(worlds), 0.05, K, rs)


def uneven_shapes(E=4096, sides=(128, 256, 384, 512), beams=(180, 360, 720), seed=BASE_SEED):
    """Map side and beam count of each of the E envs of `uneven`."""
    pick = np.random.default_rng(seed - 1)
    side = pick.choice(np.asarray(sides), size=E)
    nb = pick.choice(np.asarray(beams), size=E)
    return side, nb


def uneven(E=4096, sides=(128, 256, 384, 512), beams=(180, 360, 720), seed=BASE_SEED, K=8,
           envs=None):
    """E envs with map side and beam count drawn uniformly from the given sets
    (`envs`: the indices to build, default all)."""
    side, nb = uneven_shapes(E, sides, beams, seed)
    envs = range(E) if envs is None else envs
    worlds, rs = [], []
    for e in envs:
        rng = np.random.default_rng(seed + e)
        s = int(side[e])
        scale = (s / 256.0) ** 2
        worlds.append(make_world_2d(
            s, s, 0.05, rng,
            n_rect=(max(1, round(20 * scale)), max(1, round(40 * scale))), rect_side=(0.2, 2.0),
            n_disc=(max(0, round(5 * scale)), max(0, round(15 * scale))), disc_r=(0.1, 0.6)))
        rs.append(np.random.default_rng(seed + 10_000_000 + e))
    return _pack_batch(worlds, [int(nb[e]) for e in envs], 0.05, K, rs)


def custom_2d(occs, beams, res, spawn):
    """Hand-made batch: explicit grids [H, W] (uint8), beams per env and spawn table."""
    E = len(occs)
    map_w = np.array([o.shape[1] for o in occs], dtype=np.int32)
    map_h = np.array([o.shape[0] for o in occs], dtype=np.int32)
    off = np.zeros(E + 1, dtype=np.int64)
    off[1:] = np.cumsum(map_w.astype(np.int64) * map_h)
    gt = np.concatenate([np.ascontiguousarray(o, dtype=np.uint8).reshape(-1) for o in occs])
    return Batch2DInputs(map_w, map_h, np.asarray(beams, dtype=np.int32), float(res), gt, off,
                         np.ascontiguousarray(spawn, dtype=np.float32))


def subset(inputs, envs):
    """The listed envs of a batch as a batch of their own (same worlds and spawns)."""
    occs, beams, spawn = [], [], []
    for e in envs:
        a, b = int(inputs.map_off[e]), int(inputs.map_off[e + 1])
        occs.append(inputs.gt[a:b].reshape(int(inputs.map_h[e]), int(inputs.map_w[e])))
        beams.append(int(inputs.n_beams[e]))
        spawn.append(inputs.spawn[e])
    return custom_2d(occs, beams, inputs.res, np.stack(spawn))


def random_actions(steps, E, seed, v_max=0.5, w_max=1.0):
    """float32 [steps, E, 2]: v ~ U[0, v_max], w ~ U[-w_max, w_max] (Eq. 4 ranges)."""
    rng = np.random.default_rng(seed)
    a = np.empty((steps, E, 2), dtype=np.float32)
    a[..., 0] = rng.uniform(0.0, v_max, size=(steps, E))
    a[..., 1] = rng.uniform(-w_max, w_max, size=(steps, E))
    return a


def random_uncertainty(steps, E, seed, lo=0.0, hi=1.5):
    """float32 [steps, E]: a bounded random walk standing in for the SLAM scalar U_t."""
    rng = np.random.default_rng(seed)
    u = np.empty((steps, E), dtype=np.float32)
    cur = rng.uniform(lo, hi, size=E)
    for s in range(steps):
        cur = np.clip(cur + rng.normal(0.0, 0.08, size=E), lo, hi)
        u[s] = cur
    return u


def logodds_maps(inputs, occupied=3.0, free=-3.0):
    """fp32 natural log-odds grids [E, H, W] of a belief that has seen the whole
    ground truth (uniform W, H): `occupied` where the world is occupied,
    `free` elsewhere.  Input for the differentiable soft raycaster."""
    E = inputs.n_envs
    W, H = int(inputs.map_w[0]), int(inputs.map_h[0])
    assert np.all(inputs.map_w == W) and np.all(inputs.map_h == H)
    occ = inputs.gt.reshape(E, H, W)
    return np.where(occ > 0, np.float32(occupied), np.float32(free)).astype(np.float32)


def perturb_poses(poses, seed, sigma=(0.05, 0.05, 0.02)):
    """poses [E, 3] plus Gaussian noise (x, y, th), float32."""
    rng = np.random.default_rng(seed)
    p = np.asarray(poses, dtype=np.float64)
    return (p + rng.normal(0.0, 1.0, p.shape) * np.asarray(sigma)).astype(np.float32)


@dataclasses.dataclass
class Batch3DInputs:
    """A batch of voxel worlds: env e is W x H x D at map_off[e], flat (k*H + j)*W + i."""
    map_w: np.ndarray
    map_h: np.ndarray
    map_d: np.ndarray
    n_beams: np.ndarray      # azimuths per ring
    res: float
    gt: np.ndarray
    map_off: np.ndarray
    spawn: np.ndarray        # [E, K, 3]

    @property
    def n_envs(self):
        return int(self.map_w.shape[0])


def make_world_3d(W, H, D, res, rng, n_box=(8, 16), box_side=(0.5, 3.0), box_h=(0.3, 3.2),
                  n_pillar=(4, 10), pillar_r=(0.1, 0.4), floor=True):
    """uint8 [D, H, W]: floor layer, boxes standing on it and full-height pillars."""
    cx = (np.arange(W) + 0.5) * res
    cy = (np.arange(H) + 0.5) * res
    cz = (np.arange(D) + 0.5) * res
    occ = np.zeros((D, H, W), np.uint8)
    for _ in range(int(rng.integers(n_box[0], n_box[1] + 1))):
        x0, y0 = rng.uniform(0, W * res), rng.uniform(0, H * res)
        sx, sy, hz = rng.uniform(*box_side), rng.uniform(*box_side), rng.uniform(*box_h)
        m2 = (np.abs(cx[None, :] - x0) <= sx / 2) & (np.abs(cy[:, None] - y0) <= sy / 2)
        occ[cz <= hz] |= m2.astype(np.uint8)
    for _ in range(int(rng.integers(n_pillar[0], n_pillar[1] + 1))):
        x0, y0, r = rng.uniform(0, W * res), rng.uniform(0, H * res), rng.uniform(*pillar_r)
        m2 = ((cx[None, :] - x0) ** 2 + (cy[:, None] - y0) ** 2) <= r * r
        occ |= m2.astype(np.uint8)[None]
    if floor:
        occ[0] = 1
    return occ


def voxel_batch(E=512, W=128, H=128, D=32, res=0.1, n_az=512, seed=BASE_SEED, K=8, clearance=0.3,
                envs=None):
    """E voxel worlds with floor, boxes and pillars (counts scaled to the floor
    area of a 128 x 128 x 0.1 m world); spawns on free columns (`envs`: the
    indices to build, default all)."""
    grids, spawns = [], []
    scale = (W * H * res * res) / (128 * 128 * 0.01)
    n_box = (int(round(8 * scale)), max(int(round(16 * scale)), 1))
    n_pillar = (int(round(4 * scale)), max(int(round(10 * scale)), 1))
    side = (0.5, max(0.6, min(3.0, 0.4 * min(W, H) * res)))
    for e in (range(E) if envs is None else envs):
        occ = make_world_3d(W, H, D, res, np.random.default_rng(seed + e), n_box=n_box,
                            box_side=side, n_pillar=n_pillar)
        grids.append(occ)
        column = World2D(W, H, res, occ[1:].max(axis=0))
        spawns.append(spawn_poses_2d(column, K, np.random.default_rng(seed + 10_000_000 + e),
                                     clearance=clearance))
    off = np.zeros(E + 1, np.int64)
    off[1:] = np.cumsum([g.size for g in grids])
    n = len(grids)
    return Batch3DInputs(np.full(n, W, np.int32), np.full(n, H, np.int32), np.full(n, D, np.int32),
                         np.full(n, n_az, np.int32), float(res),
                         np.concatenate([g.reshape(-1) for g in grids]), off, np.stack(spawns))
