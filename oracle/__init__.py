"""CPU oracle of the batched Active-SLAM step -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this package.  It shares no code with the CUDA path
(paper_2603_25834_gb300); both only take inputs from the seeded generators in
paper_2603_25834_gb300.synth.

The arithmetic lives in plain C (aslam_oracle.c, soft_range_oracle.c,
raycast3d_oracle.c, slam_oracle.c); this module compiles them with gcc and marshals numpy
arrays through ctypes.  Every function cites the passage it follows in the
C sources.  Pins: tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SOURCES = ["aslam_oracle.c", "soft_range_oracle.c", "raycast3d_oracle.c", "slam_oracle.c"]
_LIB = None
_LOCK = threading.Lock()

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    """Compile the oracle sources into oracle/_build/liborc.so (gcc, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liborc.so")
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(out) >= newest:
            return out
    tmp = out + ".tmp%d" % os.getpid()
    # OpenMP only spreads orc_step2d's independent envs over threads (the
    # all-cores CPU baseline); without it the same code runs serially
    r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", *srcs, "-o", tmp, "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.check_call(["gcc", *CFLAGS, *srcs, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def set_threads(n: int) -> int:
    """Threads orc_step2d spreads its envs over; returns the count in effect
    (1 when the oracle was built without OpenMP)."""
    L = lib()
    n = max(1, int(n)) if L.orc_openmp() else 1
    L.orc_set_threads(n)
    return n


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = C.CDLL(build())
            _declare(_LIB)
    return _LIB


P = C.c_void_p


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OrcCfg(C.Structure):
    _fields_ = [
        ("n_envs", C.c_int32), ("b_max", C.c_int32), ("n_spawn", C.c_int32),
        ("hit_q", C.c_int32), ("miss_q", C.c_int32), ("clamp_q", C.c_int32),
        ("t_episode", C.c_int32), ("pad0", C.c_int32), ("seed", C.c_uint64),
        ("res", C.c_float), ("r_max", C.c_float), ("fov", C.c_float), ("sigma", C.c_float),
        ("dt", C.c_float), ("v_max", C.c_float), ("w_max", C.c_float), ("d_crash", C.c_float),
        ("d_full", C.c_float), ("visit_cell", C.c_float), ("r_min", C.c_float),
        ("dec_scale", C.c_float),
        ("logodds_scale", C.c_double),
        ("lam_col", C.c_double), ("lam_explore", C.c_double), ("lam_abs", C.c_double),
        ("lam_delta", C.c_double), ("kappa", C.c_double), ("u_hi", C.c_double),
        ("map_w", P), ("map_h", P), ("n_beams", P), ("map_off", P), ("visit_off", P),
        ("env_id", P),
        ("u_mode", C.c_int32), ("uq_samples", C.c_int32), ("uq_step", C.c_float),
        ("uq_range_sigma", C.c_float), ("uq_odo", C.c_float * 3), ("uq_prior", C.c_float * 3),
        ("uq_u_scale", C.c_float),
        ("slam_window", C.c_int32), ("slam_iters", C.c_int32), ("csm_n_xy", C.c_int32),
        ("csm_n_th", C.c_int32), ("csm_sep", C.c_int32), ("csm_dth", C.c_float),
        ("slam_meas_info", C.c_float * 3), ("slam_prior_info", C.c_float * 3),
        ("slam_weighted", C.c_int32), ("slam_gn_iters", C.c_int32),
    ]


class OrcState(C.Structure):
    _fields_ = [("gt", P), ("belief", P), ("x", P), ("y", P), ("th", P), ("u_prev", P),
                ("t", P), ("g", P), ("ep", P), ("done", P), ("visit", P), ("spawn", P),
                ("sigma", P), ("win_x", P), ("win_odo", P), ("win_meas", P), ("win_minfo", P),
                ("win_n", P), ("slam_match", P), ("slam_pose", P), ("slam_scores", P),
                ("slam_upd_w", P), ("slam_gn_pose", P)]


class OrcOut(C.Structure):
    _fields_ = [("z", P), ("z_true", P), ("hit", P), ("cnt_h", P), ("cnt_m", P),
                ("terms", P), ("reward_ent", P), ("reward_comp", P), ("obs", P),
                ("ray_cells", P), ("gt_cells", P)]


class OrcCfg3D(C.Structure):
    _fields_ = [
        ("n_envs", C.c_int32), ("n_rings", C.c_int32), ("n_az", C.c_int32), ("n_spawn", C.c_int32),
        ("hit_q", C.c_int32), ("miss_q", C.c_int32), ("clamp_q", C.c_int32), ("t_episode", C.c_int32),
        ("seed", C.c_uint64),
        ("res", C.c_float), ("r_max", C.c_float), ("sigma", C.c_float), ("dt", C.c_float),
        ("v_max", C.c_float), ("w_max", C.c_float), ("d_crash", C.c_float), ("d_full", C.c_float),
        ("visit_cell", C.c_float), ("sensor_z", C.c_float), ("r_min", C.c_float),
        ("dec_scale", C.c_float),
        ("el_min", C.c_double), ("el_max", C.c_double), ("logodds_scale", C.c_double),
        ("lam_col", C.c_double), ("lam_explore", C.c_double), ("lam_abs", C.c_double),
        ("lam_delta", C.c_double), ("kappa", C.c_double), ("u_hi", C.c_double),
        ("map_w", P), ("map_h", P), ("map_d", P), ("map_off", P), ("visit_off", P),
        ("env_id", P),
    ]


class OrcOut3D(C.Structure):
    _fields_ = [("z", P), ("z_true", P), ("hit", P), ("cnt_h", P), ("cnt_m", P), ("terms", P),
                ("obs", P), ("ray_cells", P), ("gt_cells", P)]


class OrcSoftCfg(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("B", C.c_int32), ("K", C.c_int32),
                ("res", C.c_double), ("ds", C.c_double), ("fov", C.c_double)]


N_TERMS = 12
TERM_NAMES = ["dH", "dcells", "I", "alpha_hug", "r_explore", "r_abs", "r_delta", "R",
              "collision", "dmin_meas", "dmin_true", "H"]


def _declare(L):
    L.orc_sincosf.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.orc_cos2pi.argtypes = [C.c_float]
    L.orc_cos2pi.restype = C.c_float
    L.orc_logf.argtypes = [C.c_float]
    L.orc_logf.restype = C.c_float
    L.orc_philox4x32_10.argtypes = [P, P, P]
    L.orc_gauss.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
    L.orc_gauss.restype = C.c_float
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_openmp.restype = C.c_int
    L.orc_walk2d.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                             C.c_int32, C.c_int32, P, P, P, C.c_int, C.POINTER(C.c_int)]
    L.orc_walk2d.restype = C.c_int
    L.orc_beam_dirs.argtypes = [C.c_int, C.c_double, P, P]
    L.orc_ray_setup.argtypes = [C.c_float] * 7 + [C.POINTER(C.c_int32)] * 4
    L.orc_measured_range.argtypes = [C.c_float] * 6
    L.orc_measured_range.restype = C.c_float
    L.orc_slam_correct_pose.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_double,
                                        C.c_int32, C.c_float, C.c_double, C.c_int32, C.c_int32,
                                        C.c_float, P, P, C.c_int, P]
    L.orc_slam_correct_pose.restype = None
    L.orc_csm.argtypes = [P, C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_int32, C.c_double,
                          P, C.c_float, C.c_float, C.c_float, C.c_int32, C.c_int32, C.c_int32,
                          C.c_float, P, P, P]
    L.orc_fixed_lag_gn.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, P, P]
    L.orc_fixed_lag_gn.restype = C.c_int
    L.orc_bridge_alpha.argtypes = [C.c_int64, C.c_int64]
    L.orc_bridge_alpha.restype = C.c_float
    L.orc_bridge_u.argtypes = [C.c_float, C.c_float, C.c_float]
    L.orc_bridge_u.restype = C.c_float
    L.orc_cell_entropy.argtypes = [C.c_double]
    L.orc_cell_entropy.restype = C.c_double
    L.orc_map_entropy.argtypes = [P, C.c_int64, C.c_double]
    L.orc_map_entropy.restype = C.c_double
    L.orc_visit_dims.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_float,
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.orc_step2d.argtypes = [C.POINTER(OrcCfg), C.POINTER(OrcState), P, P, C.POINTER(OrcOut)]
    L.orc_step2d.restype = C.c_int
    L.orc_soft_ranges.argtypes = [C.POINTER(OrcSoftCfg), P, P, C.c_int, P, P, P, P]
    L.orc_walk3d.argtypes = [C.c_int32] * 6 + [C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                               P, P, P, C.c_int, C.POINTER(C.c_int)]
    L.orc_walk3d.restype = C.c_int
    L.orc_beams3d.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, P, P, P, P]
    L.orc_step3d.argtypes = [C.POINTER(OrcCfg3D), C.POINTER(OrcState), P, P, C.POINTER(OrcOut3D)]
    L.orc_step3d.restype = C.c_int
    L.orc_soft_jacobian.argtypes = [C.POINTER(OrcSoftCfg), P, P, C.c_int, P, P]
    L.orc_gn_batch.argtypes = [C.POINTER(OrcSoftCfg), P, P, P, C.c_int, C.c_int, C.c_double, P, P]


# ---------------------------------------------------------------- scalar helpers
def sincosf(x):
    s, c = C.c_float(), C.c_float()
    lib().orc_sincosf(C.c_float(x), C.byref(s), C.byref(c))
    return s.value, c.value


def cos2pi(u):
    return lib().orc_cos2pi(C.c_float(u))


def logf(u):
    return lib().orc_logf(C.c_float(u))


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def gauss(seed, env, step, beam):
    return lib().orc_gauss(C.c_uint64(seed), env, step, beam)


def walk2d(Px, Py, Dx, Dy, T, W, H):
    """Visited in-map cells (flat j*W+i), entry numerators/denominators, left-map flag."""
    cap = W + H + 8
    cells = np.zeros(cap, dtype=np.int64)
    en = np.zeros(cap, dtype=np.int64)
    ea = np.zeros(cap, dtype=np.int64)
    left = C.c_int()
    n = lib().orc_walk2d(Px, Py, Dx, Dy, T, W, H, _ptr(cells), _ptr(en), _ptr(ea), cap,
                         C.byref(left))
    return cells[:n].copy(), en[:n].copy(), ea[:n].copy(), bool(left.value)


def beam_dirs(B, fov):
    cb = np.zeros(max(B, 1), dtype=np.float32)
    sb = np.zeros(max(B, 1), dtype=np.float32)
    lib().orc_beam_dirs(B, C.c_double(fov), _ptr(cb), _ptr(sb))
    return cb[:B], sb[:B]


def ray_setup(x, y, c, s, cb, sb, res):
    o = [C.c_int32() for _ in range(4)]
    lib().orc_ray_setup(x, y, c, s, cb, sb, res, *[C.byref(v) for v in o])
    return tuple(v.value for v in o)


def cell_entropy(l):
    return lib().orc_cell_entropy(C.c_double(l))


def map_entropy(L, scale):
    L = np.ascontiguousarray(L, dtype=np.int16)
    return lib().orc_map_entropy(_ptr(L), L.size, C.c_double(scale))


def visit_dims(W, H, res, vc):
    a, b = C.c_int32(), C.c_int32()
    lib().orc_visit_dims(W, H, C.c_float(res), C.c_float(vc), C.byref(a), C.byref(b))
    return a.value, b.value


def dec_scale(decimals):
    """10^decimals as an fp32 scale of the range rounding (0: no rounding)."""
    return 0.0 if decimals is None or decimals < 0 else float(np.float32(10.0 ** int(decimals)))


def measured_range(z_true, g, sigma, r_min, r_max, decimals=-1):
    return lib().orc_measured_range(C.c_float(z_true), C.c_float(g), C.c_float(sigma),
                                    C.c_float(r_min), C.c_float(r_max),
                                    C.c_float(dec_scale(decimals)))


def slam_correct(belief, res, fov, z, pose, iters=2, K=64, ds=0.0, logodds_scale=1.0 / 1024.0,
                 n_xy=5, n_th=5, dth=0.01):
    """Scan-to-map Gauss-Newton correction of a matched pose on the soft
    range model of an int16 belief [H, W] (orc_slam_correct_pose)."""
    Lb = np.ascontiguousarray(belief, dtype=np.int16)
    H, W = Lb.shape
    zz = np.ascontiguousarray(z, dtype=np.float32).ravel()
    pm = np.ascontiguousarray(pose, dtype=np.float32).ravel()
    out = np.zeros(3, np.float32)
    lib().orc_slam_correct_pose(_ptr(Lb), W, H, zz.size, res, fov, K, ds, logodds_scale, n_xy,
                                n_th, dth, _ptr(zz), _ptr(pm), int(iters), _ptr(out))
    return out


def csm(belief, res, r_max, fov, z, pose, n_xy=5, n_th=5, sep=1, dth=0.01):
    """Correlative scan match of one env: belief int16 [H, W], ranges z [B],
    predicted pose (x, y, th).  Returns (pose_out [3] fp32, match [3] fp32,
    scores [3] int64 = best, second, best index)."""
    Lb = np.ascontiguousarray(belief, dtype=np.int16)
    H, W = Lb.shape
    zz = np.ascontiguousarray(z, dtype=np.float32)
    pose = np.asarray(pose, np.float32)
    po = np.zeros(3, np.float32)
    mt = np.zeros(3, np.float32)
    sc = np.zeros(3, np.int64)
    lib().orc_csm(_ptr(Lb), W, H, res, r_max, zz.size, fov, _ptr(zz), float(pose[0]),
                  float(pose[1]), float(pose[2]), n_xy, n_th, sep, dth, _ptr(po), _ptr(mt),
                  _ptr(sc))
    return po, mt, sc


def fixed_lag_gn(x, odo, meas, meas_info, prior, prior_info, odo_info, iters=3):
    """One env's window (fp64): returns (x [L, 3], cov_last [3, 3], status)."""
    x = np.array(x, np.float64).reshape(-1, 3).copy()
    L = x.shape[0]
    odo = np.ascontiguousarray(np.asarray(odo, np.float64).reshape(max(L - 1, 0), 3))
    args = [np.ascontiguousarray(np.asarray(v, np.float64)) for v in
            (meas, meas_info, prior, prior_info, odo_info)]
    cov = np.zeros(9, np.float64)
    rc = lib().orc_fixed_lag_gn(L, int(iters), _ptr(x), _ptr(odo), *[_ptr(a) for a in args],
                                _ptr(cov))
    return x, cov.reshape(3, 3), rc


def bridge_u(u_old, u_new, t, t_bridge):
    """Bridged uncertainty (fp32 arrays) at fine-tuning step t."""
    a = lib().orc_bridge_alpha(int(t), int(t_bridge))
    uo = np.asarray(u_old, np.float32).ravel()
    un = np.asarray(u_new, np.float32).ravel()
    return np.array([lib().orc_bridge_u(float(x), float(y), a) for x, y in zip(uo, un)],
                    np.float32)


# ---------------------------------------------------------------- batched 2-D step
DEFAULTS = dict(r_max=5.0, r_min=0.0, decimals=-1, fov=0.0, sigma=0.0, dt=0.1, v_max=0.5, w_max=1.0,
                hit_q=870, miss_q=-410, clamp_q=3584, logodds_scale=1.0 / 1024.0,
                t_episode=2048, d_crash=0.15, d_full=0.5, visit_cell=0.5,
                lam_col=10.0, lam_explore=1.0, lam_abs=0.1, lam_delta=1.0, kappa=0.05,
                u_hi=1.0, seed=20260325, u_mode=0, uq_samples=64, uq_step=0.0,
                uq_range_sigma=0.01, uq_odo=(0.01, 0.01, 0.01), uq_prior=(0.01, 0.01, 0.01),
                uq_u_scale=0.0, slam_window=8, slam_iters=3, csm_n_xy=5, csm_n_th=5, csm_sep=1,
                csm_dth=0.01, slam_meas_info=(4e4, 4e4, 1e6), slam_prior_info=(1e4, 1e4, 1e4),
                slam_weighted=0, slam_gn_iters=0)


class OracleBatch2D:
    """Owns the numpy state of E environments and steps them with orc_step2d."""

    def __init__(self, inputs, env_ids=None, **params):
        p = dict(DEFAULTS)
        p.update(params)
        self.p = p
        self.inp = inputs
        E = inputs.n_envs
        self.E = E
        self.map_w = np.ascontiguousarray(inputs.map_w, dtype=np.int32)
        self.map_h = np.ascontiguousarray(inputs.map_h, dtype=np.int32)
        self.n_beams = np.ascontiguousarray(inputs.n_beams, dtype=np.int32)
        self.map_off = np.ascontiguousarray(inputs.map_off, dtype=np.int64)
        self.b_max = int(self.n_beams.max()) if E else 0
        dims = [visit_dims(int(w), int(h), inputs.res, p["visit_cell"])
                for w, h in zip(self.map_w, self.map_h)]
        self.visit_dims = dims
        self.visit_off = np.zeros(E + 1, dtype=np.int64)
        self.visit_off[1:] = np.cumsum([a * b for a, b in dims])
        self.gt = np.ascontiguousarray(inputs.gt, dtype=np.uint8)
        self.spawn = np.ascontiguousarray(inputs.spawn, dtype=np.float32)
        self.env_ids = None if env_ids is None else np.ascontiguousarray(env_ids, dtype=np.int32)
        ncell = int(self.map_off[-1])
        self.belief = np.zeros(ncell, dtype=np.int16)
        self.x = self.spawn[:, 0, 0].copy()
        self.y = self.spawn[:, 0, 1].copy()
        self.th = self.spawn[:, 0, 2].copy()
        self.u_prev = np.zeros(E, dtype=np.float32)
        self.t = np.zeros(E, dtype=np.int32)
        self.g = np.zeros(E, dtype=np.int32)
        self.ep = np.zeros(E, dtype=np.int32)
        self.done = np.zeros(E, dtype=np.uint8)
        self.visit = np.full(int(self.visit_off[-1]), -1, dtype=np.int32)
        # pose covariance (xx, xy, xt, yy, yt, tt): the prior until the first scan
        pr = np.asarray(p["uq_prior"], np.float32).astype(np.float64)
        self.sigma = np.zeros((E, 6), np.float64)
        self.sigma[:, 0], self.sigma[:, 3], self.sigma[:, 5] = pr[0] ** 2, pr[1] ** 2, pr[2] ** 2
        Lw = int(p["slam_window"])
        self.win_x = np.zeros((E, Lw, 3), np.float32)
        self.win_odo = np.zeros((E, Lw, 3), np.float32)
        self.win_meas = np.zeros((E, Lw, 3), np.float32)
        self.win_minfo = np.zeros((E, Lw, 3), np.float32)
        self.win_n = np.zeros(E, np.int32)
        self.slam_match = np.zeros((E, 3), np.float32)
        self.slam_pose = np.zeros((E, 3), np.float32)
        self.slam_scores = np.zeros((E, 3), np.int64)
        self.slam_upd_w = np.zeros(E, np.float32)
        self.slam_gn_pose = np.zeros((E, 3), np.float32)
        self.cfg = OrcCfg(
            n_envs=E, b_max=self.b_max, n_spawn=self.spawn.shape[1],
            hit_q=p["hit_q"], miss_q=p["miss_q"], clamp_q=p["clamp_q"],
            t_episode=p["t_episode"], pad0=0, seed=p["seed"], res=inputs.res,
            r_max=p["r_max"], r_min=p["r_min"], dec_scale=dec_scale(p["decimals"]),
            fov=p["fov"], sigma=p["sigma"], dt=p["dt"], v_max=p["v_max"],
            w_max=p["w_max"], d_crash=p["d_crash"], d_full=p["d_full"],
            visit_cell=p["visit_cell"], logodds_scale=p["logodds_scale"],
            lam_col=p["lam_col"], lam_explore=p["lam_explore"], lam_abs=p["lam_abs"],
            lam_delta=p["lam_delta"], kappa=p["kappa"], u_hi=p["u_hi"],
            map_w=_ptr(self.map_w), map_h=_ptr(self.map_h), n_beams=_ptr(self.n_beams),
            map_off=_ptr(self.map_off), visit_off=_ptr(self.visit_off),
            env_id=_ptr(self.env_ids), u_mode=p["u_mode"], uq_samples=p["uq_samples"],
            uq_step=p["uq_step"], uq_range_sigma=p["uq_range_sigma"],
            uq_odo=(C.c_float * 3)(*p["uq_odo"]), uq_prior=(C.c_float * 3)(*p["uq_prior"]),
            uq_u_scale=p["uq_u_scale"], slam_window=p["slam_window"], slam_iters=p["slam_iters"],
            csm_n_xy=p["csm_n_xy"], csm_n_th=p["csm_n_th"], csm_sep=p["csm_sep"],
            csm_dth=p["csm_dth"], slam_meas_info=(C.c_float * 3)(*p["slam_meas_info"]),
            slam_prior_info=(C.c_float * 3)(*p["slam_prior_info"]),
            slam_weighted=p["slam_weighted"], slam_gn_iters=p["slam_gn_iters"])

    def _state(self):
        return OrcState(gt=_ptr(self.gt), belief=_ptr(self.belief), x=_ptr(self.x),
                        y=_ptr(self.y), th=_ptr(self.th), u_prev=_ptr(self.u_prev),
                        t=_ptr(self.t), g=_ptr(self.g), ep=_ptr(self.ep), done=_ptr(self.done),
                        visit=_ptr(self.visit), spawn=_ptr(self.spawn), sigma=_ptr(self.sigma),
                        win_x=_ptr(self.win_x), win_odo=_ptr(self.win_odo),
                        win_meas=_ptr(self.win_meas), win_minfo=_ptr(self.win_minfo),
                        win_n=_ptr(self.win_n), slam_match=_ptr(self.slam_match),
                        slam_pose=_ptr(self.slam_pose), slam_scores=_ptr(self.slam_scores),
                        slam_upd_w=_ptr(self.slam_upd_w), slam_gn_pose=_ptr(self.slam_gn_pose))

    def step(self, actions, u=None, counts=False):
        """One step for all envs; returns a dict of this step's outputs."""
        E, Bm = self.E, self.b_max
        a = np.ascontiguousarray(actions, dtype=np.float32).reshape(E, 2)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float32).reshape(E)
        ncell = int(self.map_off[-1])
        o = dict(z=np.zeros((E, Bm), np.float32), z_true=np.zeros((E, Bm), np.float32),
                 hit=np.zeros((E, Bm), np.uint8), terms=np.zeros((E, N_TERMS), np.float64),
                 reward_ent=np.zeros(E, np.float32), reward_comp=np.zeros(E, np.float32),
                 obs=np.zeros((E, Bm + 2), np.float32), ray_cells=np.zeros(E, np.int64),
                 gt_cells=np.zeros(E, np.int64))
        if counts:
            o["cnt_h"] = np.zeros(ncell, np.int32)
            o["cnt_m"] = np.zeros(ncell, np.int32)
        out = OrcOut(z=_ptr(o["z"]), z_true=_ptr(o["z_true"]), hit=_ptr(o["hit"]),
                     cnt_h=_ptr(o.get("cnt_h")), cnt_m=_ptr(o.get("cnt_m")),
                     terms=_ptr(o["terms"]), reward_ent=_ptr(o["reward_ent"]),
                     reward_comp=_ptr(o["reward_comp"]), obs=_ptr(o["obs"]),
                     ray_cells=_ptr(o["ray_cells"]), gt_cells=_ptr(o["gt_cells"]))
        st = self._state()
        rc = lib().orc_step2d(C.byref(self.cfg), C.byref(st), _ptr(a), _ptr(uu), C.byref(out))
        if rc != 0:
            raise RuntimeError("orc_step2d failed (%d)" % rc)
        return o

    def env_belief(self, e):
        a, b = int(self.map_off[e]), int(self.map_off[e + 1])
        return self.belief[a:b].reshape(int(self.map_h[e]), int(self.map_w[e]))


# ---------------------------------------------------------------- soft range / GN
def soft_cfg(W, H, B, K=64, res=0.05, ds=0.05, fov=0.0):
    return OrcSoftCfg(W=W, H=H, B=B, K=K, res=res, ds=ds, fov=fov)


def soft_ranges(cfg, L, pose, gr=None, grad_pose=False, grad_map=False):
    """Soft ranges [E, B] (fp64) of fp32 log-odds L [E, H, W] at poses [E, 3];
    optionally the adjoints of sum(gr * r) w.r.t. pose and L."""
    L = np.ascontiguousarray(L, dtype=np.float32)
    E = L.shape[0]
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(E, 3)
    r = np.zeros((E, cfg.B), np.float64)
    gp = np.zeros((E, 3), np.float64) if grad_pose else None
    gm = np.zeros(L.shape, np.float64) if grad_map else None
    g = None if gr is None else np.ascontiguousarray(gr, dtype=np.float64).reshape(E, cfg.B)
    lib().orc_soft_ranges(C.byref(cfg), _ptr(L), _ptr(pose), E, _ptr(g), _ptr(r), _ptr(gp), _ptr(gm))
    return r, gp, gm


def gn(cfg, L, pose_in, z, iters=5, mu=1e-6):
    """Gauss-Newton pose correction: final poses [E, 3] and damped normal matrices [E, 3, 3]."""
    L = np.ascontiguousarray(L, dtype=np.float32)
    E = L.shape[0]
    pin = np.ascontiguousarray(pose_in, dtype=np.float64).reshape(E, 3)
    zz = np.ascontiguousarray(z, dtype=np.float32).reshape(E, cfg.B)
    pout = np.zeros((E, 3), np.float64)
    A = np.zeros((E, 9), np.float64)
    lib().orc_gn_batch(C.byref(cfg), _ptr(L), _ptr(pin), _ptr(zz), E, iters, C.c_double(mu),
                       _ptr(pout), _ptr(A))
    return pout, A.reshape(E, 3, 3)


def soft_jacobian(cfg, L, pose):
    """Ranges [E, B] and per-beam Jacobians [E, B, 3] (fp64)."""
    L = np.ascontiguousarray(L, dtype=np.float32)
    E = L.shape[0]
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(E, 3)
    r = np.zeros((E, cfg.B), np.float64)
    J = np.zeros((E, cfg.B, 3), np.float64)
    lib().orc_soft_jacobian(C.byref(cfg), _ptr(L), _ptr(pose), E, _ptr(r), _ptr(J))
    return r, J


# ---------------------------------------------------------------- 3-D variant
def walk3d(Px, Py, Pz, Dx, Dy, Dz, T, W, H, D):
    cap = W + H + D + 8
    cells = np.zeros(cap, dtype=np.int64)
    en = np.zeros(cap, dtype=np.int64)
    ea = np.zeros(cap, dtype=np.int64)
    left = C.c_int()
    n = lib().orc_walk3d(Px, Py, Pz, Dx, Dy, Dz, T, W, H, D, _ptr(cells), _ptr(en), _ptr(ea), cap,
                         C.byref(left))
    return cells[:n].copy(), en[:n].copy(), ea[:n].copy(), bool(left.value)


DEFAULTS3D = dict(r_max=20.0, r_min=0.0, decimals=-1, sigma=0.0, dt=0.1, v_max=0.5, w_max=1.0, hit_q=870, miss_q=-410,
                  clamp_q=3584, logodds_scale=1.0 / 1024.0, t_episode=2048, d_crash=0.15,
                  d_full=0.5, visit_cell=0.5, sensor_z=0.5, el_min=-15.0 * np.pi / 180,
                  el_max=15.0 * np.pi / 180, lam_col=10.0, lam_explore=1.0, lam_abs=0.1,
                  lam_delta=1.0, kappa=0.05, u_hi=1.0, seed=20260325)


class OracleBatch3D:
    """Numpy state of E voxel environments stepped by orc_step3d."""

    def __init__(self, inputs, n_rings=16, env_ids=None, **params):
        p = dict(DEFAULTS3D)
        p.update(params)
        # the elevation limits and sensor height are fp32 quantities of the
        # sensor description: both implementations start from the same floats
        for k in ("el_min", "el_max", "sensor_z"):
            p[k] = float(np.float32(p[k]))
        self.p = p
        self.inp = inputs
        E = inputs.n_envs
        self.E = E
        self.R, self.A = int(n_rings), int(inputs.n_beams[0])
        assert np.all(inputs.n_beams == self.A)
        self.B = self.R * self.A
        self.map_w = np.ascontiguousarray(inputs.map_w, dtype=np.int32)
        self.map_h = np.ascontiguousarray(inputs.map_h, dtype=np.int32)
        self.map_d = np.ascontiguousarray(inputs.map_d, dtype=np.int32)
        self.map_off = np.ascontiguousarray(inputs.map_off, dtype=np.int64)
        dims = [visit_dims(int(w), int(h), inputs.res, p["visit_cell"])
                for w, h in zip(self.map_w, self.map_h)]
        self.visit_off = np.zeros(E + 1, dtype=np.int64)
        self.visit_off[1:] = np.cumsum([a * b for a, b in dims])
        self.gt = np.ascontiguousarray(inputs.gt, dtype=np.uint8)
        self.spawn = np.ascontiguousarray(inputs.spawn, dtype=np.float32)
        self.belief = np.zeros(int(self.map_off[-1]), dtype=np.int16)
        self.x = self.spawn[:, 0, 0].copy()
        self.y = self.spawn[:, 0, 1].copy()
        self.th = self.spawn[:, 0, 2].copy()
        self.u_prev = np.zeros(E, np.float32)
        self.t = np.zeros(E, np.int32)
        self.g = np.zeros(E, np.int32)
        self.ep = np.zeros(E, np.int32)
        self.done = np.zeros(E, np.uint8)
        self.visit = np.full(int(self.visit_off[-1]), -1, np.int32)
        self.env_ids = None if env_ids is None else np.ascontiguousarray(env_ids, dtype=np.int32)
        self.cfg = OrcCfg3D(
            n_envs=E, n_rings=self.R, n_az=self.A, n_spawn=self.spawn.shape[1],
            hit_q=p["hit_q"], miss_q=p["miss_q"], clamp_q=p["clamp_q"], t_episode=p["t_episode"],
            seed=p["seed"], res=inputs.res, r_max=p["r_max"], r_min=p["r_min"],
            dec_scale=dec_scale(p["decimals"]), sigma=p["sigma"], dt=p["dt"],
            v_max=p["v_max"], w_max=p["w_max"], d_crash=p["d_crash"], d_full=p["d_full"],
            visit_cell=p["visit_cell"], sensor_z=p["sensor_z"], el_min=p["el_min"],
            el_max=p["el_max"], logodds_scale=p["logodds_scale"], lam_col=p["lam_col"],
            lam_explore=p["lam_explore"], lam_abs=p["lam_abs"], lam_delta=p["lam_delta"],
            kappa=p["kappa"], u_hi=p["u_hi"], map_w=_ptr(self.map_w), map_h=_ptr(self.map_h),
            map_d=_ptr(self.map_d), map_off=_ptr(self.map_off), visit_off=_ptr(self.visit_off),
            env_id=_ptr(self.env_ids))

    def step(self, actions, u=None, counts=False):
        E, B = self.E, self.B
        a = np.ascontiguousarray(actions, dtype=np.float32).reshape(E, 2)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float32).reshape(E)
        n = int(self.map_off[-1])
        o = dict(z=np.zeros((E, B), np.float32), z_true=np.zeros((E, B), np.float32),
                 hit=np.zeros((E, B), np.uint8), terms=np.zeros((E, N_TERMS), np.float64),
                 obs=np.zeros((E, B + 2), np.float32), ray_cells=np.zeros(E, np.int64),
                 gt_cells=np.zeros(E, np.int64))
        if counts:
            o["cnt_h"] = np.zeros(n, np.int32)
            o["cnt_m"] = np.zeros(n, np.int32)
        out = OrcOut3D(z=_ptr(o["z"]), z_true=_ptr(o["z_true"]), hit=_ptr(o["hit"]),
                       cnt_h=_ptr(o.get("cnt_h")), cnt_m=_ptr(o.get("cnt_m")), terms=_ptr(o["terms"]),
                       obs=_ptr(o["obs"]), ray_cells=_ptr(o["ray_cells"]), gt_cells=_ptr(o["gt_cells"]))
        st = OrcState(gt=_ptr(self.gt), belief=_ptr(self.belief), x=_ptr(self.x), y=_ptr(self.y),
                      th=_ptr(self.th), u_prev=_ptr(self.u_prev), t=_ptr(self.t), g=_ptr(self.g),
                      ep=_ptr(self.ep), done=_ptr(self.done), visit=_ptr(self.visit),
                      spawn=_ptr(self.spawn))
        if lib().orc_step3d(C.byref(self.cfg), C.byref(st), _ptr(a), _ptr(uu), C.byref(out)) != 0:
            raise RuntimeError("orc_step3d failed")
        return o
