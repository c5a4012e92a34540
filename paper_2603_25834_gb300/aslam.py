"""Thin ctypes binding of libaslam (include/aslam.h): argument marshalling only.

Every step of the environment runs in the library's CUDA kernels; PyTorch
only provides device memory (the workspace and I/O tensors) and streams.
There is no CPU fallback: if the library cannot be built or loaded, or no
CUDA device is present, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_LIB = None

P = C.c_void_p

ASLAM_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "workspace error",
          4: "reserved", 5: "invalid state", 6: "unsupported",
          7: "device-side check failed"}
FLAG_DEBUG = 0x1
FLAG_CHECKS = 0x2
REWARD_ENTROPY = 0
REWARD_COMPOSITE = 1
U_CALLER = 0
U_SCANMATCH = 1
U_FIXEDLAG = 2
N_TERMS = 12
TERM_NAMES = ["dH", "dcells", "I", "alpha_hug", "r_explore", "r_abs", "r_delta", "R",
              "collision", "dmin_meas", "dmin_true", "H"]
CONFIG_VERSION = 2


class AslamError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libaslam: %s (%s)" % (msg, STATUS.get(status, status)))
        self.status = status


class AslamConfig(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("version", C.c_uint32),
        ("n_envs", C.c_int32), ("dims", C.c_int32), ("n_spawn", C.c_int32),
        ("reward_mode", C.c_int32),
        ("h_map_w", P), ("h_map_h", P), ("h_n_beams", P),
        ("res_m", C.c_float), ("r_max_m", C.c_float), ("fov_rad", C.c_float),
        ("noise_sigma_m", C.c_float), ("dt_s", C.c_float), ("v_max", C.c_float),
        ("w_max", C.c_float), ("d_crash", C.c_float), ("d_full", C.c_float),
        ("visit_cell_m", C.c_float),
        ("l_hit_q", C.c_int32), ("l_miss_q", C.c_int32), ("l_clamp_q", C.c_int32),
        ("t_episode", C.c_int32), ("logodds_scale", C.c_float), ("threads_per_cta", C.c_int32),
        ("lam_col", C.c_double), ("lam_explore", C.c_double), ("lam_abs", C.c_double),
        ("lam_delta", C.c_double), ("kappa", C.c_double), ("u_hi", C.c_double),
        ("seed", C.c_uint64), ("flags", C.c_int32), ("window_cells", C.c_int32),
        ("h_map_d", P), ("n_rings", C.c_int32), ("sensor_z_m", C.c_float),
        ("elev_min_rad", C.c_float), ("elev_max_rad", C.c_float), ("env_base", C.c_int32),
        ("r_min_m", C.c_float), ("range_decimals", C.c_int32),
        ("u_mode", C.c_int32), ("uq_samples", C.c_int32), ("uq_step_m", C.c_float),
        ("uq_range_sigma_m", C.c_float), ("uq_odo_sigma", C.c_float * 3),
        ("uq_prior_sigma", C.c_float * 3), ("uq_u_scale", C.c_float),
        ("slam_window", C.c_int32), ("slam_iters", C.c_int32), ("csm_n_xy", C.c_int32),
        ("csm_n_th", C.c_int32), ("csm_sep", C.c_int32), ("csm_dth_rad", C.c_float),
        ("slam_meas_info", C.c_float * 3), ("slam_prior_info", C.c_float * 3),
        ("slam_weighted_update", C.c_int32), ("slam_gn_iters", C.c_int32),
    ]


class AslamStatePtrs(C.Structure):
    _fields_ = [("x", P), ("y", P), ("th", P), ("u_prev", P), ("t", P), ("g", P), ("ep", P),
                ("done", P), ("belief", P), ("z", P), ("z_true", P), ("hit", P), ("counts", P),
                ("ray_cells", P), ("gt_cells", P), ("terms", P), ("h_map_off", P),
                ("h_ray_off", P), ("b_max", C.c_int32), ("pose_cov", P), ("slam_window", P),
                ("slam_count", P), ("slam_match", P), ("slam_scores", P), ("slam_match_pose", P),
                ("slam_gn_pose", P)]


class AslamCsmConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("n_xy", C.c_int32), ("n_th", C.c_int32),
                ("sep", C.c_int32), ("dth_rad", C.c_float)]


class AslamFlgnConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("n_envs", C.c_int32), ("window", C.c_int32),
                ("iters", C.c_int32), ("odo_info", C.c_float * 3), ("u_scale", C.c_float)]


class AslamSoftConfig(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("n_envs", C.c_int32), ("map_w", C.c_int32),
                ("map_h", C.c_int32), ("n_beams", C.c_int32), ("n_samples", C.c_int32),
                ("res_m", C.c_float), ("sample_step_m", C.c_float), ("fov_rad", C.c_float),
                ("gn_damping", C.c_float), ("range_sigma_m", C.c_float)]


EXPORTS = {
    "aslam_config_init": ([C.POINTER(AslamConfig)], C.c_int),
    "aslam_workspace_bytes": ([C.POINTER(AslamConfig), C.POINTER(C.c_size_t)], C.c_int),
    "aslam_create_batch": ([C.POINTER(AslamConfig), P, C.c_size_t, P, P, P, P,
                            C.POINTER(P)], C.c_int),
    "aslam_step": ([P, P, P, P], C.c_int),
    "aslam_step_fused": ([P, P, P, P, P, P], C.c_int),
    "aslam_step_host": ([P, P, P, P, P, P], C.c_int),
    "aslam_reward": ([P, P, P], C.c_int),
    "aslam_reward_terms": ([P, P, P], C.c_int),
    "aslam_observe": ([P, P, P], C.c_int),
    "aslam_reset": ([P, P, P], C.c_int),
    "aslam_get_state": ([P, C.POINTER(AslamStatePtrs)], C.c_int),
    "aslam_sync_status": ([P, P], C.c_int),
    "aslam_capture_graph": ([P, P, P, P, P, P], C.c_int),
    "aslam_graph_step": ([P, P], C.c_int),
    "aslam_autotune": ([P, P, P], C.c_int),
    "aslam_state_bytes": ([P, C.POINTER(C.c_size_t)], C.c_int),
    "aslam_save_state": ([P, P, C.c_size_t, P], C.c_int),
    "aslam_load_state": ([P, P, C.c_size_t, P], C.c_int),
    "aslam_bridge_u": ([P, P, P, C.c_int64, C.c_int64, P, P, P], C.c_int),
    "aslam_csm_config_init": ([C.POINTER(AslamCsmConfig)], C.c_int),
    "aslam_flgn_config_init": ([C.POINTER(AslamFlgnConfig)], C.c_int),
    "aslam_fixed_lag_gn": ([C.POINTER(AslamFlgnConfig), P, P, P, P, P, P, P, P, P, P], C.c_int),
    "aslam_csm": ([P, C.POINTER(AslamCsmConfig), P, P, P, P, P, P], C.c_int),
    "aslam_profile_begin": ([P, C.c_int32], C.c_int),
    "aslam_profile_end": ([P, P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
    "aslam_kernel_name": ([P, C.c_int32], C.c_char_p),
    "aslam_destroy_batch": ([P], None),
    "aslam_status_string": ([C.c_int], C.c_char_p),
    "aslam_last_error": ([P], C.c_char_p),
    "aslam_debug_detmath": ([P, P, C.c_int32, P, P, P, P, C.c_uint64, P, P], C.c_int),
    "aslam_scan_update_noalloc": ([C.POINTER(AslamConfig), P, P, P, P, P, P, P], C.c_int),
    "aslam_soft_config_init": ([C.POINTER(AslamSoftConfig)], C.c_int),
    "aslam_soft_range_fwd": ([C.POINTER(AslamSoftConfig), P, P, P, P], C.c_int),
    "aslam_soft_range_jac": ([C.POINTER(AslamSoftConfig), P, P, P, P, P], C.c_int),
    "aslam_soft_range_bwd": ([C.POINTER(AslamSoftConfig), P, P, P, P, P, P], C.c_int),
    "aslam_gn_correct": ([C.POINTER(AslamSoftConfig), P, P, P, C.c_int32, P, P, P, P], C.c_int),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libaslam.so (building it in-tree first when it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise AslamError(2, "libaslam.so is not built")
    lib = C.CDLL(_build.LIB)
    for name, (args, res) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _check(rc, batch_handle=None):
    if rc != ASLAM_OK:
        msg = _LIB.aslam_last_error(batch_handle)
        raise AslamError(rc, msg.decode() if msg else "error")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise AslamError(1, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise AslamError(1, "expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(t):
    if t is None:
        return None
    if t.is_cuda:
        raise AslamError(1, "expected a host (CPU) tensor")
    if not t.is_contiguous() or t.dtype != torch.float32:
        raise AslamError(1, "expected a contiguous float32 tensor")
    return C.c_void_p(t.data_ptr())


def config_defaults() -> AslamConfig:
    lib = load()
    c = AslamConfig()
    _check(lib.aslam_config_init(C.byref(c)))
    return c


_FLOAT_KEYS = {"res_m", "r_max_m", "fov_rad", "noise_sigma_m", "dt_s", "v_max", "w_max",
               "sensor_z_m", "elev_min_rad", "elev_max_rad", "r_min_m", "uq_step_m",
               "uq_range_sigma_m", "uq_u_scale", "csm_dth_rad",
               "d_crash", "d_full", "visit_cell_m", "logodds_scale", "lam_col", "lam_explore",
               "lam_abs", "lam_delta", "kappa", "u_hi"}


class Batch2D:
    """A batch of environments stepped by libaslam on the current CUDA device:
    planar grids (synth.Batch2DInputs) or voxel volumes (synth.Batch3DInputs,
    then `n_rings` and the elevation / sensor-height fields apply)."""

    def __init__(self, inputs, device="cuda", **cfg):
        if not torch.cuda.is_available():
            raise AslamError(2, "no CUDA device")
        lib = load()
        self.lib = lib
        self.device = torch.device(device)
        self.inputs = inputs
        E = inputs.n_envs
        self.E = E
        self._w = np.ascontiguousarray(inputs.map_w, dtype=np.int32)
        self._h = np.ascontiguousarray(inputs.map_h, dtype=np.int32)
        self._b = np.ascontiguousarray(inputs.n_beams, dtype=np.int32)
        c = config_defaults()
        c.n_envs = E
        c.dims = 2
        c.n_spawn = int(inputs.spawn.shape[1])
        c.res_m = float(inputs.res)
        c.h_map_w = self._w.ctypes.data_as(P)
        c.h_map_h = self._h.ctypes.data_as(P)
        c.h_n_beams = self._b.ctypes.data_as(P)
        self.dims = 3 if hasattr(inputs, "map_d") else 2
        if self.dims == 3:
            self._d = np.ascontiguousarray(inputs.map_d, dtype=np.int32)
            c.dims = 3
            c.h_map_d = self._d.ctypes.data_as(P)
            c.n_rings = 16
            c.sensor_z_m = 0.5
            c.elev_min_rad = -15.0 * np.pi / 180
            c.elev_max_rad = 15.0 * np.pi / 180
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise AslamError(1, "unknown config field %s" % k)
            if isinstance(v, (tuple, list, np.ndarray)):
                setattr(c, k, (C.c_float * len(v))(*[float(q) for q in v]))
            else:
                setattr(c, k, float(v) if k in _FLOAT_KEYS else int(v))
        self.cfg = c
        nbytes = C.c_size_t()
        _check(lib.aslam_workspace_bytes(C.byref(c), C.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        gt = torch.from_numpy(np.ascontiguousarray(inputs.gt, dtype=np.uint8)).to(self.device)
        spawn = torch.from_numpy(np.ascontiguousarray(inputs.spawn, dtype=np.float32)).to(self.device)
        self._gt_off = np.ascontiguousarray(inputs.map_off, dtype=np.int64)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.aslam_create_batch(C.byref(c), _dptr(self.workspace), nbytes.value,
                                        _dptr(gt), self._gt_off.ctypes.data_as(P), _dptr(spawn),
                                        _stream(), C.byref(h))
        _check(rc)
        self.handle = h
        sp = AslamStatePtrs()
        _check(lib.aslam_get_state(h, C.byref(sp)), h)
        self._sp = sp
        self.b_max = int(sp.b_max)
        self.map_off = np.ctypeslib.as_array(C.cast(sp.h_map_off, C.POINTER(C.c_int64)),
                                             shape=(E + 1,)).copy()
        self.ray_off = np.ctypeslib.as_array(C.cast(sp.h_ray_off, C.POINTER(C.c_int64)),
                                             shape=(E + 1,)).copy()
        self._graph_bufs = None

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.aslam_destroy_batch(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ views
    def _view(self, ptr, n, dtype):
        if not ptr:
            return None
        base = self.workspace.data_ptr()
        off = int(ptr) - base
        nb = n * torch.empty((), dtype=dtype).element_size()
        return self.workspace[off:off + nb].view(dtype)

    def state(self):
        sp, E = self._sp, self.E
        cells = int(self.map_off[-1])
        rays = max(int(self.ray_off[-1]), 1)
        return dict(
            x=self._view(sp.x, E, torch.float32), y=self._view(sp.y, E, torch.float32),
            th=self._view(sp.th, E, torch.float32), u_prev=self._view(sp.u_prev, E, torch.float32),
            t=self._view(sp.t, E, torch.int32), g=self._view(sp.g, E, torch.int32),
            ep=self._view(sp.ep, E, torch.int32), done=self._view(sp.done, E, torch.int32),
            belief=self._view(sp.belief, cells, torch.int16),
            z=self._view(sp.z, rays, torch.float32),
            z_true=self._view(sp.z_true, rays, torch.float32),
            hit=self._view(sp.hit, rays, torch.uint8),
            counts=self._view(sp.counts, cells, torch.int32),
            ray_cells=self._view(sp.ray_cells, E, torch.int64),
            gt_cells=self._view(sp.gt_cells, E, torch.int64),
            terms=self._view(sp.terms, E * N_TERMS, torch.float32).view(E, N_TERMS),
            pose_cov=(self._view(sp.pose_cov, 6 * E, torch.float64).view(E, 6)
                      if sp.pose_cov else None),
            slam_window=(self._view(sp.slam_window, 3 * E * self.cfg.slam_window, torch.float32)
                         .view(E, self.cfg.slam_window, 3) if sp.slam_window else None),
            slam_count=self._view(sp.slam_count, E, torch.int32) if sp.slam_count else None,
            slam_match=(self._view(sp.slam_match, 3 * E, torch.float32).view(E, 3)
                        if sp.slam_match else None),
            slam_scores=(self._view(sp.slam_scores, 3 * E, torch.int64).view(E, 3)
                         if sp.slam_scores else None),
            slam_match_pose=(self._view(sp.slam_match_pose, 3 * E, torch.float32).view(E, 3)
                             if sp.slam_match_pose else None),
            slam_gn_pose=(self._view(sp.slam_gn_pose, 3 * E, torch.float32).view(E, 3)
                          if sp.slam_gn_pose else None))

    def env_belief(self, e):
        st = self.state()["belief"]
        a = int(self.map_off[e])
        W, H = int(self._w[e]), int(self._h[e])
        if self.dims == 3:
            D = int(self._d[e])
            return st[a:a + W * H * D].view(D, H, W)
        return st[a:a + W * H].view(H, W)

    # ------------------------------------------------------------------ calls
    def step(self, actions, u=None, stream=None):
        _check(self.lib.aslam_step(self.handle, _dptr(actions), _dptr(u), _stream(stream)),
               self.handle)

    def step_fused(self, actions, u=None, reward=None, obs=None, stream=None):
        _check(self.lib.aslam_step_fused(self.handle, _dptr(actions), _dptr(u), _dptr(reward),
                                         _dptr(obs), _stream(stream)), self.handle)

    def step_host(self, actions, u=None, reward=None, obs=None, stream=None):
        """One step from and to host tensors (page-locked for asynchronous
        copies); the outputs are valid after the stream is synchronised."""
        _check(self.lib.aslam_step_host(self.handle, _hptr(actions), _hptr(u), _hptr(reward),
                                        _hptr(obs), _stream(stream)), self.handle)

    def reward(self, out=None, stream=None):
        if out is None:
            out = torch.empty(self.E, dtype=torch.float32, device=self.device)
        _check(self.lib.aslam_reward(self.handle, _dptr(out), _stream(stream)), self.handle)
        return out

    def reward_terms(self, out=None, stream=None):
        if out is None:
            out = torch.empty(self.E, N_TERMS, dtype=torch.float32, device=self.device)
        _check(self.lib.aslam_reward_terms(self.handle, _dptr(out), _stream(stream)), self.handle)
        return out

    def observe(self, out=None, stream=None):
        if out is None:
            out = torch.empty(self.E, self.b_max + 2, dtype=torch.float32, device=self.device)
        _check(self.lib.aslam_observe(self.handle, _dptr(out), _stream(stream)), self.handle)
        return out

    def reset(self, mask=None, stream=None):
        _check(self.lib.aslam_reset(self.handle, _dptr(mask), _stream(stream)), self.handle)

    def sync_status(self, stream=None):
        _check(self.lib.aslam_sync_status(self.handle, _stream(stream)), self.handle)

    def capture_graph(self, actions, u=None, reward=None, obs=None, stream=None):
        self._graph_bufs = (actions, u, reward, obs)
        _check(self.lib.aslam_capture_graph(self.handle, _dptr(actions), _dptr(u), _dptr(reward),
                                            _dptr(obs), _stream(stream)), self.handle)

    def graph_step(self, stream=None):
        _check(self.lib.aslam_graph_step(self.handle, _stream(stream)), self.handle)

    def autotune(self, stream=None):
        best = (C.c_int32 * 2)()
        _check(self.lib.aslam_autotune(self.handle, best, _stream(stream)), self.handle)
        return int(best[0]), int(best[1])

    def bridge_u(self, u_old, u_new, t, t_bridge, out=None, obs=None, stream=None):
        """Blend the uncertainty of two estimators for fine-tuning step t (Eq. 21-22);
        writes `out` (allocated when both out and obs are None) and/or obs[:, b_max+1]."""
        if out is None and obs is None:
            out = torch.empty(self.E, dtype=torch.float32, device=self.device)
        _check(self.lib.aslam_bridge_u(self.handle, _dptr(u_old), _dptr(u_new), int(t),
                                       int(t_bridge), _dptr(out), _dptr(obs), _stream(stream)),
               self.handle)
        return out

    def csm(self, pose_pred, ranges=None, n_xy=5, n_th=5, sep=1, dth_rad=0.01, stream=None):
        """Correlative scan matching of each env's scan against its grid (Sec. III-D).
        Returns (pose_out [E,3] fp32, match [E,3] = score_norm, margin, w,
        scores [E,3] int64 = best, second, best index)."""
        c = AslamCsmConfig()
        _check(self.lib.aslam_csm_config_init(C.byref(c)))
        c.n_xy, c.n_th, c.sep, c.dth_rad = int(n_xy), int(n_th), int(sep), float(dth_rad)
        pose_out = torch.empty(self.E, 3, dtype=torch.float32, device=self.device)
        match = torch.empty(self.E, 3, dtype=torch.float32, device=self.device)
        scores = torch.empty(self.E, 3, dtype=torch.int64, device=self.device)
        _check(self.lib.aslam_csm(self.handle, C.byref(c), _dptr(pose_pred), _dptr(ranges),
                                  _dptr(pose_out), _dptr(match), _dptr(scores), _stream(stream)),
               self.handle)
        return pose_out, match, scores

    def profile_begin(self, max_steps):
        """Time each kernel of the next max_steps steps with CUDA events."""
        _check(self.lib.aslam_profile_begin(self.handle, int(max_steps)), self.handle)

    def kernel_names(self):
        """Names of the kernels one step of this batch launches, in order."""
        out = []
        while True:
            n = self.lib.aslam_kernel_name(self.handle, len(out))
            if not n:
                return out
            out.append(n.decode())

    def profile_end(self):
        """{kernel name: summed device ms} and the number of timed steps."""
        ms = (C.c_double * 8)()
        nk, ns = C.c_int32(), C.c_int32()
        _check(self.lib.aslam_profile_end(self.handle, ms, C.byref(nk), C.byref(ns)), self.handle)
        names = [self.lib.aslam_kernel_name(self.handle, k).decode() for k in range(nk.value)]
        return {n: float(ms[k]) for k, n in enumerate(names)}, int(ns.value)

    def save_state(self, stream=None):
        n = C.c_size_t()
        _check(self.lib.aslam_state_bytes(self.handle, C.byref(n)), self.handle)
        buf = np.empty(int(n.value), dtype=np.uint8)
        _check(self.lib.aslam_save_state(self.handle, buf.ctypes.data_as(P), buf.nbytes,
                                         _stream(stream)), self.handle)
        return buf

    def load_state(self, buf, stream=None):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(self.lib.aslam_load_state(self.handle, buf.ctypes.data_as(P), buf.nbytes,
                                         _stream(stream)), self.handle)


def debug_detmath(x, u, seed):
    """The library's deterministic sin/cos/log/cos2pi/gauss on CUDA tensors x, u."""
    lib = load()
    n = x.numel()
    outs = [torch.empty_like(x) for _ in range(5)]
    _check(lib.aslam_debug_detmath(_dptr(x), _dptr(u), n, *[_dptr(o) for o in outs[:4]],
                                   C.c_uint64(seed), _dptr(outs[4]), _stream()))
    return outs


def scan_update_noalloc(inputs, gt, pose, step, belief, ranges, stream=None, **cfg):
    """One scan per env into caller-owned grids, with no device allocation.

    For callers that may not allocate device memory: `gt` (uint8, packed like
    inputs.gt), `pose` [E, 3] float, `step` [E] int32 (noise counter),
    `belief` (int16, packed like inputs.gt, updated in place) and `ranges`
    [E, B] float are the caller's CUDA tensors; the library's scratch is a
    fixed array of its own.  Calls that overlap on the GPU share that array
    and must be serialised.
    """
    lib = load()
    c = config_defaults()
    E = inputs.n_envs
    w = np.ascontiguousarray(inputs.map_w, dtype=np.int32)
    h = np.ascontiguousarray(inputs.map_h, dtype=np.int32)
    b = np.ascontiguousarray(inputs.n_beams, dtype=np.int32)
    off = np.ascontiguousarray(inputs.map_off, dtype=np.int64)
    # The C side cannot see device buffer sizes: every tensor is checked here
    # against the sizes the kernels will index, so a wrong buffer is an
    # exception instead of an out-of-bounds access.
    cells = int(off[-1])
    B = int(b[0]) if E > 0 else 0
    want = [("gt", gt, torch.uint8, cells), ("belief", belief, torch.int16, cells),
            ("pose", pose, torch.float32, 3 * E), ("step", step, torch.int32, E),
            ("ranges", ranges, torch.float32, E * B)]
    dev = gt.device if isinstance(gt, torch.Tensor) else None
    for name, t, dt, n in want:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise AslamError(1, "%s must be a CUDA tensor" % name)
        if t.dtype != dt:
            raise AslamError(1, "%s must be %s, got %s" % (name, dt, t.dtype))
        if t.numel() != n:
            raise AslamError(1, "%s must have %d elements, got %d" % (name, n, t.numel()))
        if not t.is_contiguous():
            raise AslamError(1, "%s must be contiguous" % name)
        if t.device != dev:
            raise AslamError(1, "every tensor must be on %s (%s is on %s)" % (dev, name, t.device))
    c.n_envs = E
    c.res_m = float(inputs.res)
    c.h_map_w = w.ctypes.data_as(P)
    c.h_map_h = h.ctypes.data_as(P)
    c.h_n_beams = b.ctypes.data_as(P)
    for k, v in cfg.items():
        setattr(c, k, float(v) if k in _FLOAT_KEYS else int(v))
    with torch.cuda.device(dev):
        _check(lib.aslam_scan_update_noalloc(C.byref(c), _dptr(gt), off.ctypes.data_as(P),
                                             _dptr(pose), _dptr(step), _dptr(belief),
                                             _dptr(ranges), _stream(stream)))


def fixed_lag_gn(x, odo, meas, meas_info, prior, prior_info, iters=3,
                 odo_info=(1e4, 1e4, 1e4), u_scale=1e-4, stream=None):
    """Batched fixed-lag window Gauss-Newton (Sec. III-D, Eq. 5-6) on device
    tensors: x [E, L, 3] (optimised in place), odo [E, L-1, 3], meas and
    meas_info [E, L, 3], prior and prior_info [E, 3].  Returns (cov [E, 3, 3],
    u [E], status [E])."""
    lib = load()
    E, L = int(x.shape[0]), int(x.shape[1])
    c = AslamFlgnConfig()
    _check(lib.aslam_flgn_config_init(C.byref(c)))
    c.n_envs, c.window, c.iters = E, L, int(iters)
    c.odo_info = (C.c_float * 3)(*[float(v) for v in odo_info])
    c.u_scale = float(u_scale)
    cov = torch.empty(E, 3, 3, dtype=torch.float32, device=x.device)
    u = torch.empty(E, dtype=torch.float32, device=x.device)
    st = torch.empty(E, dtype=torch.int32, device=x.device)
    _check(lib.aslam_fixed_lag_gn(C.byref(c), _dptr(x), _dptr(odo), _dptr(meas),
                                  _dptr(meas_info), _dptr(prior), _dptr(prior_info), _dptr(cov),
                                  _dptr(u), _dptr(st), _stream(stream)))
    return cov, u, st
