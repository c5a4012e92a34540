"""Differentiable soft expected-range raycaster and Gauss-Newton pose correction.

Binding of the aslam_soft_* / aslam_gn_correct C entry points (argument
marshalling only; the math runs in libaslam's kernels) and a
torch.autograd.Function whose backward calls the hand-written adjoint kernel.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import aslam as _a


def soft_config(E, W, H, B, K=64, res=0.05, ds=0.05, fov=0.0, mu=1e-6, sigma=0.01):
    lib = _a.load()
    c = _a.AslamSoftConfig()
    _a._check(lib.aslam_soft_config_init(C.byref(c)))
    c.n_envs, c.map_w, c.map_h, c.n_beams, c.n_samples = E, W, H, B, K
    c.res_m, c.sample_step_m, c.fov_rad = res, ds, fov
    c.gn_damping, c.range_sigma_m = mu, sigma
    return c


def _cfg_for(logodds, n_beams, n_samples, res, ds, fov, mu=1e-6, sigma=0.01):
    E, H, W = logodds.shape
    return soft_config(E, W, H, n_beams, n_samples, res, ds, fov, mu, sigma)


def _f32(t):
    if t.dtype != torch.float32 or not t.is_contiguous():
        t = t.float().contiguous()
    return t


def soft_range_fwd(cfg, logodds, pose, out=None, stream=None):
    out = out if out is not None else torch.empty(cfg.n_envs, cfg.n_beams, device=logodds.device)
    _a._check(_a.load().aslam_soft_range_fwd(C.byref(cfg), _a._dptr(logodds), _a._dptr(pose),
                                             _a._dptr(out), _a._stream(stream)))
    return out


def soft_range_jac(cfg, logodds, pose, stream=None):
    r = torch.empty(cfg.n_envs, cfg.n_beams, device=logodds.device)
    J = torch.empty(cfg.n_envs, cfg.n_beams, 3, device=logodds.device)
    _a._check(_a.load().aslam_soft_range_jac(C.byref(cfg), _a._dptr(logodds), _a._dptr(pose),
                                             _a._dptr(r), _a._dptr(J), _a._stream(stream)))
    return r, J


def soft_range_bwd(cfg, logodds, pose, grad_r, grad_map=True, stream=None):
    gp = torch.empty(cfg.n_envs, 3, device=logodds.device)
    gm = torch.zeros_like(logodds) if grad_map else None
    _a._check(_a.load().aslam_soft_range_bwd(C.byref(cfg), _a._dptr(logodds), _a._dptr(pose),
                                             _a._dptr(grad_r), _a._dptr(gp), _a._dptr(gm),
                                             _a._stream(stream)))
    return gp, gm


def gn_correct(cfg, logodds, pose, z, iters=5, stream=None):
    """Gauss-Newton scan-to-map correction: (pose_out [E,3], cov [E,3,3], U [E])."""
    dev = logodds.device
    po = torch.empty(cfg.n_envs, 3, device=dev)
    cov = torch.empty(cfg.n_envs, 3, 3, device=dev)
    u = torch.empty(cfg.n_envs, device=dev)
    _a._check(_a.load().aslam_gn_correct(C.byref(cfg), _a._dptr(logodds), _a._dptr(pose),
                                         _a._dptr(z), int(iters), _a._dptr(po), _a._dptr(cov),
                                         _a._dptr(u), _a._stream(stream)))
    return po, cov, u


class SoftRange(torch.autograd.Function):
    """ranges = SoftRange.apply(pose [E,3], logodds [E,H,W], n_beams, n_samples, res, ds, fov)."""

    @staticmethod
    def forward(ctx, pose, logodds, n_beams, n_samples=64, res=0.05, ds=0.05, fov=0.0):
        pose = _f32(pose.detach())
        logodds = _f32(logodds.detach())
        cfg = _cfg_for(logodds, n_beams, n_samples, res, ds, fov)
        ctx.save_for_backward(pose, logodds)
        ctx.cfg_args = (n_beams, n_samples, res, ds, fov)
        return soft_range_fwd(cfg, logodds, pose)

    @staticmethod
    def backward(ctx, grad_r):
        pose, logodds = ctx.saved_tensors
        cfg = _cfg_for(logodds, *ctx.cfg_args)
        gp, gm = soft_range_bwd(cfg, logodds, pose, _f32(grad_r),
                                grad_map=ctx.needs_input_grad[1])
        return gp if ctx.needs_input_grad[0] else None, gm, None, None, None, None, None


def soft_range(pose, logodds, n_beams, n_samples=64, res=0.05, ds=0.05, fov=0.0):
    return SoftRange.apply(pose, logodds, n_beams, n_samples, res, ds, fov)
