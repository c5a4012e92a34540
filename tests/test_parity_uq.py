"""GPU parity of the in-step pose uncertainty (u_mode ASLAM_U_SCANMATCH;
Sec. III-D, Eq. 5-6) through the C ABI against the oracle.

The map, ranges, counts and poses stay bit-exact (U_t feeds only the reward
and the observation).  Tolerances for what U_t touches, from the arithmetic:
* the kernel evaluates the soft-range Jacobian with the accurate model of
  the differentiable form (fp64 directions, exact sample fractions,
  correctly rounded sigmoid), within 5e-5 of its largest entry (the
  soft-range parity bound; measured 1.7e-5), and sums J J^T in fp64: A is
  within ~1e-4 relative of the oracle's fp64 A.  The fp64 fusion
  ((Sigma_{t-1} + Q)^-1 + A)^-1 keeps that relative error on Sigma_t (A is
  added to a positive definite prior, so no direction is amplified), and
  det^(1/3) divides it by three: U within 1e-4 relative, Sigma entries within
  1e-4 of the largest diagonal entry (measured on GB300: <= 1.8e-6 and
  2.0e-6);
* the reward terms that read U (I, R_explore*, R_abs, R_delta*, R_t) move
  by at most |dR/dU| * dU with |dR/dU| <= lam_explore (2/U_hi + 1/kappa) +
  lam_abs e^U (1 + U) + lam_delta e^U (2 + U) per U (U_{t-1} and U_t).
"""
import math

import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import ABS, REL, compare_step, orc_params

pytestmark = pytest.mark.gpu

U_REL = 1e-4
COV_TOL = 1e-4
UQ_GPU = dict(u_mode=1, uq_samples=64, uq_range_sigma_m=0.01, uq_odo_sigma=(0.01, 0.01, 0.01),
              uq_prior_sigma=(0.01, 0.01, 0.01))
UQ_ORC = dict(u_mode=1, uq_samples=64, uq_range_sigma=0.01, uq_odo=(0.01, 0.01, 0.01),
              uq_prior=(0.01, 0.01, 0.01))


def reward_bound(u_prev, u):
    lam_explore, lam_abs, lam_delta, kappa, u_hi = 1.0, 0.1, 1.0, 0.05, 1.0
    m = max(u_prev, u)
    k = lam_explore * (2 / u_hi + 1 / kappa) + lam_abs * math.exp(m) * (1 + m) + \
        lam_delta * math.exp(m) * (2 + m)
    return k * U_REL * (u_prev + u) + 1e-6


def run_uq(aslam, orc, inp, steps, seed, e_sample=None, act_v_max=0.5, **cfg):
    gb = aslam.Batch2D(inp, flags=aslam.FLAG_DEBUG, reward_mode=aslam.REWARD_COMPOSITE,
                       **UQ_GPU, **cfg)
    envs = list(range(inp.n_envs)) if e_sample is None else list(e_sample)
    sub = inp if e_sample is None else synth.subset(inp, envs)
    ob = orc.OracleBatch2D(sub, env_ids=None if e_sample is None else np.asarray(envs),
                           **UQ_ORC, **orc_params(cfg))
    acts = synth.random_actions(steps, inp.n_envs, seed, v_max=act_v_max)
    u_prev_orc = np.zeros(len(envs))
    for s in range(steps):
        gb.step(torch.from_numpy(acts[s]).cuda())
        torch.cuda.synchronize()
        o = ob.step(acts[s][envs], counts=e_sample is None)
        # everything U does not touch: bit-exact / the usual tolerances
        compare_step(gb, ob, o, e_map=None if e_sample is None else envs,
                     check_counts=e_sample is None, tag="uq step %d" % s, skip_terms=(2, 4, 5, 6, 7))
        st = gb.state()
        u_gpu = st["u_prev"].cpu().numpy()[envs].astype(np.float64)
        u_orc = ob.u_prev.astype(np.float64)
        np.testing.assert_allclose(u_gpu, u_orc, rtol=U_REL, atol=1e-9, err_msg="U step %d" % s)
        cov = st["pose_cov"].cpu().numpy()[envs]
        scale = ob.sigma[:, [0, 3, 5]].max(axis=1, keepdims=True)
        assert np.all(np.abs(cov - ob.sigma) <= COV_TOL * scale), s
        terms = st["terms"].cpu().numpy()[envs].astype(np.float64)
        for le in range(len(envs)):
            tol = reward_bound(u_prev_orc[le], u_orc[le])
            for k in (2, 4, 5, 6, 7):
                ref = o["terms"][le, k]
                assert abs(terms[le, k] - ref) <= REL * abs(ref) + ABS + tol, (s, le, k)
        u_prev_orc = u_orc
    gb.sync_status()
    return gb, ob


def test_scan_match_uncertainty_small_batch(aslam_gpu, orc):
    inp = synth.paper_scale(E=5, W=128, B=90, seed=606)
    run_uq(aslam_gpu, orc, inp, 15, 41, r_max_m=6.0, noise_sigma_m=0.01)


def test_scan_match_uncertainty_resets(aslam_gpu, orc):
    # a long run with collisions: the covariance restarts from the prior
    inp = synth.paper_scale(E=4, W=96, B=64, seed=607)
    gb, ob = run_uq(aslam_gpu, orc, inp, 50, 42, act_v_max=1.5, r_max_m=4.0, noise_sigma_m=0.01,
                    v_max=1.5)
    assert ob.ep.sum() > 0                     # at least one env was reset


def test_scan_match_uncertainty_paper_sensor_full_size(aslam_gpu, orc):
    inp = synth.paper_scale(E=750, B=128)
    run_uq(aslam_gpu, orc, inp, 3, 43, e_sample=[0, 401, 749], fov_rad=math.pi, r_min_m=0.1,
           range_decimals=2, r_max_m=10.0, noise_sigma_m=0.01)


def test_u_enters_the_observation(aslam_gpu):
    inp = synth.paper_scale(E=3, W=96, B=64, seed=608)
    b = aslam_gpu.Batch2D(inp, r_max_m=4.0, **UQ_GPU)
    obs = torch.zeros(3, b.b_max + 2, device="cuda")
    rew = torch.zeros(3, device="cuda")
    b.step_fused(torch.zeros(3, 2, device="cuda"), None, rew, obs)
    torch.cuda.synchronize()
    # first scan of an all-unknown map: Sigma = prior + Q, U = 2 exactly in fp64
    np.testing.assert_allclose(obs[:, -1].cpu().numpy(), 2.0, rtol=1e-6)
    assert torch.equal(obs[:, -1], b.state()["u_prev"])
    st = b.save_state()
    b2 = aslam_gpu.Batch2D(inp, r_max_m=4.0, **UQ_GPU)
    b2.load_state(st)
    assert torch.equal(b2.state()["pose_cov"], b.state()["pose_cov"])
