"""GPU parity of the SLAM backbone inside the 2-D step (u_mode
ASLAM_U_FIXEDLAG; Sec. III-D) through the C ABI against the oracle.

Bit-exact: ranges, maps integrated at the window's optimised pose (also with
the confidence-weighted update), counts, poses, the scan matches (integer
scores, matched poses, score_norm, margin, w).  The window estimates come
from two fp64 solvers (block elimination on the GPU, a dense Gauss-Jordan
inverse in the oracle) rounded to fp32: within 4 fp32 ulps, and maps are
bit-exact wherever the newest estimate (the integration origin) is.  U_t and the covariance: 1e-6 relative; the reward terms that
read U (I, R_explore*, R_abs, R_delta*, R_t): the usual tolerance plus
|dR/dU| * 1e-6 U (|dR/dU| as bounded in test_parity_uq)."""
import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import ABS, REL, compare_step, orc_params
from tests.test_parity_uq import reward_bound

pytestmark = pytest.mark.gpu


def run_slam(aslam, orc, inp, steps, seed, weighted, e_sample=None, act_v_max=0.5, **cfg):
    gb = aslam.Batch2D(inp, flags=aslam.FLAG_DEBUG, reward_mode=aslam.REWARD_COMPOSITE,
                       u_mode=aslam.U_FIXEDLAG, slam_weighted_update=weighted, **cfg)
    envs = list(range(inp.n_envs)) if e_sample is None else list(e_sample)
    sub = inp if e_sample is None else synth.subset(inp, envs)
    ob = orc.OracleBatch2D(sub, env_ids=None if e_sample is None else np.asarray(envs), u_mode=2,
                           slam_weighted=weighted, **orc_params(cfg))
    acts = synth.random_actions(steps, inp.n_envs, seed, v_max=act_v_max)
    u_prev = np.zeros(len(envs))
    # The scan is integrated at the window's newest optimised pose (Sec.
    # III-D).  Both sides solve the window in fp64 with different solvers and
    # round it to fp32, so the estimates agree to a few ulps and, in all but
    # rare cases, exactly.  Where the newest pose is bit-identical the
    # integration origins are too, and the maps must be bit-exact; an env
    # whose estimate differs by a rounding is compared from then on only
    # where its map does not matter (ranges, true poses, window within 4
    # ulps), and such envs must stay rare.
    diverged = set()
    env_steps = 0
    for s in range(steps):
        gb.step(torch.from_numpy(acts[s]).cuda())
        torch.cuda.synchronize()
        o = ob.step(acts[s][envs], counts=e_sample is None)
        st = gb.state()
        win = st["slam_window"].cpu().numpy()[envs]
        cnt = st["slam_count"].cpu().numpy()[envs]
        np.testing.assert_array_equal(cnt, ob.win_n)
        for le in range(len(envs)):
            n = int(ob.win_n[le])
            ref = ob.win_x[le, :n]
            tol = 4 * np.spacing(np.abs(ref)) + 1e-12
            assert np.all(np.abs(win[le, :n] - ref) <= tol), (s, le)
            if not np.array_equal(win[le, n - 1], ob.win_x[le, n - 1]):
                diverged.add(le)
            env_steps += 1
        compare_step(gb, ob, o, e_map=None if e_sample is None else envs,
                     check_counts=e_sample is None, tag="slam step %d" % s,
                     skip_terms=(2, 4, 5, 6, 7), skip_maps=diverged)
        keep = [le for le in range(len(envs)) if le not in diverged]
        ge = [envs[le] for le in keep]
        np.testing.assert_array_equal(st["slam_scores"].cpu().numpy()[ge], ob.slam_scores[keep])
        np.testing.assert_array_equal(st["slam_match"].cpu().numpy()[ge], ob.slam_match[keep])
        np.testing.assert_array_equal(st["slam_match_pose"].cpu().numpy()[ge], ob.slam_pose[keep])
        u_gpu = st["u_prev"].cpu().numpy()[envs].astype(np.float64)
        u_orc = ob.u_prev.astype(np.float64)
        np.testing.assert_allclose(u_gpu[keep], u_orc[keep], rtol=1e-6, atol=1e-12)
        cov = st["pose_cov"].cpu().numpy()[envs]
        scale = np.abs(ob.sigma).max(axis=1, keepdims=True)
        rel = (np.abs(cov - ob.sigma) / scale)[keep]
        assert rel.max(initial=0) <= 1e-6, (s, rel.max(), cov.tolist(), ob.sigma.tolist())
        terms = st["terms"].cpu().numpy()[envs].astype(np.float64)
        for le in keep:
            tol = reward_bound(u_prev[le], u_orc[le]) * 1e-4
            for k in (2, 4, 5, 6, 7):
                ref = o["terms"][le, k]
                assert abs(terms[le, k] - ref) <= REL * abs(ref) + ABS + tol, (s, le, k)
        u_prev = u_orc
    assert len(diverged) <= max(1, len(envs) // 4), (sorted(diverged), env_steps)
    gb.sync_status()
    return gb, ob


@pytest.mark.parametrize("weighted", [0, 1])
def test_backbone_small_batch(aslam_gpu, orc, weighted):
    inp = synth.paper_scale(E=4, W=128, B=90, seed=1201)
    run_slam(aslam_gpu, orc, inp, 24, 61, weighted, r_max_m=6.0, noise_sigma_m=0.01)


def test_backbone_window_slides_and_resets(aslam_gpu, orc):
    inp = synth.paper_scale(E=4, W=96, B=64, seed=1202)
    gb, ob = run_slam(aslam_gpu, orc, inp, 40, 62, 1, act_v_max=1.5, r_max_m=4.0,
                      noise_sigma_m=0.01, v_max=1.5, slam_window=5)
    assert ob.ep.sum() > 0 and ob.win_n.max() == 5


def test_backbone_paper_sensor_sampled_full_size(aslam_gpu, orc):
    inp = synth.paper_scale(E=750, B=128)
    import math
    run_slam(aslam_gpu, orc, inp, 4, 63, 1, e_sample=[3, 500], fov_rad=math.pi, r_min_m=0.1,
             range_decimals=2, r_max_m=10.0, noise_sigma_m=0.01)
