"""The host-buffer step (aslam_step_host) against the device-buffer step
(aslam_step_fused): two batches built from the same seeded worlds and
stepped with the same actions and U give bit-identical rewards,
observations, reward terms and maps.  Every fourth step omits U and both
outputs on both sides.  Page-locked host buffers are read and written by
the kernels in place, pageable ones go through copies: both, and a mix of
the two, are checked, for a 2-D batch and for a voxel batch.  A device
tensor passed as a host buffer is rejected by the binding."""
import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth

pytestmark = pytest.mark.gpu


def _host(shape, pinned):
    t = torch.empty(*shape)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("mode", ["pinned", "pageable", "mixed", "outputs-pinned"])
def test_host_step_matches_device_step(aslam_gpu, mode):
    inp = synth.paper_scale(E=24, W=256, B=360, seed=2101)
    cfg = dict(r_max_m=12.0, noise_sigma_m=0.01, reward_mode=aslam_gpu.REWARD_COMPOSITE)
    gd = aslam_gpu.Batch2D(inp, **cfg)
    gh = aslam_gpu.Batch2D(inp, **cfg)
    E, nb = inp.n_envs, gd.b_max + 2
    acts = synth.random_actions(12, E, 61)
    uu = synth.random_uncertainty(12, E, 62)
    d_rew = torch.empty(E, device="cuda")
    d_obs = torch.empty(E, nb, device="cuda")
    pin_in = mode in ("pinned", "mixed")
    pin_out = mode in ("pinned", "outputs-pinned")
    h_act = _host((E, 2), pin_in)
    h_u = _host((E,), pin_in)
    h_rew = _host((E,), pin_out)
    h_obs = _host((E, nb), pin_out)
    for s in range(12):
        bare = s % 4 == 3
        h_act.copy_(torch.from_numpy(acts[s]))
        h_u.copy_(torch.from_numpy(uu[s]))
        if bare:
            gd.step_fused(torch.from_numpy(acts[s]).cuda(), None, None, None)
            gh.step_host(h_act, None, None, None)
        else:
            gd.step_fused(torch.from_numpy(acts[s]).cuda(), torch.from_numpy(uu[s]).cuda(),
                          d_rew, d_obs)
            gh.step_host(h_act, h_u, h_rew, h_obs)
        torch.cuda.synchronize()
        if not bare:
            np.testing.assert_array_equal(h_rew.numpy(), d_rew.cpu().numpy(), err_msg="reward %d" % s)
            np.testing.assert_array_equal(h_obs.numpy(), d_obs.cpu().numpy(), err_msg="obs %d" % s)
        sd, sh = gd.state(), gh.state()
        for k in ("belief", "terms", "x", "y", "th", "done"):
            np.testing.assert_array_equal(sd[k].cpu().numpy(), sh[k].cpu().numpy(),
                                          err_msg="%s step %d" % (k, s))
    with pytest.raises(aslam_gpu.AslamError):
        gh.step_host(torch.zeros(E, 2, device="cuda"))
    gd.close()
    gh.close()


def test_voxel_host_step_matches_device_step(aslam_gpu):
    """The 3-D step writes its reward and observation through the same
    pointers: page-locked host buffers in place against device buffers."""
    inp = synth.voxel_batch(E=3, W=32, H=32, D=8, n_az=24, K=4, seed=2102)
    cfg = dict(n_rings=4, reward_mode=aslam_gpu.REWARD_COMPOSITE)
    gd = aslam_gpu.Batch2D(inp, **cfg)
    gh = aslam_gpu.Batch2D(inp, **cfg)
    E, nb = inp.n_envs, gd.b_max + 2
    acts = synth.random_actions(6, E, 63)
    uu = synth.random_uncertainty(6, E, 64)
    d_rew = torch.empty(E, device="cuda")
    d_obs = torch.empty(E, nb, device="cuda")
    h_act, h_u = torch.empty(E, 2).pin_memory(), torch.empty(E).pin_memory()
    h_rew, h_obs = torch.empty(E).pin_memory(), torch.empty(E, nb).pin_memory()
    for s in range(6):
        h_act.copy_(torch.from_numpy(acts[s]))
        h_u.copy_(torch.from_numpy(uu[s]))
        gd.step_fused(torch.from_numpy(acts[s]).cuda(), torch.from_numpy(uu[s]).cuda(), d_rew, d_obs)
        gh.step_host(h_act, h_u, h_rew, h_obs)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(h_rew.numpy(), d_rew.cpu().numpy(), err_msg="reward %d" % s)
        np.testing.assert_array_equal(h_obs.numpy(), d_obs.cpu().numpy(), err_msg="obs %d" % s)
        np.testing.assert_array_equal(gd.state()["belief"].cpu().numpy(),
                                      gh.state()["belief"].cpu().numpy(), err_msg="belief %d" % s)
    gd.close()
    gh.close()
