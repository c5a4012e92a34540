"""GPU parity of the paper sensor mode (Sec. IV-A: 128 rays over the 180-degree
front field of view, minimum range 0.1 m, two decimal places, 10 m, v in
(0, 0.4)) and of the uncertainty bridge (Sec. III-G, Eq. 21-22), through the
C ABI, against the oracle.  Ranges, maps and counts bit-exact; rewards within
the tolerances of parity_util; the bridged uncertainty bit-exact (the same
fp32 operations on both sides)."""
import math

import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import run_parity
from tests.test_parity_step3d import run3

pytestmark = pytest.mark.gpu

PAPER_SENSOR = dict(fov_rad=math.pi, r_min_m=0.1, range_decimals=2, r_max_m=10.0,
                    noise_sigma_m=0.01, v_max=0.4)


def test_paper_sensor_mode_2d(aslam_gpu, orc):
    inp = synth.paper_scale(E=6, B=128, seed=4242)
    acts = synth.random_actions(25, 6, 31, v_max=0.4)
    u = synth.random_uncertainty(25, 6, 32)
    gb, ob = run_parity(aslam_gpu, orc, inp, acts, u=u, tag="paper-sensor", **PAPER_SENSOR)
    z = gb.state()["z"].cpu().numpy()
    hit = gb.state()["hit"].cpu().numpy().astype(bool)
    assert z.min() >= np.float32(0.1) and z.max() <= np.float32(10.0)
    np.testing.assert_allclose(z[hit] * 100, np.rint(z[hit] * 100), atol=1e-3)


def test_paper_sensor_mode_sampled_at_full_size(aslam_gpu, orc):
    inp = synth.paper_scale(E=750, B=128)
    acts = synth.random_actions(4, 750, 33, v_max=0.4)
    run_parity(aslam_gpu, orc, inp, acts, e_sample=[0, 377, 749], counts=False,
               tag="paper-sensor-750", **PAPER_SENSOR)


def test_range_rounding_and_minimum_range_3d(aslam_gpu, orc):
    inp = synth.voxel_batch(E=3, W=48, H=48, D=12, n_az=64, K=2)
    run3(aslam_gpu, orc, inp, 4, 6, r_max_m=6.0, noise_sigma_m=0.01, r_min_m=0.3,
         range_decimals=2)


def test_bridge_u_matches_oracle(aslam_gpu, orc):
    inp = synth.paper_scale(E=5, W=64, B=16, seed=77)
    b = aslam_gpu.Batch2D(inp, r_max_m=3.0)
    rng = np.random.default_rng(3)
    u_old = rng.uniform(0, 1.5, 5).astype(np.float32)
    u_new = rng.uniform(0, 3.0, 5).astype(np.float32)
    obs = torch.full((5, b.b_max + 2), -7.0, device="cuda")
    for t, T in [(0, 1000), (17, 1000), (500, 1000), (999, 1000), (1000, 1000), (12345, 1000),
                 (3, 7)]:
        out = b.bridge_u(torch.from_numpy(u_old).cuda(), torch.from_numpy(u_new).cuda(), t, T,
                         obs=obs)
        o = obs.cpu().numpy()
        ref = orc.bridge_u(u_old, u_new, t, T)
        np.testing.assert_array_equal(out.cpu().numpy() if out is not None else o[:, -1], ref)
        np.testing.assert_array_equal(o[:, -1], ref)
        assert np.all(o[:, :-1] == -7.0)
    with pytest.raises(aslam_gpu.AslamError):
        b.bridge_u(torch.from_numpy(u_old).cuda(), torch.from_numpy(u_new).cuda(), 5, 0)
    b.close()
