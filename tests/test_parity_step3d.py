"""GPU parity of the 3-D voxel step (through the C ABI) against the oracle:
bit-exact ranges, hit flags, per-voxel hit/miss counts, int16 voxel
log-odds, cell counts and poses; entropy gain and rewards within the
tolerances derived in parity_util."""
import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import ABS, REL

pytestmark = pytest.mark.gpu

NAMES3 = dict(r_max_m="r_max", noise_sigma_m="sigma", sensor_z_m="sensor_z",
              elev_min_rad="el_min", elev_max_rad="el_max", t_episode="t_episode",
              d_crash="d_crash", d_full="d_full", r_min_m="r_min", range_decimals="decimals")


def run3(aslam, orc, inp, rings, steps, envs=None, seed=5, counts=True, **cfg):
    g = aslam.Batch2D(inp, flags=aslam.FLAG_DEBUG, n_rings=rings, **cfg)
    sel = list(range(inp.n_envs)) if envs is None else list(envs)
    sub = inp if envs is None else subset3(inp, sel)
    ob = orc.OracleBatch3D(sub, n_rings=rings, env_ids=None if envs is None else sel,
                           **{NAMES3[k]: v for k, v in cfg.items()})
    acts = synth.random_actions(steps, inp.n_envs, seed)
    u = synth.random_uncertainty(steps, inp.n_envs, seed + 1)
    for s in range(steps):
        g.step(torch.from_numpy(acts[s]).cuda(), torch.from_numpy(u[s]).cuda())
        torch.cuda.synchronize()
        o = ob.step(acts[s][sel], u[s][sel], counts=counts)
        st = g.state()
        z, zt, hit = (st[k].cpu().numpy() for k in ("z", "z_true", "hit"))
        bel = st["belief"].cpu().numpy()
        cnt = st["counts"].cpu().numpy().view(np.uint32)
        terms = st["terms"].cpu().numpy()
        for le, ge in enumerate(sel):
            B = ob.B
            r0 = int(g.ray_off[ge])
            np.testing.assert_array_equal(z[r0:r0 + B], o["z"][le], err_msg="z step %d env %d" % (s, ge))
            np.testing.assert_array_equal(zt[r0:r0 + B], o["z_true"][le])
            np.testing.assert_array_equal(hit[r0:r0 + B], o["hit"][le])
            n = int(ob.map_off[le + 1] - ob.map_off[le])
            m0, a0 = int(g.map_off[ge]), int(ob.map_off[le])
            np.testing.assert_array_equal(bel[m0:m0 + n], ob.belief[a0:a0 + n],
                                          err_msg="belief step %d env %d" % (s, ge))
            if counts:
                np.testing.assert_array_equal(cnt[m0:m0 + n] >> 16, o["cnt_h"][a0:a0 + n])
                np.testing.assert_array_equal(cnt[m0:m0 + n] & 0xFFFF, o["cnt_m"][a0:a0 + n])
            assert int(st["ray_cells"][ge]) == int(o["ray_cells"][le])
            assert int(st["gt_cells"][ge]) == int(o["gt_cells"][le])
            for k in (0, 1, 2, 3, 4, 5, 6, 7):
                assert abs(terms[ge, k] - o["terms"][le, k]) <= REL * abs(o["terms"][le, k]) + ABS, (s, ge, k)
            assert abs(terms[ge, 11] - o["terms"][le, 11]) <= 2.0 ** -23 * abs(o["terms"][le, 11]) + ABS
        for k in ("x", "y", "th"):
            np.testing.assert_array_equal(st[k].cpu().numpy()[sel], getattr(ob, k))
    g.sync_status()
    return g, ob


def subset3(inp, envs):
    grids, spawn = [], []
    for e in envs:
        grids.append(inp.gt[int(inp.map_off[e]):int(inp.map_off[e + 1])])
        spawn.append(inp.spawn[e])
    off = np.zeros(len(envs) + 1, np.int64)
    off[1:] = np.cumsum([g.size for g in grids])
    return synth.Batch3DInputs(inp.map_w[envs], inp.map_h[envs], inp.map_d[envs], inp.n_beams[envs],
                               inp.res, np.concatenate(grids), off, np.stack(spawn))


def test_small_voxel_batch(aslam_gpu, orc):
    inp = synth.voxel_batch(E=3, W=32, H=32, D=8, n_az=24, K=4, seed=11)
    run3(aslam_gpu, orc, inp, 4, 5, r_max_m=4.0, noise_sigma_m=0.01)


def test_level_ring_and_single_elevation(aslam_gpu, orc):
    inp = synth.voxel_batch(E=2, W=40, H=24, D=6, n_az=64, K=2, seed=12)
    run3(aslam_gpu, orc, inp, 1, 3, r_max_m=3.0, noise_sigma_m=0.02, elev_min_rad=0.0,
         elev_max_rad=0.0, sensor_z_m=0.35)


def test_paper_3d_size_two_envs(aslam_gpu, orc):
    """128 x 128 x 32 voxels at 0.1 m, 16 rings x 512 azimuths, 20 m."""
    inp = synth.voxel_batch(E=2, seed=13)
    run3(aslam_gpu, orc, inp, 16, 2, r_max_m=20.0, noise_sigma_m=0.01)


def test_full_3d_batch_sampled(aslam_gpu, orc):
    """The 512-env voxel workload in one launch; 2 sampled envs replayed."""
    inp = synth.voxel_batch(E=512, seed=14)
    run3(aslam_gpu, orc, inp, 16, 2, envs=[0, 511], counts=False, r_max_m=20.0,
         noise_sigma_m=0.01)
