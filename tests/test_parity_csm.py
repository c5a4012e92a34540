"""GPU parity of the batched correlative scan matcher (Sec. III-D) through the
C ABI against the oracle: integer scores, best index, second best and the
matched pose bit-exact; score_norm, margin and w identical (both evaluate
the same integers in fp64 and round once).  Each side matches its own map
and ranges after stepping the same seeded worlds (which agree bit for bit,
as the step parity tests show)."""
import math

import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import orc_params

pytestmark = pytest.mark.gpu


def stepped(aslam, orc, inp, steps, seed, **cfg):
    gb = aslam.Batch2D(inp, **cfg)
    ob = orc.OracleBatch2D(inp, **orc_params(cfg))
    acts = synth.random_actions(steps, inp.n_envs, seed)
    for s in range(steps):
        gb.step(torch.from_numpy(acts[s]).cuda())
        o = ob.step(acts[s])
    torch.cuda.synchronize()
    return gb, ob, o


def check(aslam, orc, inp, steps, seed, csm_kw, fov=0.0, **cfg):
    gb, ob, o = stepped(aslam, orc, inp, steps, seed, fov_rad=fov, **cfg)
    true = np.stack([ob.x, ob.y, ob.th], axis=1).astype(np.float32)
    pred = synth.perturb_poses(true, seed + 1, sigma=(0.06, 0.06, 0.02)).astype(np.float32)
    po, mt, sc = gb.csm(torch.from_numpy(pred).cuda(), **csm_kw)
    po, mt, sc = po.cpu().numpy(), mt.cpu().numpy(), sc.cpu().numpy()
    kw = dict(n_xy=csm_kw.get("n_xy", 5), n_th=csm_kw.get("n_th", 5), sep=csm_kw.get("sep", 1),
              dth=csm_kw.get("dth_rad", 0.01))
    moved = 0
    for e in range(inp.n_envs):
        B = int(inp.n_beams[e])
        ro, rm, rs = orc.csm(ob.env_belief(e), inp.res, cfg["r_max_m"], fov, o["z"][e, :B],
                             pred[e], **kw)
        np.testing.assert_array_equal(sc[e], rs, err_msg="scores env %d" % e)
        np.testing.assert_array_equal(po[e], ro, err_msg="pose env %d" % e)
        np.testing.assert_array_equal(mt[e], rm, err_msg="match env %d" % e)
        moved += int(np.abs(ro - pred[e]).max() > 0)
    return moved


def test_csm_paper_scale_small_batch(aslam_gpu, orc):
    inp = synth.paper_scale(E=6, W=256, B=360, seed=909)
    assert check(aslam_gpu, orc, inp, 12, 51, {}, r_max_m=12.0, noise_sigma_m=0.01) > 0


def test_csm_paper_sensor_and_search_sizes(aslam_gpu, orc):
    inp = synth.paper_scale(E=4, W=256, B=128, seed=910)
    for kw in ({"n_xy": 8, "n_th": 8, "sep": 2, "dth_rad": 0.005}, {"n_xy": 0, "n_th": 0},
               {"n_xy": 3, "n_th": 0, "sep": 0}):
        check(aslam_gpu, orc, inp, 8, 52, kw, fov=math.pi, r_max_m=10.0, noise_sigma_m=0.01,
              r_min_m=0.1, range_decimals=2)


def test_csm_large_map_reads_global(aslam_gpu, orc):
    # a 512^2 map does not fit the shared budget: the global-read path
    occ = [synth.paper_scale(E=1, W=512, B=8, seed=911).gt.reshape(512, 512),
           synth.paper_scale(E=1, W=128, B=8, seed=912).gt.reshape(128, 128)]
    spawn = np.stack([synth.paper_scale(E=1, W=512, B=8, seed=911).spawn[0, :4],
                      synth.paper_scale(E=1, W=128, B=8, seed=912).spawn[0, :4]])
    inp = synth.custom_2d(occ, [180, 96], 0.05, spawn)
    check(aslam_gpu, orc, inp, 6, 53, {"n_xy": 4, "n_th": 2}, r_max_m=8.0, noise_sigma_m=0.01)


def test_csm_ragged_widths_stage_cell_by_cell(aslam_gpu, orc):
    # widths that are not a multiple of 8 take the one-cell-at-a-time staging
    rng = np.random.default_rng(913)
    occ, spawn = [], []
    for W, H in ((100, 90), (77, 64), (136, 41)):
        g = np.zeros((H, W), np.uint8)
        g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = 1
        g[rng.integers(1, H - 1, 25), rng.integers(1, W - 1, 25)] = 1
        g[H // 2 - 1:H // 2 + 2, W // 2 - 1:W // 2 + 2] = 0
        occ.append(g)
        cx, cy = (W // 2 + 0.5) * 0.05, (H // 2 + 0.5) * 0.05
        spawn.append([[cx, cy, 0.3], [cx, cy, -1.2]])
    inp = synth.custom_2d(occ, [120, 64, 90], 0.05, np.array(spawn, np.float32))
    for kw in ({"n_xy": 5, "n_th": 3}, {"n_xy": 8, "n_th": 1, "sep": 3}, {"n_xy": 1, "n_th": 2}):
        check(aslam_gpu, orc, inp, 6, 54, kw, r_max_m=4.0, noise_sigma_m=0.01)


def test_csm_rejects_bad_config(aslam_gpu):
    b = aslam_gpu.Batch2D(synth.plain_1env(), r_max_m=5.0)
    pred = torch.zeros(1, 3, device="cuda")
    with pytest.raises(aslam_gpu.AslamError):
        b.csm(pred, n_xy=9)
    with pytest.raises(aslam_gpu.AslamError):
        b.csm(pred, dth_rad=0.0)
    b.close()
