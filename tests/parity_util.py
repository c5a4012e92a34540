"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare them step by step.

Tolerances (derived from the arithmetic):
  * ranges, hit flags, traversed-cell counts, int16 log-odds, poses and the
    observation are computed from identical IEEE fp32 operation sequences
    and exact integer geometry on both sides -> compared bit-exactly;
  * the entropy gain dH: the oracle sums h(L) over the whole map in fp64
    (error <= N*2^-53*H), the kernel sums table entries rounded to 2^-41
    nats over the touched cells and stores fp32 -> |dH_gpu - dH_orc| <=
    1e-5*|dH_orc| + 1e-6 nats;
  * the composite reward: fp64 on both sides from identical fp32 inputs,
    stored as fp32 -> 1e-5 relative + 1e-6 absolute;
  * the absolute entropy H_t (term 11) is stored as fp32: one rounding,
    2^-24 relative, plus the dH error above -> 2^-23 relative + 1e-6.
"""
import numpy as np
import torch

from paper_2603_25834_gb300.synth import subset  # noqa: F401

REL = 1e-5
ABS = 1e-6


def gpu_batch(aslam, inputs, **cfg):
    return aslam.Batch2D(inputs, flags=aslam.FLAG_DEBUG, **cfg)


def orc_params(cfg):
    """Map libaslam config names to the oracle's parameter names."""
    names = dict(r_max_m="r_max", fov_rad="fov", noise_sigma_m="sigma", dt_s="dt",
                 v_max="v_max", w_max="w_max", l_hit_q="hit_q", l_miss_q="miss_q",
                 l_clamp_q="clamp_q", t_episode="t_episode", d_crash="d_crash",
                 d_full="d_full", visit_cell_m="visit_cell", lam_col="lam_col",
                 lam_explore="lam_explore", lam_abs="lam_abs", lam_delta="lam_delta",
                 kappa="kappa", u_hi="u_hi", seed="seed", r_min_m="r_min",
                 range_decimals="decimals", slam_window="slam_window",
                 slam_iters="slam_iters", csm_n_xy="csm_n_xy", csm_n_th="csm_n_th",
                 csm_sep="csm_sep", csm_dth_rad="csm_dth", slam_gn_iters="slam_gn_iters")
    return {names[k]: v for k, v in cfg.items() if k in names}


def compare_step(gb, ob, o, e_map=None, check_counts=True, tag="", skip_terms=(), skip_maps=()):
    """Compare the GPU batch's last step with the oracle's step output `o`.
    skip_maps: local env indices whose maps, counts, ray-cell counts and
    reward terms are not compared (their integration origins differ)."""
    st = gb.state()
    E = ob.E
    envs = list(range(E)) if e_map is None else list(e_map)
    # a batch created without ASLAM_FLAG_DEBUG (the bench's configuration)
    # keeps no noise-free ranges, hit flags or per-cell counts
    debug = st["z_true"] is not None
    check_counts = check_counts and debug
    z = st["z"].cpu().numpy()
    zt = st["z_true"].cpu().numpy() if debug else None
    hit = st["hit"].cpu().numpy() if debug else None
    terms = st["terms"].cpu().numpy()
    bel = st["belief"].cpu().numpy()
    cnt = st["counts"].cpu().numpy().view(np.uint32) if check_counts else None
    for le, ge in enumerate(envs):
        B = int(ob.n_beams[le])
        r0 = int(gb.ray_off[ge])
        np.testing.assert_array_equal(z[r0:r0 + B], o["z"][le, :B], err_msg="z %s env %d" % (tag, ge))
        if debug:
            np.testing.assert_array_equal(zt[r0:r0 + B], o["z_true"][le, :B],
                                          err_msg="z_true %s env %d" % (tag, ge))
            np.testing.assert_array_equal(hit[r0:r0 + B], o["hit"][le, :B],
                                          err_msg="hit %s env %d" % (tag, ge))
        W, H = int(ob.map_w[le]), int(ob.map_h[le])
        m0 = int(gb.map_off[ge])
        if le in skip_maps:
            assert np.abs(bel[m0:m0 + W * H].astype(np.int32)).max(initial=0) <= ob.p["clamp_q"]
            continue
        np.testing.assert_array_equal(bel[m0:m0 + W * H], ob.belief[ob.map_off[le]:ob.map_off[le] + W * H],
                                      err_msg="belief %s env %d" % (tag, ge))
        if check_counts:
            c = cnt[m0:m0 + W * H]
            oh = o["cnt_h"][ob.map_off[le]:ob.map_off[le] + W * H]
            om = o["cnt_m"][ob.map_off[le]:ob.map_off[le] + W * H]
            np.testing.assert_array_equal(c >> 16, oh, err_msg="hits %s env %d" % (tag, ge))
            np.testing.assert_array_equal(c & 0xFFFF, om, err_msg="misses %s env %d" % (tag, ge))
        assert int(st["ray_cells"][ge]) == int(o["ray_cells"][le]), (tag, ge)
        assert int(st["gt_cells"][ge]) == int(o["gt_cells"][le]), (tag, ge)
        ot = o["terms"][le]
        gt_ = terms[ge].astype(np.float64)
        for k in (0, 1, 2, 3, 4, 5, 6, 7, 11):
            if k in skip_terms:
                continue
            tol = REL * abs(ot[k]) + ABS
            if k == 11:
                # absolute map entropy H (up to ~2e5 nats) is stored as fp32
                tol = 2.0 ** -23 * abs(ot[k]) + ABS
            assert abs(gt_[k] - ot[k]) <= tol, (tag, ge, k, gt_[k], ot[k])
        assert gt_[8] == ot[8] and np.float32(gt_[9]) == np.float32(ot[9]) and \
            np.float32(gt_[10]) == np.float32(ot[10]), (tag, ge)
    for k in ("x", "y", "th"):
        g = st[k].cpu().numpy()[envs]
        np.testing.assert_array_equal(g, getattr(ob, k), err_msg="%s %s" % (k, tag))
    for k in ("t", "ep", "done", "g"):
        g = st[k].cpu().numpy()[envs]
        np.testing.assert_array_equal(g, getattr(ob, k).astype(np.int32), err_msg="%s %s" % (k, tag))


def run_parity(aslam, orc, inputs, actions, u=None, e_sample=None, counts=True, tag="",
               gpu_kw=None, **cfg):
    """Step both sides for len(actions) steps and compare after every step."""
    kw = dict(gpu_kw or {})
    gb = aslam.Batch2D(inputs, flags=aslam.FLAG_DEBUG | kw.pop("flags", 0), **kw, **cfg)
    if e_sample is None:
        ob = orc.OracleBatch2D(inputs, **orc_params(cfg))
        envs = None
    else:
        sub = subset(inputs, e_sample)
        ob = orc.OracleBatch2D(sub, env_ids=np.asarray(e_sample, np.int32), **orc_params(cfg))
        envs = e_sample
    dev = gb.device
    steps = actions.shape[0]
    for s in range(steps):
        a = torch.from_numpy(actions[s]).to(dev)
        uu = None if u is None else torch.from_numpy(u[s]).to(dev)
        gb.step(a, uu)
        torch.cuda.synchronize()
        if envs is None:
            o = ob.step(actions[s], None if u is None else u[s], counts=counts)
        else:
            o = ob.step(actions[s][envs], None if u is None else u[s][envs], counts=counts)
        compare_step(gb, ob, o, e_map=envs, check_counts=counts, tag="%s step %d" % (tag, s))
    gb.sync_status()
    return gb, ob


def compare_obs(obs, ob, o, b_max, e_map=None, tag=""):
    """Element-by-element comparison of observation rows [E, b_max + 2] (Eq. 3)
    with the oracle's: the env's B ranges, r_max padding up to b_max, the
    yaw and U_t.  Every element is an fp32 value both sides form with the
    same operations, so the comparison is bit-exact."""
    obs = obs.cpu().numpy() if hasattr(obs, "cpu") else np.asarray(obs)
    envs = list(range(ob.E)) if e_map is None else list(e_map)
    for le, ge in enumerate(envs):
        B = int(ob.n_beams[le])
        row = obs[ge]
        oro = o["obs"][le]
        ob_max = oro.shape[0] - 2
        np.testing.assert_array_equal(row[:B], oro[:B], err_msg="obs ranges %s env %d" % (tag, ge))
        assert np.all(row[B:b_max] == np.float32(ob.p["r_max"])), ("obs padding", tag, ge)
        assert np.all(oro[B:ob_max] == np.float32(ob.p["r_max"])), ("oracle padding", tag, ge)
        assert row[b_max] == oro[ob_max], ("obs yaw", tag, ge, row[b_max], oro[ob_max])
        assert row[b_max + 1] == oro[ob_max + 1], ("obs U", tag, ge, row[b_max + 1], oro[ob_max + 1])
