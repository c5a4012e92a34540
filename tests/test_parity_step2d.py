"""GPU parity of the 2-D step (CUDA path through the C ABI) against the oracle.

Bit-exact: ranges, hit flags, per-cell hit/miss counts of every step, int16
log-odds maps, ray/ground-truth cell counts, poses.  Tolerance (see
parity_util): entropy gain and rewards.
"""
import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import compare_step, orc_params, run_parity, subset

pytestmark = pytest.mark.gpu


def test_detmath_bit_equal_to_oracle(aslam_gpu, orc):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-8, 8, 20000), np.linspace(-3.5, 3.5, 7001),
                        [0.0, np.pi, -np.pi, np.pi / 2, 1e-7]]).astype(np.float32)
    u = np.concatenate([(np.arange(1, x.size // 2 + 1) / 16777216.0),
                        rng.uniform(0, 1, x.size - x.size // 2)]).astype(np.float32)[:x.size]
    u = np.maximum(u, np.float32(1.0 / 16777216.0))
    seed = 0x1234_5678_9ABC
    s, c, l, c2, g = [t.cpu().numpy() for t in aslam_gpu.debug_detmath(
        torch.from_numpy(x).cuda(), torch.from_numpy(u).cuda(), seed)]
    for q in range(0, x.size, 7):
        os_, oc = orc.sincosf(float(x[q]))
        assert s[q] == np.float32(os_) and c[q] == np.float32(oc), q
        assert l[q] == np.float32(orc.logf(float(u[q]))), q
        uu = np.float32(u[q] - np.floor(u[q]))
        assert c2[q] == np.float32(orc.cos2pi(float(uu))), q
        assert g[q] == np.float32(orc.gauss(seed, q % 7, q // 7, q)), q


@pytest.mark.parametrize("sigma", [0.0, 0.01])
def test_plain_1env_100_steps(aslam_gpu, orc, sigma):
    inp = synth.plain_1env()
    acts = synth.random_actions(100, 1, 101)
    u = synth.random_uncertainty(100, 1, 102)
    gb, ob = run_parity(aslam_gpu, orc, inp, acts, u=u, tag="cfg0", r_max_m=5.0,
                        noise_sigma_m=sigma, reward_mode=1)
    # rewards through the public calls
    r = gb.reward().cpu().numpy()
    t = gb.reward_terms().cpu().numpy()
    assert r[0] == t[0, 7]


def test_paper_scale_small_batch(aslam_gpu, orc):
    inp = synth.paper_scale(E=6)
    acts = synth.random_actions(12, 6, 7)
    u = synth.random_uncertainty(12, 6, 8)
    run_parity(aslam_gpu, orc, inp, acts, u=u, tag="cfg1-6", r_max_m=12.0,
               noise_sigma_m=0.01)


@pytest.mark.parametrize("B", [97, 194])
def test_beam_counts_with_the_fallback_map_stride(aslam_gpu, orc, B):
    """The update kernel lists an env's beams in its chunk map by a stride
    coprime with B: 97, or 89 when 97 divides B.  Beam counts that take the
    fallback stride, bit-exact against the oracle."""
    inp = synth.paper_scale(E=4, B=B, seed=4242)
    acts = synth.random_actions(6, 4, 43)
    run_parity(aslam_gpu, orc, inp, acts, tag="stride-B%d" % B, r_max_m=12.0,
               noise_sigma_m=0.01)


@pytest.mark.parametrize("window,threads", [(64, 128), (128, 160), (200, 256)])
def test_partial_window_and_global_counters(aslam_gpu, orc, window, threads):
    inp = synth.paper_scale(E=4, seed=777)
    acts = synth.random_actions(6, 4, 9)
    run_parity(aslam_gpu, orc, inp, acts, tag="partial-%d" % window, r_max_m=12.0,
               noise_sigma_m=0.01, gpu_kw=dict(window_cells=window, threads_per_cta=threads))


def test_uneven_maps_and_beams(aslam_gpu, orc):
    inp = synth.uneven(E=10, seed=4242)
    acts = synth.random_actions(4, 10, 5)
    run_parity(aslam_gpu, orc, inp, acts, tag="uneven", r_max_m=12.0, noise_sigma_m=0.01)
    run_parity(aslam_gpu, orc, inp, acts[:2], tag="uneven-w128", r_max_m=12.0,
               noise_sigma_m=0.01, gpu_kw=dict(window_cells=128))


def edge_inputs():
    occs, beams, spawn = [], [], []
    # a 1 x 37 column and a 29 x 1 row (rays leave the map at once)
    occs.append(np.zeros((37, 1), np.uint8)); beams.append(16); spawn.append((0.05, 1.03, 0.3))
    row = np.zeros((1, 29), np.uint8); row[0, 20] = 1
    occs.append(row); beams.append(16); spawn.append((0.52, 0.05, 0.0))
    # no beams at all
    o = np.zeros((16, 16), np.uint8); o[0, :] = 1
    occs.append(o); beams.append(0); spawn.append((0.8, 0.8, 0.0))
    # one beam; the maximum beam count
    occs.append(np.pad(np.zeros((30, 30), np.uint8), 1, constant_values=1)); beams.append(1)
    spawn.append((1.6, 1.6, 0.7))
    occs.append(np.pad(np.zeros((62, 62), np.uint8), 1, constant_values=1)); beams.append(1024)
    spawn.append((1.1, 3.3, -2.0))
    # empty map without walls, robot exactly on a grid corner looking along a diagonal
    occs.append(np.zeros((32, 32), np.uint8)); beams.append(8)
    spawn.append((1.0, 1.0, float(np.float32(np.pi / 4))))
    # robot on a vertical grid line next to an obstacle corner
    o = np.zeros((24, 24), np.uint8); o[12:16, 12:16] = 1
    occs.append(o); beams.append(90); spawn.append((1.1, 1.1, 0.0))
    sp = np.array([[s, s] for s in spawn], np.float32)
    return synth.custom_2d(occs, beams, 0.1, sp)


def test_edge_cases(aslam_gpu, orc):
    inp = edge_inputs()
    E = inp.n_envs
    acts = synth.random_actions(8, E, 31, v_max=0.3)
    acts[0, :, :] = 0.0
    run_parity(aslam_gpu, orc, inp, acts, tag="edge", r_max_m=2.5, noise_sigma_m=0.02)
    # ranges exactly hitting cell boundaries: r_max on a grid line, no noise
    run_parity(aslam_gpu, orc, inp, acts[:3], tag="edge-exact", r_max_m=1.0, noise_sigma_m=0.0)


def test_collisions_resets_and_long_run(aslam_gpu, orc):
    """Many steps of random driving with a small episode: resets via both paths."""
    inp = synth.paper_scale(E=3, W=64, B=90, seed=99)
    acts = synth.random_actions(60, 3, 12)
    gb, ob = run_parity(aslam_gpu, orc, inp, acts, tag="resets", r_max_m=3.0,
                        noise_sigma_m=0.01, t_episode=17, d_crash=0.3, d_full=0.8,
                        counts=False)
    assert ob.ep.sum() >= 3


def test_full_size_sampled_envs(aslam_gpu, orc):
    """750 envs of 256^2 at 0.05 m, 360 beams, 12 m (the bench workload), in the
    bench's launch configuration; 6 sampled envs replayed by the oracle."""
    inp = synth.paper_scale(E=750)
    acts = synth.random_actions(3, 750, 2026)
    u = synth.random_uncertainty(3, 750, 2027)
    sample = [0, 1, 137, 374, 600, 749]
    gb, ob = run_parity(aslam_gpu, orc, inp, acts, u=u, e_sample=sample, tag="cfg1-full",
                        r_max_m=12.0, noise_sigma_m=0.01, reward_mode=1)
    st = gb.state()
    bel = st["belief"]
    assert int(bel.abs().max()) <= 3584
    assert int(st["ray_cells"].min()) > 0


def test_graph_replay_matches_plain_steps(aslam_gpu):
    inp = synth.paper_scale(E=16, seed=5)
    acts = synth.random_actions(5, 16, 3)
    a = aslam_gpu.Batch2D(inp, r_max_m=12.0, noise_sigma_m=0.01)
    b = aslam_gpu.Batch2D(inp, r_max_m=12.0, noise_sigma_m=0.01)
    dev = a.device
    abuf = torch.zeros(16, 2, device=dev)
    rew = torch.zeros(16, device=dev)
    obs = torch.zeros(16, b.b_max + 2, device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.capture_graph(abuf, None, rew, obs, stream=s)
    for k in range(5):
        at = torch.from_numpy(acts[k]).to(dev)
        a.step(at)
        abuf.copy_(at)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            b.graph_step(stream=s)
        s.synchronize()
        assert torch.equal(a.state()["belief"], b.state()["belief"])
        assert torch.equal(a.observe(), obs)
        assert torch.equal(a.reward(), rew)


def test_checkpoint_resume_is_bit_exact(aslam_gpu):
    inp = synth.paper_scale(E=8, seed=11)
    acts = synth.random_actions(6, 8, 4)
    g = aslam_gpu.Batch2D(inp, r_max_m=12.0, noise_sigma_m=0.01)
    dev = g.device
    for k in range(3):
        g.step(torch.from_numpy(acts[k]).to(dev))
    buf = g.save_state()
    for k in range(3, 6):
        g.step(torch.from_numpy(acts[k]).to(dev))
    ref = g.state()["belief"].clone(), g.observe().clone()
    g.load_state(buf)
    for k in range(3, 6):
        g.step(torch.from_numpy(acts[k]).to(dev))
    assert torch.equal(g.state()["belief"], ref[0])
    assert torch.equal(g.observe(), ref[1])


def test_autotune_then_parity(aslam_gpu, orc):
    inp = synth.paper_scale(E=12, seed=21)
    g = aslam_gpu.Batch2D(inp, r_max_m=12.0, noise_sigma_m=0.01, flags=aslam_gpu.FLAG_DEBUG)
    blk, win = g.autotune()
    assert blk % 32 == 0 and win >= 64
    ob = orc.OracleBatch2D(inp, **orc_params(dict(r_max_m=12.0, noise_sigma_m=0.01)))
    acts = synth.random_actions(3, 12, 6)
    for k in range(3):
        g.step(torch.from_numpy(acts[k]).cuda())
        torch.cuda.synchronize()
        o = ob.step(acts[k], counts=True)
        compare_step(g, ob, o, tag="tuned %d" % k)


def test_reset_mask_and_observe(aslam_gpu, orc):
    inp = synth.paper_scale(E=4, W=64, B=45, seed=3)
    g = aslam_gpu.Batch2D(inp, r_max_m=3.0, noise_sigma_m=0.0)
    dev = g.device
    z = torch.zeros(4, 2, device=dev)
    g.step(z)
    g.reset(torch.tensor([0, 1, 0, 1], dtype=torch.uint8, device=dev))
    g.step(z)
    st = g.state()
    assert st["ep"].cpu().tolist() == [0, 1, 0, 1]
    assert st["t"].cpu().tolist() == [2, 1, 2, 1]
    obs = g.observe().cpu().numpy()
    zz = st["z"].cpu().numpy()
    for e in range(4):
        np.testing.assert_array_equal(obs[e, :45], zz[g.ray_off[e]:g.ray_off[e] + 45])
        assert obs[e, 45] == st["th"].cpu().numpy()[e]
    g.sync_status()


@pytest.mark.parametrize("sigma,window", [(0.3, 0), (0.3, 64), (0.08, 0)])
def test_large_noise_moves_endpoint_far_from_hit(aslam_gpu, orc, sigma, window):
    """Noise of several cells: endpoints both far before the hit cell (the
    committed misses past it must be removed) and far beyond it."""
    inp = synth.paper_scale(E=4, seed=606)
    acts = synth.random_actions(4, 4, 60)
    run_parity(aslam_gpu, orc, inp, acts, tag="noise-%g-%d" % (sigma, window), r_max_m=12.0,
               noise_sigma_m=sigma, gpu_kw=dict(window_cells=window))


def test_env_base_shard_draws_the_global_noise(aslam_gpu, orc):
    """Envs [3, 6) of a 6-env set in a batch of their own with env_base = 3
    match the oracle stepping those envs under their global ids 3..5."""
    part = synth.paper_scale(E=6, W=128, B=90, seed=55, envs=range(3, 6))
    acts = synth.random_actions(5, 6, 4)[:, 3:]
    gb = aslam_gpu.Batch2D(part, flags=aslam_gpu.FLAG_DEBUG, env_base=3, r_max_m=6.0,
                           noise_sigma_m=0.02)
    ob = orc.OracleBatch2D(part, env_ids=np.arange(3, 6), r_max=6.0, sigma=0.02)
    for s in range(acts.shape[0]):
        gb.step(torch.from_numpy(acts[s]).cuda())
        torch.cuda.synchronize()
        compare_step(gb, ob, ob.step(acts[s], counts=True), tag="env_base step %d" % s)
    with pytest.raises(aslam_gpu.AslamError):
        aslam_gpu.Batch2D(part, env_base=-1, r_max_m=6.0)

