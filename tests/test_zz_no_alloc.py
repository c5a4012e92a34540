"""The allocation-free scan update (for callers that may not allocate device
memory) against the batched step, through the C ABI.

aslam_scan_update_noalloc keeps its counters in a fixed array inside the
library instead of a caller-allocated workspace.  A robot given a zero action
does not move, so one aslam_step integrates exactly one scan from the spawn
pose; two such steps in a row must give the same ranges and the same int16
log-odds as two no-alloc calls with the same poses and noise counters (both
bit-exact, as in the other parity tests).  The second configuration is the
paper's sensor (front 180 degrees, minimum range, ranges to two decimals) on
maps of three different sizes, which exercises the entry point's own copies
of the front-arc beam table, the range quantisation and the per-env offsets.
"""
import math

import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = {
    "full-turn": (lambda: synth.paper_scale(E=6, W=128, B=180, seed=4321),
                  dict(r_max_m=6.0, noise_sigma_m=0.01)),
    "paper-sensor-uneven": (lambda: synth.uneven(E=6, sides=(96, 128, 160), beams=(128,),
                                                 seed=8765),
                            dict(fov_rad=math.pi, r_min_m=0.1, range_decimals=2, r_max_m=10.0,
                                 noise_sigma_m=0.01)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_scan_update_matches_step_twice(aslam_gpu, case):
    aslam = aslam_gpu
    make, cfg = CASES[case]
    inp = make()
    E, B = inp.n_envs, int(inp.n_beams[0])
    assert np.all(inp.n_beams == B)
    batch = aslam.Batch2D(inp, **cfg)
    dev = batch.device
    gt = torch.from_numpy(inp.gt).to(dev)
    pose = torch.from_numpy(np.ascontiguousarray(inp.spawn[:, 0, :])).to(dev)
    belief = torch.zeros(int(inp.map_off[-1]), dtype=torch.int16, device=dev)
    ranges = torch.empty(E, B, dtype=torch.float32, device=dev)
    zero = torch.zeros(E, 2, device=dev)
    for call in range(2):
        batch.step(zero)
        step = torch.full((E,), call, dtype=torch.int32, device=dev)
        aslam.scan_update_noalloc(inp, gt, pose, step, belief, ranges, **cfg)
        torch.cuda.synchronize()
        st = batch.state()
        assert int(st["done"].sum()) == 0
        z = st["z"].cpu().numpy()
        got = ranges.cpu().numpy()
        for e in range(E):
            np.testing.assert_array_equal(got[e], z[batch.ray_off[e]:batch.ray_off[e] + B])
            a, b = int(inp.map_off[e]), int(inp.map_off[e + 1])
            np.testing.assert_array_equal(belief[a:b].view(int(inp.map_h[e]), int(inp.map_w[e])).cpu(),
                                          batch.env_belief(e).cpu())
        assert int((belief != 0).sum()) > 0


def test_noalloc_rejects_oversized_requests(aslam_gpu):
    aslam = aslam_gpu
    occ = np.zeros((2048, 2100), np.uint8)
    inp = synth.custom_2d([occ], [8], 0.05, np.zeros((1, 1, 3), np.float32))
    dev = torch.device("cuda")
    with pytest.raises(aslam.AslamError, match="static scratch maximum"):
        aslam.scan_update_noalloc(inp, torch.zeros(occ.size, dtype=torch.uint8, device=dev),
                                  torch.zeros(1, 3, device=dev),
                                  torch.zeros(1, dtype=torch.int32, device=dev),
                                  torch.zeros(occ.size, dtype=torch.int16, device=dev),
                                  torch.zeros(1, 8, device=dev))


def test_noalloc_rejects_wrong_buffers_and_capture(aslam_gpu):
    """Buffers of the wrong dtype or size are refused before any launch, and a
    call on a stream that is being captured is refused by the library."""
    aslam = aslam_gpu
    inp = synth.paper_scale(E=2, W=64, B=16, seed=12)
    dev = torch.device("cuda")
    n = int(inp.map_off[-1])
    gt = torch.from_numpy(inp.gt).to(dev)
    pose = torch.from_numpy(np.ascontiguousarray(inp.spawn[:, 0, :])).to(dev)
    step = torch.zeros(2, dtype=torch.int32, device=dev)
    belief = torch.zeros(n, dtype=torch.int16, device=dev)
    ranges = torch.empty(2, 16, device=dev)
    with pytest.raises(aslam.AslamError, match="belief must be torch.int16"):
        aslam.scan_update_noalloc(inp, gt, pose, step, belief.float(), ranges)
    with pytest.raises(aslam.AslamError, match="belief must have"):
        aslam.scan_update_noalloc(inp, gt, pose, step, belief[:-1], ranges)
    with pytest.raises(aslam.AslamError, match="ranges must have"):
        aslam.scan_update_noalloc(inp, gt, pose, step, belief, ranges[:1])
    with pytest.raises(aslam.AslamError, match="pose must be"):
        aslam.scan_update_noalloc(inp, gt, pose.double(), step, belief, ranges)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device=dev)
    torch.cuda.synchronize()
    err = None
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        try:
            aslam.scan_update_noalloc(inp, gt, pose, step, belief, ranges, stream=s)
        except aslam.AslamError as ex:
            err = ex
    assert err is not None and "captured" in str(err)
    assert int((belief != 0).sum()) == 0
