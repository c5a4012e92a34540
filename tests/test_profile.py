"""Per-kernel timing of the step through the C ABI (aslam_profile_begin/end).

The timed steps must stay bit-identical to untimed ones (the events only
bracket the launches), every kernel of the step must report a positive
device time, and only the requested number of steps is timed.
"""
import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(aslam, inp, acts, profile, **cfg):
    b = aslam.Batch2D(inp, **cfg)
    a = torch.from_numpy(acts).cuda()
    if profile:
        b.profile_begin(3)
    for k in range(acts.shape[0]):
        b.step(a[k])
    out = b.profile_end() if profile else None
    torch.cuda.synchronize()
    belief = b.state()["belief"].cpu().numpy().copy()
    b.close()
    return belief, out


@pytest.mark.parametrize("dims", [2, 3])
def test_profile_names_counts_and_no_side_effects(aslam_gpu, dims):
    if dims == 2:
        inp = synth.paper_scale(E=8, W=128, B=90, seed=31)
        cfg = dict(r_max_m=6.0, noise_sigma_m=0.01)
        names = ["sense2d_kernel", "update2d_kernel"]
    else:
        inp = synth.voxel_batch(E=4, W=32, H=32, D=8, n_az=32, K=2)
        cfg = dict(r_max_m=4.0, noise_sigma_m=0.01, n_rings=4)
        names = ["step3d_kernel"]
    acts = synth.random_actions(5, inp.map_w.size, 3)
    ref, _ = _run(aslam_gpu, inp, acts, False, **cfg)
    got, (ms, n_steps) = _run(aslam_gpu, inp, acts, True, **cfg)
    assert np.array_equal(ref, got)
    assert n_steps == 3
    assert list(ms) == names
    assert all(v > 0.0 for v in ms.values())


def test_profile_end_without_begin_is_an_error(aslam_gpu):
    b = aslam_gpu.Batch2D(synth.plain_1env(), r_max_m=5.0)
    with pytest.raises(aslam_gpu.AslamError):
        b.profile_end()
    with pytest.raises(aslam_gpu.AslamError):
        b.profile_begin(0)
    b.close()
