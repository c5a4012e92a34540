"""Failure detection on the GPU without a GPU fault (through the C ABI).

* ASLAM_FLAG_CHECKS turns on index checks in the 2-D sensing and update walks
  (a failed check records the sticky error word and skips the access; no
  kernel traps): with every check passing, the step is bit-identical to the
  oracle, as without the flag, and aslam_sync_status reports success.
* Non-finite inputs injected by the host: a NaN or infinite action is clamped
  to a defined value on both sides (fmaxf / fminf return the non-NaN
  operand), so the step still matches the oracle; with ASLAM_FLAG_CHECKS the
  batch also reports it through aslam_sync_status as ASLAM_ERR_DEVICE, and a
  non-finite U_t likewise.  The batch stays usable after the report.
"""
import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import synth
from tests.parity_util import compare_step, orc_params, run_parity
from tests.test_parity_step2d import edge_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["paper", "uneven-window", "edge"])
def test_checks_flag_leaves_results_unchanged(aslam_gpu, orc, case):
    aslam = aslam_gpu
    if case == "paper":
        inp, kw = synth.paper_scale(E=4, seed=31), {}
    elif case == "uneven-window":
        inp, kw = synth.uneven(E=8, seed=32), dict(window_cells=128)
    else:
        inp, kw = edge_inputs(), {}
    E = inp.n_envs
    acts = synth.random_actions(4, E, 33, v_max=0.3)
    gb, _ = run_parity(aslam, orc, inp, acts, tag="checks-" + case, r_max_m=6.0,
                       noise_sigma_m=0.01, gpu_kw=dict(kw, flags=aslam.FLAG_CHECKS))
    gb.sync_status()


def bad_actions(E):
    a = synth.random_actions(1, E, 9)[0].copy()
    a[0] = [np.nan, 0.5]
    a[1] = [0.3, np.nan]
    a[2] = [np.inf, -np.inf]
    a[3] = [-np.inf, np.inf]
    return a


@pytest.mark.parametrize("checks", [False, True])
def test_nonfinite_actions_are_clamped_and_reported(aslam_gpu, orc, checks):
    aslam = aslam_gpu
    inp = synth.paper_scale(E=5, W=128, B=90, seed=41)
    cfg = dict(r_max_m=6.0, noise_sigma_m=0.01)
    flags = aslam.FLAG_DEBUG | (aslam.FLAG_CHECKS if checks else 0)
    gb = aslam.Batch2D(inp, flags=flags, **cfg)
    ob = orc.OracleBatch2D(inp, **orc_params(cfg))
    a = bad_actions(5)
    gb.step(torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    compare_step(gb, ob, ob.step(a, counts=True), tag="nonfinite actions")
    if checks:
        with pytest.raises(aslam.AslamError) as ei:
            gb.sync_status()
        assert ei.value.status == 7
    else:
        gb.sync_status()
    # the batch goes on stepping after the report
    good = synth.random_actions(1, 5, 10)[0]
    gb.step(torch.from_numpy(good).cuda())
    torch.cuda.synchronize()
    compare_step(gb, ob, ob.step(good, counts=True), tag="after report")


def test_nonfinite_u_is_reported(aslam_gpu):
    aslam = aslam_gpu
    inp = synth.paper_scale(E=3, W=64, B=45, seed=42)
    gb = aslam.Batch2D(inp, flags=aslam.FLAG_CHECKS, r_max_m=3.0, reward_mode=1)
    z = torch.zeros(3, 2, device="cuda")
    gb.step(z, torch.tensor([0.1, 0.2, 0.3], device="cuda"))
    gb.sync_status()
    gb.step(z, torch.tensor([0.1, float("nan"), 0.3], device="cuda"))
    with pytest.raises(aslam.AslamError) as ei:
        gb.sync_status()
    assert ei.value.status == 7
    r = gb.reward().cpu().numpy()
    assert np.isfinite(r[0]) and np.isfinite(r[2])
