"""GPU parity of the batched fixed-lag window Gauss-Newton (Sec. III-D,
Eq. 5-6) through the C ABI against the oracle.  The kernel eliminates the
block-tridiagonal system in fp64; the oracle inverts the dense system in
fp64 (Gauss-Jordan).  Both start from the same fp32 inputs, so the windows
agree to fp64 rounding before the fp32 store: poses within 4 fp32 ulps of
their magnitude (plus 1e-9), covariances and U within 1e-6 relative."""
import math

import numpy as np
import pytest
import torch

from paper_2603_25834_gb300 import aslam
from tests.test_oracle_flgn import odometry, trajectory

pytestmark = pytest.mark.gpu


def problem(E, L, seed):
    rng = np.random.default_rng(seed)
    xt = np.stack([trajectory(rng, L) for _ in range(E)])
    odo = np.stack([odometry(x) for x in xt]).reshape(E, max(L - 1, 0), 3)
    odo = odo + rng.normal(0, [0.004, 0.004, 0.003], size=odo.shape)
    meas = xt + rng.normal(0, [0.01, 0.01, 0.005], size=xt.shape)
    info = np.zeros((E, L, 3))
    pick = rng.random((E, L)) < 0.4
    info[pick] = rng.uniform(1e3, 1e4, size=(pick.sum(), 3))
    x0 = xt + rng.normal(0, [0.03, 0.03, 0.02], size=xt.shape)
    prior = xt[:, 0] + rng.normal(0, 0.01, size=(E, 3))
    pinfo = np.full((E, 3), 1e3)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return f(x0), f(odo), f(meas), f(info), f(prior), f(pinfo)


@pytest.mark.parametrize("E,L,iters", [(200, 8, 4), (33, 16, 2), (17, 1, 3), (9, 2, 0)])
def test_fixed_lag_gn_matches_oracle(aslam_gpu, orc, E, L, iters):
    x0, odo, meas, info, prior, pinfo = problem(E, L, E + L)
    wo = np.float32([2e3, 2e3, 5e3])
    dev = lambda a: torch.from_numpy(a).cuda()
    x = dev(x0.copy())
    cov, u, st = aslam.fixed_lag_gn(x, dev(odo) if L > 1 else dev(np.zeros((E, 1, 3), np.float32)),
                                    dev(meas), dev(info), dev(prior), dev(pinfo), iters=iters,
                                    odo_info=wo, u_scale=1e-4)
    x, cov, u, st = x.cpu().numpy(), cov.cpu().numpy(), u.cpu().numpy(), st.cpu().numpy()
    for e in range(E):
        rx, rc, rs = orc.fixed_lag_gn(x0[e].astype(np.float64), odo[e].astype(np.float64),
                                      meas[e].astype(np.float64), info[e].astype(np.float64),
                                      prior[e].astype(np.float64), pinfo[e].astype(np.float64),
                                      wo.astype(np.float64), iters=iters)
        assert st[e] == (0 if rs == 0 else 1)
        tol = 4 * np.spacing(np.abs(rx).astype(np.float32)).astype(np.float64) + 1e-9
        assert np.all(np.abs(x[e] - rx) <= tol), e
        np.testing.assert_allclose(cov[e], rc, rtol=1e-6, atol=1e-6 * np.abs(rc).max())
        U = np.cbrt(np.linalg.det(rc)) / 1e-4
        assert u[e] == pytest.approx(U, rel=1e-6)


def test_singular_window_reports_status(aslam_gpu, orc):
    # a one-pose window without any factor: the normal matrix is exactly zero
    E, L = 4, 1
    x0, odo, meas, info, prior, pinfo = problem(E, L, 77)
    info[:] = 0.0
    pinfo[:] = 0.0
    dev = lambda a: torch.from_numpy(a).cuda()
    x = dev(x0.copy())
    cov, u, st = aslam.fixed_lag_gn(x, dev(np.zeros((E, 1, 3), np.float32)), dev(meas), dev(info),
                                    dev(prior), dev(pinfo))
    assert torch.all(st == 1) and torch.isnan(u).all()
    _, _, rs = orc.fixed_lag_gn(x0[0].astype(np.float64), np.zeros((0, 3)), meas[0], info[0],
                                prior[0], pinfo[0], [1e4] * 3)
    assert rs != 0
