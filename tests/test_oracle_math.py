"""Pins of the oracle's deterministic elementary functions and random draws.

The sensor model of Sec. IV-A adds N(0, sigma^2) noise to every range; the
oracle draws it with Philox4x32-10 and Box-Muller on its own fp32 log and
cos.  These tests tie those functions to libm (fp64) and to the normal
distribution, independently of the oracle's own code.
"""
import math

import numpy as np
import pytest


def ulp_err(got, ref):
    ref32 = np.float32(ref)
    spacing = np.spacing(np.abs(ref32)) if ref32 != 0 else np.float32(1.4e-45)
    return abs(float(got) - ref) / float(spacing)


def test_sincos_close_to_libm(orc):
    xs = np.linspace(-8.0, 8.0, 4001, dtype=np.float32)
    worst = 0.0
    for x in xs:
        s, c = orc.sincosf(float(x))
        es = abs(s - math.sin(float(x)))
        ec = abs(c - math.cos(float(x)))
        worst = max(worst, es, ec)
    # a few fp32 ulps of 1.0
    assert worst < 4e-7


def test_sincos_special_values(orc):
    s, c = orc.sincosf(0.0)
    assert s == 0.0 and c == 1.0
    # quadrant symmetry: sin(-x) = -sin(x), cos(-x) = cos(x)
    for x in [0.1, 0.7, 1.3, 2.9, 3.14159]:
        s1, c1 = orc.sincosf(x)
        s2, c2 = orc.sincosf(-x)
        assert s1 == -s2 and c1 == c2
    # Pythagoras to fp32 accuracy
    for x in np.linspace(-3.2, 3.2, 97):
        s, c = orc.sincosf(float(x))
        assert abs(s * s + c * c - 1.0) < 1e-6


def test_log_close_to_libm(orc):
    us = np.concatenate([np.arange(1, 5000) / 16777216.0,
                         np.linspace(1e-3, 1.0, 5000)]).astype(np.float32)
    worst = 0.0
    for u in us:
        got = orc.logf(float(u))
        ref = math.log(float(u))
        worst = max(worst, ulp_err(got, ref))
    assert worst <= 3.0
    assert orc.logf(1.0) == 0.0
    assert orc.logf(0.5) == np.float32(-math.log(2.0))


def test_cos2pi_close_to_libm(orc):
    us = (np.arange(0, 1 << 12) / float(1 << 12)).astype(np.float32)
    worst = max(abs(orc.cos2pi(float(u)) - math.cos(2 * math.pi * float(u))) for u in us)
    assert worst < 3e-7
    assert orc.cos2pi(0.0) == 1.0
    assert orc.cos2pi(0.5) == -1.0
    assert orc.cos2pi(0.25) == 0.0 or abs(orc.cos2pi(0.25)) < 1e-7


def test_philox_uniformity_and_avalanche(orc):
    rng = np.random.default_rng(1)
    words = []
    for k in range(4000):
        words.append(orc.philox([k, 7, 3, 0], [0x1234, 0x5678]))
    w = np.asarray(words, dtype=np.uint64).reshape(-1)
    u = w / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.005
    # byte histogram, chi-square with 255 dof (p ~ 1e-6 threshold ~ 360)
    by = np.concatenate([(w >> s) & 0xFF for s in (0, 8, 16, 24)]).astype(np.int64)
    hist = np.bincount(by, minlength=256)
    expct = by.size / 256
    chi2 = ((hist - expct) ** 2 / expct).sum()
    assert chi2 < 360
    # avalanche: one flipped counter bit changes about half the 128 output bits
    flips = []
    for k in range(300):
        c = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        a = orc.philox(c, key)
        bit = int(rng.integers(0, 128))
        c2 = list(c)
        c2[bit // 32] ^= 1 << (bit % 32)
        b = orc.philox(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68
    # distinct keys give distinct streams
    assert not np.array_equal(orc.philox([0, 0, 0, 0], [1, 0]), orc.philox([0, 0, 0, 0], [2, 0]))


def test_gauss_is_standard_normal(orc):
    from scipy import stats
    n = [orc.gauss(20260325, e, s, b) for e in range(5) for s in range(40) for b in range(100)]
    n = np.asarray(n, dtype=np.float64)
    assert abs(n.mean()) < 0.03
    assert abs(n.std() - 1.0) < 0.03
    ks = stats.kstest(n, "norm")
    assert ks.pvalue > 1e-4
    assert np.all(np.isfinite(n))
