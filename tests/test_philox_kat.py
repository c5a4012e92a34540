"""Known-answer pins of the oracle's Philox4x32-10 (the range-noise
generator, Sec. IV-A Gaussian noise) against two implementations of the
published generator that share nothing with this repository:

  * on the host, PyTorch's header-only Philox engine (ATen), compiled here
    with g++ (runs with `-m "not gpu"`);
  * on the GPU, cuRAND's device function curand_Philox4x32_10, compiled with
    nvcc for sm_103a (`-m gpu`).

Every output word must be bit-identical.  A wrong multiplier, Weyl constant,
word order or key schedule in the oracle fails both.  The CUDA path's own
generator is pinned to the oracle bit for bit by the Gaussian draws of
test_parity_step2d.py::test_detmath_bit_equal_to_oracle.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def pairs(n, seed=20260325):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # structured cases: zero and all-ones words, the noise counter layout
    # (beam, env, step, 0) under the default key, single set bits
    special_c = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 0x80000000],
                 [359, 749, 999, 0], [0, 0, 0, 0]]
    special_k = [[0, 0], [0xFFFFFFFF] * 2, [0, 0], [0, 0], [20260325, 0], [0x9E3779B9, 0xBB67AE85]]
    ctr[:len(special_c)] = np.asarray(special_c, np.uint32)
    key[:len(special_k)] = np.asarray(special_k, np.uint32)
    return np.ascontiguousarray(ctr), np.ascontiguousarray(key)


def oracle_words(orc, ctr, key):
    return np.stack([orc.philox(c, k) for c, k in zip(ctr, key)])


def test_oracle_philox_matches_aten_engine(orc, tmp_path):
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("this PyTorch ships no ATen/core/PhiloxRNGEngine.h")
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    so = str(tmp_path / "aten_philox.so")
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", inc,
                           os.path.join(HERE, "kat", "aten_philox.cpp"), "-o", so])
    lib = C.CDLL(so)
    lib.aten_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    ctr, key = pairs(20000)
    out = np.zeros_like(ctr)
    lib.aten_philox4x32_10(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, len(ctr))
    np.testing.assert_array_equal(oracle_words(orc, ctr, key), out)


@pytest.mark.gpu
def test_oracle_philox_matches_curand(orc, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu-marked test run without a CUDA device")
    from paper_2603_25834_gb300 import build
    so = str(tmp_path / "curand_philox.so")
    subprocess.check_call([build.nvcc(), *build.ARCH, "-O2", "-shared", "-Xcompiler", "-fPIC",
                           os.path.join(HERE, "kat", "curand_philox.cu"), "-o", so])
    lib = C.CDLL(so)
    lib.curand_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.curand_philox4x32_10.restype = C.c_int
    ctr, key = pairs(10000, seed=7)
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    dk = torch.from_numpy(key.view(np.int32)).cuda()
    do = torch.zeros_like(dc)
    torch.cuda.synchronize()
    assert lib.curand_philox4x32_10(dc.data_ptr(), dk.data_ptr(), do.data_ptr(), len(ctr)) == 0
    got = do.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(oracle_words(orc, ctr, key), got)
