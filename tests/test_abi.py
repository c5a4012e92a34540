"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and rejects bad arguments on the host before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(aslam\w*)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2603_25834_gb300 import aslam
    return aslam.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2603_25834_gb300 import aslam
    missing = declared_functions() - set(aslam.EXPORTS) - set(getattr(aslam, "EXPORTS_EXTRA", {}))
    assert not missing, missing


def small_config(aslam, **kw):
    c = aslam.config_defaults()
    w = np.array([16, 24], np.int32)
    h = np.array([16, 8], np.int32)
    b = np.array([8, 0], np.int32)
    c.n_envs = 2
    c.h_map_w = w.ctypes.data_as(C.c_void_p)
    c.h_map_h = h.ctypes.data_as(C.c_void_p)
    c.h_n_beams = b.ctypes.data_as(C.c_void_p)
    for k, v in kw.items():
        setattr(c, k, v)
    return c, (w, h, b)


def test_config_and_workspace_size(lib):
    from paper_2603_25834_gb300 import aslam
    c, keep = small_config(aslam)
    n = C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n)) == 0
    assert n.value > 16 * 16 * 2 and n.value % 256 == 0
    c.flags = aslam.FLAG_DEBUG
    n2 = C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n2)) == 0
    assert n2.value > n.value


@pytest.mark.parametrize("field,value", [
    ("n_envs", 0), ("res_m", 0.0), ("r_max_m", -1.0), ("l_clamp_q", 0), ("t_episode", 0),
    ("d_full", 0.1), ("kappa", 0.0), ("reward_mode", 7), ("threads_per_cta", 100),
    ("window_cells", 60), ("struct_size", 12), ("dims", 5), ("n_spawn", 0),
])
def test_invalid_configs_are_rejected_on_the_host(lib, field, value):
    from paper_2603_25834_gb300 import aslam
    c, keep = small_config(aslam, **{field: value})
    n = C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n)) == 1
    assert lib.aslam_last_error(None)


def test_bad_beam_count_and_map_side(lib):
    from paper_2603_25834_gb300 import aslam
    c, keep = small_config(aslam)
    keep[2][0] = 5000
    n = C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n)) == 1
    keep[2][0] = 8
    keep[0][1] = 0
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n)) == 1


def test_create_rejects_missing_or_misaligned_workspace(lib):
    from paper_2603_25834_gb300 import aslam
    c, keep = small_config(aslam)
    off = np.array([0, 256, 448], np.int64)
    out = C.c_void_p()
    rc = lib.aslam_create_batch(C.byref(c), None, 1 << 20, C.c_void_p(16), off.ctypes.data_as(
        C.c_void_p), C.c_void_p(16), None, C.byref(out))
    assert rc == 3 and not out.value
    rc = lib.aslam_create_batch(C.byref(c), C.c_void_p(4096 + 8), 1 << 20, C.c_void_p(16),
                                off.ctypes.data_as(C.c_void_p), C.c_void_p(16), None, C.byref(out))
    assert rc == 3
    rc = lib.aslam_create_batch(C.byref(c), C.c_void_p(4096), 1 << 20, None,
                                off.ctypes.data_as(C.c_void_p), C.c_void_p(16), None, C.byref(out))
    assert rc == 1


def test_status_strings(lib):
    for s in range(8):
        assert lib.aslam_status_string(s)
    assert lib.aslam_graph_step(None, None) == 1
    assert lib.aslam_step(None, None, None, None) == 1


@pytest.mark.parametrize("field", ["res_m", "r_max_m", "noise_sigma_m", "dt_s", "v_max",
                                   "w_max", "lam_col", "lam_abs", "kappa", "d_crash",
                                   "visit_cell_m", "uq_u_scale", "sensor_z_m"])
@pytest.mark.parametrize("value", [float("nan"), float("inf"), float("-inf")])
def test_nonfinite_config_values_are_rejected(lib, field, value):
    """Fault injection on the host: a NaN or infinite constant never reaches a
    kernel (fields whose sign checks +Inf would pass included)."""
    from paper_2603_25834_gb300 import aslam
    c, keep = small_config(aslam, **{field: value})
    n = C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n)) == 1
    assert b"NaN or infinite" in lib.aslam_last_error(None)


def test_timeout_status_is_reserved(lib):
    """No kernel of this build waits on another: the status exists in the ABI
    (value 4) with its string, but no call returns it."""
    assert lib.aslam_status_string(4)
    assert b"reserved" in lib.aslam_status_string(4)
    for f in os.listdir(os.path.join(ROOT, "paper_2603_25834_gb300", "csrc")):
        src = open(os.path.join(ROOT, "paper_2603_25834_gb300", "csrc", f)).read()
        assert "return ASLAM_ERR_TIMEOUT" not in src and "kErrTimeout" not in src, f


@pytest.mark.parametrize("iters", [-1, 11])
def test_scan_to_map_iterations_out_of_range_are_rejected(lib, iters):
    from paper_2603_25834_gb300 import aslam
    c, keep = small_config(aslam, u_mode=aslam.U_FIXEDLAG, slam_gn_iters=iters)
    n = C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c), C.byref(n)) == 1
    assert b"slam_gn_iters" in lib.aslam_last_error(None)


def test_scan_to_map_correction_adds_its_workspace(lib):
    from paper_2603_25834_gb300 import aslam
    c0, keep0 = small_config(aslam, u_mode=aslam.U_FIXEDLAG)
    c1, keep1 = small_config(aslam, u_mode=aslam.U_FIXEDLAG, slam_gn_iters=2)
    n0, n1 = C.c_size_t(), C.c_size_t()
    assert lib.aslam_workspace_bytes(C.byref(c0), C.byref(n0)) == 0
    assert lib.aslam_workspace_bytes(C.byref(c1), C.byref(n1)) == 0
    assert n1.value > n0.value          # the corrected poses and the beams' fp64 directions
