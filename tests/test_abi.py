"""C-ABI library: builds, loads, exports every declared symbol (CPU only).

No compute call is made here; on a machine without a GPU rm_create must fail
cleanly with RM_ECUDA rather than crash.
"""
import ctypes
import os
import re

import pytest

from paper_1909_07321_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmgb.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rm_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def so():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_boundary():
    names = _declared()
    for must in ["rm_create", "rm_destroy", "rm_load_poles", "rm_set_channels",
                 "rm_solve_energies", "rm_collision_strengths", "rm_strerror", "rm_last_error"]:
        assert must in names


def test_every_declared_symbol_exported(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_strerror_and_defaults(so):
    from paper_1909_07321_gb300 import rmgb
    for code in [0, -1, -2, -3, -4, -5, -6, -7, 1, 2, 3, 4, 99]:
        assert isinstance(rmgb.rm_strerror(code), str) and rmgb.rm_strerror(code)
    o = rmgb.rm_default_opts()
    assert o.precision == rmgb.RM_FP64 and o.eps_thr == 1e-10 and o.delta_pole == 1e-3
    assert o.nu_margin == 0.1 and o.fnumin == 0.0


def test_create_without_gpu_fails_cleanly(so):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1909_07321_gb300 import rmgb
    with pytest.raises(rmgb.RmError) as ei:
        rmgb.rm_create()
    assert ei.value.code in (rmgb.RM_ECUDA, rmgb.RM_EINVAL)


def test_null_context_is_rejected(so):
    from paper_1909_07321_gb300 import rmgb
    L = rmgb.lib()
    assert L.rm_solve_energies(None, 0, 1, None, 0, None, None, None) == rmgb.RM_EINVAL
    assert L.rm_collision_strengths(None, None, 0) == rmgb.RM_EINVAL
    assert L.rm_sync(None) == rmgb.RM_EINVAL
    L.rm_destroy(None)
    assert L.rm_last_error(None)


def test_null_context_rejected_by_new_calls(so):
    from paper_1909_07321_gb300 import rmgb
    L = rmgb.lib()
    assert L.rm_set_multipoles(None, 0, 1, None, 10.0, 100) == rmgb.RM_EINVAL
    assert L.rm_collision_strengths_async(None, None, 0) == rmgb.RM_EINVAL


def test_null_context_rejected_by_lane_calls(so):
    from paper_1909_07321_gb300 import rmgb
    L = rmgb.lib()
    assert L.rm_lane_solve_energies(None, 0, 0, 1, None, 0, None, None, None) == rmgb.RM_EINVAL
    assert L.rm_lane_collision_strengths(None, 0, None, 0) == rmgb.RM_EINVAL
    assert L.rm_lane_query(None, 0) == rmgb.RM_EINVAL
    assert L.rm_lane_sync(None, 0) == rmgb.RM_EINVAL
    assert L.rm_lane_stream(None, 0) is None
    assert L.rm_lane_reserve(None, 0, 0, 1, None) == rmgb.RM_EINVAL
    assert L.rm_pw_bytes(None, 0, None) == rmgb.RM_EINVAL
    assert L.rm_unload_pw(None, 0) == rmgb.RM_EINVAL
    assert L.rm_solve_batch(None, 1, None, 1, None, 0, 1) == rmgb.RM_EINVAL
    assert L.rm_autotune_info(None, 0, None, None, None, None) == rmgb.RM_EINVAL
    o = rmgb.rm_default_opts()
    assert o.lanes == 1 and o.autotune == 0


def test_multipole_shape_checked_before_the_library(so):
    """The binding rejects coefficients that do not match the loaded wave's
    channel count (the C call reads lambda_max n^2 doubles) without calling
    the library."""
    import numpy as np
    from paper_1909_07321_gb300 import rmgb
    ctx = rmgb.Context.__new__(rmgb.Context)
    ctx.h = None
    ctx._n_ch = {0: 4}
    for bad in (np.zeros((2, 3, 3)), np.zeros((4, 4)), np.zeros((1, 4, 5))):
        with pytest.raises(ValueError):
            ctx.set_multipoles(0, bad, 15.0, 100)
