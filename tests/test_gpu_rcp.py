"""The channel functions' reciprocal (hardware approximation + two
Newton-Raphson steps) against the IEEE division on the device: at most 2 ulp
over the magnitudes the continued fractions produce, and the same sign; the
FP32 solve's pivot reciprocal (hardware approximation + one step) within one
ulp of the correctly rounded reciprocal over the normal range."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so = str(tmp_path_factory.mktemp("rcp") / "rcp_check.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                    "-Xcompiler", "-fPIC", "-o", so, os.path.join(HERE, "cuda", "rcp_check.cu")],
                   check=True)
    L = ctypes.CDLL(so)
    L.rcp_pair.restype = ctypes.c_int
    L.rcp_pair.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.rcp_pair_f32.restype = ctypes.c_int
    L.rcp_pair_f32.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return L


def test_rcp_within_two_ulp(lib):
    rng = np.random.default_rng(11)
    n = 1 << 20
    x = np.concatenate([
        rng.uniform(-1.0, 1.0, n // 4) * 10.0 ** rng.uniform(-300, 300, n // 4),
        rng.uniform(0.5, 2.0, n // 4),
        np.arange(1, n // 4 + 1, dtype=np.float64),          # integers (l + n)
        -rng.uniform(1e-300, 1e-290, n // 4),
    ])
    x = np.ascontiguousarray(x[np.abs(x) > 1e-300])
    r_nr = np.empty_like(x)
    r_div = np.empty_like(x)
    assert lib.rcp_pair(x.ctypes.data, x.size, r_nr.ctypes.data, r_div.ctypes.data) == 0
    assert np.array_equal(np.sign(r_nr), np.sign(r_div))
    ulp = np.spacing(np.abs(r_div))
    assert np.max(np.abs(r_nr - r_div) / ulp) <= 2.0


def test_rcp_f32_within_one_ulp(lib):
    rng = np.random.default_rng(12)
    n = 1 << 20
    x = np.concatenate([
        rng.uniform(-1.0, 1.0, n // 2) * 10.0 ** rng.uniform(-37, 37, n // 2),
        rng.uniform(1.0, 8.0, n // 4),                         # |d|^2 of the scaled complex pivots
        np.float32(1.0) + np.arange(n // 4) * np.float32(2.0 ** -23),   # consecutive floats above 1
    ]).astype(np.float32)
    x = np.ascontiguousarray(x[np.abs(x) >= np.finfo(np.float32).tiny])
    r_nr = np.empty_like(x)
    r_rn = np.empty_like(x)
    assert lib.rcp_pair_f32(x.ctypes.data, x.size, r_nr.ctypes.data, r_rn.ctypes.data) == 0
    assert np.all(np.isfinite(r_nr)) and np.array_equal(np.sign(r_nr), np.sign(r_rn))
    ulp = np.spacing(np.abs(r_rn))
    assert np.max(np.abs(r_nr.astype(np.float64) - r_rn) / ulp) <= 1.0
