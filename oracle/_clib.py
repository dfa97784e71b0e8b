"""Build and load the oracle's binary128 C core (coulomb_ref.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__ and bench.py's
CPU-baseline leg, never by the product package.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coulomb_ref.c")
_LIB = os.path.join(_HERE, "_coulomb_ref.so")
_lib = None


def build(force=False):
    """Compile coulomb_ref.c with gcc into oracle/_coulomb_ref.so (plain C,
    no target-specific flags, so x86_64 and aarch64 builds agree)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.ref_coulomb_open_batch.argtypes = [ctypes.c_int, ip, dp, dp, dp, ip]
        L.ref_whittaker_logderiv_batch.argtypes = [ctypes.c_int, ip, dp, dp, dp, ip]
        L.ref_regular_analytic_batch.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp, ip]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def coulomb_open(l, eta, rho):
    """Coulomb F, F', G, G' (rho-derivatives) for arrays l, eta, rho.
    Returns (out[n,4], status[n]); status != 0 marks a continued fraction that
    did not settle."""
    l, eta, rho = np.broadcast_arrays(_i(l), _d(eta), _d(rho))
    l, eta, rho = _i(l.ravel()), _d(eta.ravel()), _d(rho.ravel())
    n = l.size
    out = np.zeros((n, 4))
    st = np.zeros(n, dtype=np.int32)
    lib().ref_coulomb_open_batch(n, _p(l, ctypes.c_int), _p(eta, ctypes.c_double),
                                 _p(rho, ctypes.c_double), _p(out, ctypes.c_double),
                                 _p(st, ctypes.c_int))
    return out, st


def whittaker_logderiv(l, nu, x):
    """d ln W_{nu,l+1/2}(x) / dx for arrays. Returns (out[n], status[n])."""
    l, nu, x = np.broadcast_arrays(_i(l), _d(nu), _d(x))
    l, nu, x = _i(l.ravel()), _d(nu.ravel()), _d(x.ravel())
    n = l.size
    out = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    lib().ref_whittaker_logderiv_batch(n, _p(l, ctypes.c_int), _p(nu, ctypes.c_double),
                                       _p(x, ctypes.c_double), _p(out, ctypes.c_double),
                                       _p(st, ctypes.c_int))
    return out, st


def regular_analytic(l, z, eps, r):
    """Energy-analytic regular solution f and df/dr at r. Returns (out[n,2], status[n])."""
    l, z, eps, r = np.broadcast_arrays(_i(l), _d(z), _d(eps), _d(r))
    l, z, eps, r = _i(l.ravel()), _d(z.ravel()), _d(eps.ravel()), _d(r.ravel())
    n = l.size
    out = np.zeros((n, 2))
    st = np.zeros(n, dtype=np.int32)
    lib().ref_regular_analytic_batch(n, _p(l, ctypes.c_int), _p(z, ctypes.c_double),
                                     _p(eps, ctypes.c_double), _p(r, ctypes.c_double),
                                     _p(out, ctypes.c_double), _p(st, ctypes.c_int))
    return out, st
