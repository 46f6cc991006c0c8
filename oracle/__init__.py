"""ctypes wrapper of the brute-force FP64 oracle (qed_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product package.

Spin configurations: ``sum_mask`` bit i set means slot i (0 = e- in,
1 = gamma in, 2 = e- out, 3.. = gamma out) is summed over its two states;
``hel`` gives the fixed state of every other slot (electrons +1/-1, photons
polarisation 1/2).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qed_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (plain g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_m2.argtypes = [ctypes.c_int, ctypes.c_longlong, _dp, ctypes.c_int, _ip,
                                ctypes.c_double, _dp, _dp, ctypes.c_int]
        L.oracle_ward.argtypes = [ctypes.c_int, ctypes.c_longlong, _dp, ctypes.c_int, ctypes.c_int,
                                  _ip, ctypes.c_double, _dp]
        L.oracle_amplitudes.argtypes = [ctypes.c_int, _dp, _ip, ctypes.c_double, _dp, _dp]
        L.oracle_grad.argtypes = [ctypes.c_int, ctypes.c_longlong, _dp, ctypes.c_int, _ip,
                                  ctypes.c_double, _dp, _dp]
        L.oracle_spinor.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp]
        L.oracle_polarisation.argtypes = [_dp, ctypes.c_int, _dp]
        L.oracle_gamma.argtypes = [ctypes.c_int, _dp]
        for f in (L.oracle_m2, L.oracle_ward, L.oracle_amplitudes, L.oracle_grad,
                  L.oracle_spinor, L.oracle_polarisation, L.oracle_gamma):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _hel_arr(k, hel):
    h = np.zeros(k + 3, dtype=np.int32)
    if hel is not None:
        h[:] = np.asarray(hel, dtype=np.int32)
    return h


def all_summed(k: int) -> int:
    return (1 << (k + 3)) - 1


def m2(momenta, sum_mask=None, hel=None, mass=1.0, threads=0, kappa=False):
    """|M|^2 per point; momenta[N][k+3][4] float64.  With kappa=True also
    returns the per-point cancellation measure kappa."""
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    n, slots, _ = mom.shape
    k = slots - 3
    if sum_mask is None:
        sum_mask = all_summed(k)
    out = np.empty(n)
    kap = np.empty(n)
    h = _hel_arr(k, hel)
    rc = lib().oracle_m2(k, n, _d(mom), int(sum_mask), h.ctypes.data_as(_ip), mass, _d(out),
                         _d(kap), int(threads))
    if rc != 0:
        raise ValueError("oracle_m2: invalid arguments")
    return (out, kap) if kappa else out


def ward(momenta, photon, sum_mask=None, hel=None, mass=1.0):
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    n, slots, _ = mom.shape
    k = slots - 3
    if sum_mask is None:
        sum_mask = all_summed(k)
    out = np.empty(n)
    h = _hel_arr(k, hel)
    rc = lib().oracle_ward(k, n, _d(mom), int(photon), int(sum_mask), h.ctypes.data_as(_ip),
                           mass, _d(out))
    if rc != 0:
        raise ValueError("oracle_ward: invalid arguments")
    return out


def amplitudes(momentum, hel, mass=1.0):
    """Per-diagram complex amplitudes for one point, lexicographic photon order."""
    mom = np.ascontiguousarray(momentum, dtype=np.float64)
    k = mom.shape[0] - 3
    nd = math.factorial(k + 1)
    re = np.empty(nd)
    im = np.empty(nd)
    h = _hel_arr(k, hel)
    rc = lib().oracle_amplitudes(k, _d(mom), h.ctypes.data_as(_ip), mass, _d(re), _d(im))
    if rc != 0:
        raise ValueError("oracle_amplitudes: invalid arguments")
    return re + 1j * im


def grad(momenta, sum_mask=None, hel=None, mass=1.0):
    """(|M|^2, d|M|^2 / d k_j) for the k outgoing photons' 3-momenta."""
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    n, slots, _ = mom.shape
    k = slots - 3
    if sum_mask is None:
        sum_mask = all_summed(k)
    out = np.empty(n)
    g = np.empty((n, k, 3))
    h = _hel_arr(k, hel)
    rc = lib().oracle_grad(k, n, _d(mom), int(sum_mask), h.ctypes.data_as(_ip), mass, _d(out),
                           _d(g))
    if rc != 0:
        raise ValueError("oracle_grad: invalid arguments")
    return out, g


def spinor(p, h, mass=1.0, bar=False):
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty(8)
    if lib().oracle_spinor(_d(p), int(h), mass, int(bar), _d(out)) != 0:
        raise ValueError("bad helicity")
    return out[0::2] + 1j * out[1::2]


def polarisation(k, pol):
    k = np.ascontiguousarray(k, dtype=np.float64)
    out = np.empty(4)
    if lib().oracle_polarisation(_d(k), int(pol), _d(out)) != 0:
        raise ValueError("bad polarisation")
    return out


def gamma(mu):
    out = np.empty(32)
    if lib().oracle_gamma(int(mu), _d(out)) != 0:
        raise ValueError("bad index")
    return (out[0::2] + 1j * out[1::2]).reshape(4, 4)
