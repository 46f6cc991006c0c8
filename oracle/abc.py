"""ctypes wrapper of the brute-force FP64 ABC-model oracle (abc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product package.

A(p) + B(k_0) -> A(p') + B(k_1) ... B(k_k); momenta [N][k+3][4] with slot
0 = A in, 1 = B in, 2 = A out, 3.. = B out.  |M|^2 is the square of the real
tree-level amplitude g^n sum_orders prod 1/(Q^2 - m^2) (paper App. F).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abc_oracle.c")
_LIB = os.path.join(_HERE, "libabc_oracle.so")
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libabc_oracle.so (plain gcc, OpenMP,
    no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared",
                               "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.abc_oracle_m2.argtypes = [ctypes.c_int, ctypes.c_longlong, _dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _dp, _dp, ctypes.c_int]
        L.abc_oracle_amplitude.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _dp]
        L.abc_oracle_m2.restype = ctypes.c_int
        L.abc_oracle_amplitude.restype = ctypes.c_int
        _lib = L
    return _lib


def m2(momenta, mass_a=1.0, mass_c=1.0, coupling=1.0, threads=0, kappa=False):
    """|M|^2 per point (and the cancellation measure kappa if asked)."""
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    n, slots, _ = mom.shape
    k = slots - 3
    out = np.empty(n, dtype=np.float64)
    kap = np.empty(n, dtype=np.float64)
    st = lib().abc_oracle_m2(k, n, mom.ctypes.data_as(_dp), float(mass_a), float(mass_c), float(coupling),
                             out.ctypes.data_as(_dp), kap.ctypes.data_as(_dp), int(threads))
    if st != 0:
        raise ValueError("abc_oracle_m2: invalid arguments")
    return (out, kap) if kappa else out


def amplitude(point, mass_a=1.0, mass_c=1.0, coupling=1.0):
    """The real amplitude M of one point [k+3][4]."""
    p = np.ascontiguousarray(point, dtype=np.float64)
    out = ctypes.c_double()
    st = lib().abc_oracle_amplitude(p.shape[0] - 3, p.ctypes.data_as(_dp), float(mass_a), float(mass_c),
                                    float(coupling), ctypes.byref(out))
    if st != 0:
        raise ValueError("abc_oracle_amplitude: invalid arguments")
    return out.value
