"""ctypes binding of the FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py use it. The CUDA product path never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

ST_OK, ST_MAPPED, ST_MAX_STEPS, ST_H_UNDERFLOW, ST_NONFINITE = 0, 1, -1, -2, -3


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def build_variant(dest: str, flags: list[str]) -> str:
    """Compile the same oracle.cpp with extra compiler flags into dest (used by
    the test that measures how much two legal builds of the same arithmetic
    disagree, e.g. with and without FMA contraction)."""
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", *flags, SRC, "-o", dest])
    return dest


class Opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double), ("max_steps", ctypes.c_int32),
                ("isothermal", ctypes.c_int32), ("fixed_h", ctypes.c_double), ("hmin_frac", ctypes.c_double),
                ("nthreads", ctypes.c_int32), ("mapping", ctypes.c_int32), ("map_Ttol", ctypes.c_double),
                ("map_Ytol", ctypes.c_double), ("map_Tmax", ctypes.c_double)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _bind(lib):
    lib.orc_load.restype = ctypes.c_void_p
    lib.orc_load.argtypes = [ctypes.c_char_p]
    lib.orc_free.argtypes = [ctypes.c_void_p]
    lib.orc_last_error.restype = ctypes.c_char_p
    lib.orc_nspecies.argtypes = [ctypes.c_void_p]
    lib.orc_nreactions.argtypes = [ctypes.c_void_p]
    lib.orc_thermo.argtypes = [ctypes.c_void_p, ctypes.c_double] + [_dp] * 4
    lib.orc_rates.argtypes = [ctypes.c_void_p, ctypes.c_double] + [_dp] * 5
    lib.orc_rhs.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, ctypes.c_int]
    lib.orc_jacobian.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, ctypes.c_int]
    lib.orc_lu_solve.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    lib.orc_ros4_coeffs.argtypes = [_dp]
    lib.orc_map_classify.restype = ctypes.c_int64
    lib.orc_map_classify.argtypes = [ctypes.c_void_p, ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_uint8)]
    lib.orc_map_buckets.restype = ctypes.c_int64
    lib.orc_map_buckets.argtypes = [ctypes.c_void_p, ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int64)]
    lib.orc_integrate.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, _dp, _dp, _dp, _dp, _dp,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(Opts), _dp]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def load_variant(path: str):
    """A separately built copy of the oracle (see build_variant); pass it to
    Oracle(..., lib=...)."""
    return _bind(ctypes.CDLL(os.path.abspath(path)))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def ros4_coefficients() -> dict:
    v = np.zeros(20)
    _load().orc_ros4_coeffs(_p(v))
    return dict(gamma=v[0], a21=v[1], a31=v[2], a32=v[3], c21=v[4], c31=v[5], c32=v[6], c41=v[7],
                c42=v[8], c43=v[9], m=v[10:14].copy(), e=v[14:18].copy())


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    if _load().orc_lu_solve(A.shape[0], _p(A), _p(b), _p(x)) != 0:
        raise np.linalg.LinAlgError("singular")
    return x


class Oracle:
    """One loaded mechanism; all state vectors are y = (T, Y_1..Y_nsp)."""

    def __init__(self, mech_path: str, lib=None):
        lib = lib if lib is not None else _load()
        self._lib = lib
        self._h = lib.orc_load(mech_path.encode())
        if not self._h:
            raise ValueError(lib.orc_last_error().decode())
        self.nsp = lib.orc_nspecies(self._h)
        self.nrx = lib.orc_nreactions(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and getattr(self, "_lib", None) is not None:
            self._lib.orc_free(self._h)
            self._h = None

    def thermo(self, T: float):
        cp, h, s, g = (np.zeros(self.nsp) for _ in range(4))
        self._lib.orc_thermo(self._h, T, _p(cp), _p(h), _p(s), _p(g))
        return cp, h, s, g

    def rates(self, p: float, y: np.ndarray):
        y = np.ascontiguousarray(y, dtype=np.float64)
        c = np.zeros(self.nsp)
        kf, kr, q = (np.zeros(self.nrx) for _ in range(3))
        self._lib.orc_rates(self._h, p, _p(y), _p(c), _p(kf), _p(kr), _p(q))
        return c, kf, kr, q

    def rhs(self, p: float, y: np.ndarray, isothermal: bool = False) -> np.ndarray:
        y = np.ascontiguousarray(y, dtype=np.float64)
        f = np.zeros(self.nsp + 1)
        self._lib.orc_rhs(self._h, p, _p(y), _p(f), int(isothermal))
        return f

    def jacobian(self, p: float, y: np.ndarray, isothermal: bool = False) -> np.ndarray:
        y = np.ascontiguousarray(y, dtype=np.float64)
        J = np.zeros((self.nsp + 1, self.nsp + 1))
        self._lib.orc_jacobian(self._h, p, _p(y), _p(J), int(isothermal))
        return J

    def map_classify(self, T, Y, Yref, Ttol, Ytol, Tmax=0.0):
        T = np.ascontiguousarray(T, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        Yref = np.ascontiguousarray(Yref, dtype=np.float64)
        flag = np.zeros(T.size, dtype=np.uint8)
        ref = self._lib.orc_map_classify(self._h, T.size, _p(T), _p(Y), _p(Yref), Ttol, Ytol, Tmax,
                                       flag.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return int(ref), flag

    def map_buckets(self, T, Y, Ttol, Ytol, Tmax=0.0):
        """One reference per state bucket: (ref[n] int64, -1 for unmapped
        cells; flag[n] uint8, 1 for mapped cells)."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        flag = np.zeros(T.size, dtype=np.uint8)
        ref = np.zeros(T.size, dtype=np.int64)
        self._lib.orc_map_buckets(self._h, T.size, _p(T), _p(Y), Ttol, Ytol, Tmax,
                                  flag.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                  ref.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return ref, flag

    def integrate(self, T, p, Y, dt, rtol=1e-6, atol=1e-10, max_steps=100000, isothermal=False,
                  fixed_h=0.0, hmin_frac=1e-20, nthreads=None, mapping=False, map_Ttol=1e-4,
                  map_Ytol=1e-4, map_Tmax=0.0, Yref=None):
        """Integrate cells over dt. T[n], p[n], Y[nsp, n] -> (T', Y', steps, status).
        mapping: 0/False none, 1/True one reference cell, 2 one reference per state bucket."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        p = np.ascontiguousarray(np.broadcast_to(p, T.shape), dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        n = T.size
        assert Y.shape == (self.nsp, n)
        Tout = np.zeros(n)
        Yout = np.zeros_like(Y)
        steps = np.zeros(n, dtype=np.int32)
        status = np.zeros(n, dtype=np.int32)
        o = Opts(rtol, atol, max_steps, int(isothermal), fixed_h, hmin_frac,
                 nthreads if nthreads else (os.cpu_count() or 1), int(mapping), map_Ttol, map_Ytol, map_Tmax)
        yr = None if Yref is None else _p(np.ascontiguousarray(Yref, dtype=np.float64))
        self._lib.orc_integrate(self._h, n, dt, _p(T), _p(p), _p(Y), _p(Tout), _p(Yout),
                              steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              status.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(o), yr)
        return Tout, Yout, steps, status
