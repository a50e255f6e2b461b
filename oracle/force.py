"""Double-precision oracle of the short-range PP acceleration.

Test infrastructure only (see the package docstring).  The heavy loop lives in
``pp_oracle.c``; this module loads it with ctypes and adds a numpy copy of the
split factor of Eq. (split) (Sec. 3.1).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
from scipy.special import erfc

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.phor_accel.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int64, i64p, dp, dp, i64p, dp, ctypes.c_double]
        lib.phor_accel.restype = None
        lib.phor_split_factor.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.phor_split_factor.restype = ctypes.c_double
        lib.phor_split_factor_v.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp]
        lib.phor_split_factor_v.restype = None
        lib.phor_mlp_factor.argtypes = [dp, ctypes.c_double, ctypes.c_double]
        lib.phor_mlp_factor.restype = ctypes.c_double
        lib.phor_accel_mlp.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, dp, ctypes.c_int64, i64p, dp]
        lib.phor_accel_mlp.restype = None
        lib.phor_num_threads.argtypes = []
        lib.phor_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def split_factor_np(s, rs):
    """Eq. (split) in numpy float64: erfc(s/2rs) + s/(rs sqrt(pi)) exp(-s^2/4rs^2)."""
    s = np.asarray(s, np.float64)
    return erfc(s / (2.0 * rs)) + s / (rs * np.sqrt(np.pi)) * np.exp(-(s * s) / (4.0 * rs * rs))


def split_factor(s, rs):
    """Eq. (split) evaluated by the C oracle (libm erfc/exp in double)."""
    lib = _load()
    s = np.ascontiguousarray(np.atleast_1d(np.asarray(s, np.float64)))
    out = np.empty_like(s)
    lib.phor_split_factor_v(s.size, _dp(s), float(rs), _dp(out))
    return out


def num_threads() -> int:
    return int(_load().phor_num_threads())


class AccelResult:
    def __init__(self, acc, abs_sum, n_within, near_abs):
        self.acc = acc
        self.abs_sum = abs_sum
        self.n_within = n_within
        self.near_abs = near_abs


def accel(pos, mass, L, G, eps, rs, rcut, targets=None, near_tol=1e-5) -> AccelResult:
    """Acceleration of each target from all sources (min image, r < rcut).

    ``pos`` [N,3] and ``mass`` [N] are converted to float64 exactly.  With
    ``targets`` (int64 indices) only those rows are returned, in that order.
    """
    lib = _load()
    pos = np.ascontiguousarray(np.asarray(pos, np.float64))
    mass = np.ascontiguousarray(np.asarray(mass, np.float64))
    n = pos.shape[0]
    if targets is None:
        nt = n
        tp = None
    else:
        targets = np.ascontiguousarray(np.asarray(targets, np.int64))
        nt = targets.size
        tp = _ip(targets)
    acc = np.zeros((nt, 3), np.float64)
    abs_sum = np.zeros(nt, np.float64)
    n_within = np.zeros(nt, np.int64)
    near_abs = np.zeros(nt, np.float64)
    if n > 0 and nt > 0:
        lib.phor_accel(n, _dp(pos), _dp(mass), float(L), float(G), float(eps), float(rs),
                       float(rcut), nt, tp, _dp(acc), _dp(abs_sum), _ip(n_within),
                       _dp(near_abs), float(near_tol))
    return AccelResult(acc, abs_sum, n_within, near_abs)


def mlp_factor(weights, r, rcut):
    """The network's factor at separations r (C oracle, double)."""
    lib = _load()
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    return np.array([lib.phor_mlp_factor(_dp(w), float(x), float(rcut)) for x in np.atleast_1d(r)])


def accel_mlp(pos, mass, L, G, eps, rcut, weights, targets=None):
    """Accelerations with the network in place of Eq. (split)."""
    lib = _load()
    pos = np.ascontiguousarray(np.asarray(pos, np.float64))
    mass = np.ascontiguousarray(np.asarray(mass, np.float64))
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    n = pos.shape[0]
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(np.asarray(targets, np.int64))
        nt, tp = targets.size, _ip(targets)
    acc = np.zeros((nt, 3))
    if n and nt:
        lib.phor_accel_mlp(n, _dp(pos), _dp(mass), float(L), float(G), float(eps), float(rcut), _dp(w), nt, tp,
                           _dp(acc))
    return acc
