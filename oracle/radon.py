"""ctypes binding of the C oracle for R_h / R_h^* (``radon_ref.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Builds the C file with gcc
on first use if the shared object is missing or older than its source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "radon_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libctr_oracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ``radon_ref.c`` into ``_build/libctr_oracle.so`` (plain gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            geo = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_rh_adjoint.argtypes = geo + [dp, dp]
            lib.oracle_rh_forward.argtypes = geo + [dp, dp]
            lib.oracle_rh_forward_entries.argtypes = geo + [dp, ctypes.c_int, ip, ip, dp]
            lib.oracle_rh_adjoint_entries.argtypes = geo + [dp, ctypes.c_int, ip, ip, dp]
            for f in (lib.oracle_rh_adjoint, lib.oracle_rh_forward,
                      lib.oracle_rh_forward_entries, lib.oracle_rh_adjoint_entries):
                f.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the C oracle's OpenMP loops use (honours OMP_NUM_THREADS)."""
    return int(_load().oracle_num_threads())


@dataclass
class Geometry:
    """Parallel-beam geometry of Sec. 3.1: n x n pixels of size h, N angles
    ``theta`` (radians), M detector bins of width ds."""
    n: int
    n_angles: int
    n_bins: int
    h: float = 1.0
    ds: float = 1.0
    theta: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.theta is None:
            self.theta = np.arange(self.n_angles, dtype=np.float64) * (np.pi / max(self.n_angles, 1))
        self.theta = np.ascontiguousarray(self.theta, dtype=np.float64)
        assert self.theta.shape == (self.n_angles,)

    @property
    def image_shape(self):
        return (self.n, self.n)

    @property
    def sino_shape(self):
        return (self.n_angles, self.n_bins)

    def _args(self):
        return (self.n, self.n_angles, self.n_bins, float(self.h), float(self.ds),
                self.theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def rh_forward(u: np.ndarray, geo: Geometry) -> np.ndarray:
    """g = R_h u (Sec. 3.1, the adjoint of linear backprojection).  FP64."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape == geo.image_shape
    g = np.empty(geo.sino_shape, dtype=np.float64)
    rc = _load().oracle_rh_forward(*geo._args(), _dptr(u), _dptr(g))
    if rc != 0:
        raise RuntimeError(f"oracle_rh_forward failed: {rc}")
    return g


def rh_adjoint(g: np.ndarray, geo: Geometry) -> np.ndarray:
    """u = R_h^* g (Sec. 3.1, linear backprojection).  FP64."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    assert g.shape == geo.sino_shape
    u = np.empty(geo.image_shape, dtype=np.float64)
    rc = _load().oracle_rh_adjoint(*geo._args(), _dptr(g), _dptr(u))
    if rc != 0:
        raise RuntimeError(f"oracle_rh_adjoint failed: {rc}")
    return u


def rh_forward_entries(u: np.ndarray, geo: Geometry, ls, ks) -> np.ndarray:
    """Selected entries (R_h u)_{l,k}, each by brute force with the hat weight."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    ls = np.ascontiguousarray(ls, dtype=np.int32)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    out = np.empty(ls.shape[0], dtype=np.float64)
    rc = _load().oracle_rh_forward_entries(*geo._args(), _dptr(u), int(ls.shape[0]), _iptr(ls), _iptr(ks), _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle_rh_forward_entries failed")
    return out


def rh_adjoint_entries(g: np.ndarray, geo: Geometry, is_, js) -> np.ndarray:
    """Selected entries (R_h^* g)_{i,j}, each by brute force with the hat weight."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    is_ = np.ascontiguousarray(is_, dtype=np.int32)
    js = np.ascontiguousarray(js, dtype=np.int32)
    out = np.empty(is_.shape[0], dtype=np.float64)
    rc = _load().oracle_rh_adjoint_entries(*geo._args(), _dptr(g), int(is_.shape[0]), _iptr(is_), _iptr(js), _dptr(out))
    if rc != 0:
        raise RuntimeError("oracle_rh_adjoint_entries failed")
    return out
