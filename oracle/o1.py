"""Python access to the plain-C oracle O1 (o1_full.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "o1_full.c")
_LIB = os.path.join(_HERE, "_o1.so")
_lib = None


def build(force=False):
    """Compile o1_full.c with gcc into oracle/_o1.so (portable C, no target flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.o1_dtn_apply.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, dp]
        _lib.o1_dtn_apply.restype = ctypes.c_int
        _lib.o1_assemble_dense.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        _lib.o1_assemble_dense.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dtn_apply(b, c, d, n, G):
    """Neumann data for the Dirichlet vectors G (4n x B) by a full banded solve."""
    lib = _load()
    b, c, d = (np.ascontiguousarray(x, dtype=np.float64) for x in (b, c, d))
    G = np.asfortranarray(np.asarray(G, dtype=np.float64).reshape(4 * n, -1))
    V = np.zeros_like(G, order="F")
    rc = lib.o1_dtn_apply(n, _p(b), _p(c), _p(d), G.shape[1], _p(G), _p(V))
    if rc:
        raise RuntimeError(f"o1_dtn_apply failed: {rc}")
    return np.ascontiguousarray(V)


def dtn_matrix(b, c, d, n):
    """The full 4n x 4n DtN matrix (columns = images of the unit vectors)."""
    return dtn_apply(b, c, d, n, np.eye(4 * n))


def assemble_dense(b, c, d, n):
    lib = _load()
    b, c, d = (np.ascontiguousarray(x, dtype=np.float64) for x in (b, c, d))
    A = np.zeros((n * n, n * n))
    lib.o1_assemble_dense(n, _p(b), _p(c), _p(d), _p(A))
    return A
