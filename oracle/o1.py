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
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.o1_apply_loads.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp]
        _lib.o1_apply_loads.restype = ctypes.c_int
        _lib.o1_net_apply.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp]
        _lib.o1_net_apply.restype = ctypes.c_int
        _lib.o1_net_assemble_dense.argtypes = [ctypes.c_int, dp, dp, dp]
        _lib.o1_net_assemble_dense.restype = ctypes.c_int
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


def _loads(n, G, idx, Fl):
    """Marshal (G, body-node indices, loads) for the two load-carrying entry points."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(-1))
    m = idx.size
    if G is None:
        nvec = 1 if Fl is None else np.asarray(Fl).reshape(m, -1).shape[1]
        G = np.zeros((4 * n, nvec))
    G = np.asfortranarray(np.asarray(G, dtype=np.float64).reshape(4 * n, -1))
    if Fl is None:
        Fl = np.zeros((m, G.shape[1]))
    Fl = np.asfortranarray(np.asarray(Fl, dtype=np.float64).reshape(m, G.shape[1]))
    return G, idx, Fl


def apply_loads(b, c, d, n, G, idx, Fl):
    """Section 6.3: v = G g + F f_hat by one full solve per vector (G: 4n x B Dirichlet
    data or None for zero; idx: body nodes, flat i + n j; Fl: len(idx) x B loads)."""
    lib = _load()
    b, c, d = (np.ascontiguousarray(x, dtype=np.float64) for x in (b, c, d))
    G, idx, Fl = _loads(n, G, idx, Fl)
    V = np.zeros_like(G, order="F")
    rc = lib.o1_apply_loads(n, _p(b), _p(c), _p(d), G.shape[1], _p(G), idx.size,
                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(Fl), _p(V))
    if rc:
        raise RuntimeError(f"o1_apply_loads failed: {rc}")
    return np.ascontiguousarray(V)


def load_matrix(b, c, d, n, idx):
    """The 4n x len(idx) body-load operator F (columns = images of unit loads)."""
    idx = np.asarray(idx).reshape(-1)
    return apply_loads(b, c, d, n, None, idx, np.eye(idx.size))


def net_apply(sx, sy, n, G, idx=(), Fl=None):
    """The conductance network's datum (ghost currents / h) for Dirichlet data G and
    optional body loads; sx, sy as in inputs.network_conductivities."""
    lib = _load()
    sx, sy = (np.ascontiguousarray(x, dtype=np.float64) for x in (sx, sy))
    if sx.size != n * (n + 1) or sy.size != n * (n + 1):
        raise ValueError("conductivity arrays must hold n (n + 1) links each")
    G, idx, Fl = _loads(n, G, idx, Fl)
    V = np.zeros_like(G, order="F")
    rc = lib.o1_net_apply(n, _p(sx), _p(sy), G.shape[1], _p(G), idx.size,
                          idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(Fl), _p(V))
    if rc:
        raise RuntimeError(f"o1_net_apply failed: {rc}")
    return np.ascontiguousarray(V)


def net_dtn_matrix(sx, sy, n):
    return net_apply(sx, sy, n, np.eye(4 * n))


def net_load_matrix(sx, sy, n, idx):
    idx = np.asarray(idx).reshape(-1)
    return net_apply(sx, sy, n, None, idx, np.eye(idx.size))


def net_assemble_dense(sx, sy, n):
    lib = _load()
    sx, sy = (np.ascontiguousarray(x, dtype=np.float64) for x in (sx, sy))
    A = np.zeros((n * n, n * n))
    lib.o1_net_assemble_dense(n, _p(sx), _p(sy), _p(A))
    return A
