"""The library's count of the root operator in HBS form (csrc/hbs_size.cpp, reported as
gm_info.hbs_operator_bytes, the paper's M(n) of Table mem) against the arrays the oracle
actually stores for the same tree and ranks: D of every leaf, U and V of every node
below the root, and the two sibling blocks of every B."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import hbs, nd_dense
from paper_1302_5995_gb300 import inputs

from test_server_host import _cuda_include

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("no CUDA headers")
    out = str(tmp_path_factory.mktemp("hbssize") / "hbs_size.so")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", inc, "-o", out,
                           os.path.join(ROOT, "tests", "hbs_size_shim.cpp"),
                           os.path.join(ROOT, "paper_1302_5995_gb300", "csrc", "hbs_size.cpp")])
    L = ctypes.CDLL(out)
    ip = ctypes.POINTER(ctypes.c_int)
    L.hbs_size.argtypes = [ctypes.c_int, ip, ip, ip]
    L.hbs_size.restype = ctypes.c_int64
    return L


@pytest.mark.parametrize("n,m,tol", [(24, 16, 1e-9), (40, 24, 1e-7), (40, 12, 1e-11)])
def test_hbs_size_counts_the_stored_factors(lib, n, m, tol):
    b, c, d = inputs.convection_fields(n, seeds=(5, 6, 7))
    S = nd_dense.build(b, c, d, n, 8).S_root
    tree = hbs.HBSTree(S.shape[0], m)
    f = hbs.compress(S, tree, tol)
    NN = 1 << (tree.L + 1)
    lo = np.zeros(NN, np.int32)
    hi = np.zeros(NN, np.int32)
    k = np.zeros(NN, np.int32)
    for t in range(1, NN):
        lo[t], hi[t] = tree.rng[t]
        k[t] = f.rank(t) if t in f.U else 0
    stored = sum(x.size for x in f.D.values()) + sum(x.size for x in f.U.values()) \
        + sum(x.size for x in f.V.values()) \
        + sum(2 * f.rank(2 * t) * f.rank(2 * t + 1) for t in f.B)  # B: its two off-diagonal blocks
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    assert lib.hbs_size(tree.L, P(lo), P(hi), P(k)) == stored
    assert tree.L >= 2  # a tree with inner nodes below the root
