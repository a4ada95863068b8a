"""gm_solve_static: the solve without any device allocation, for callers that cannot let
a library allocate (a serving loop that must not touch the allocator once running, or a
host whose device memory belongs to another runtime's pool).  Its result must equal the
allocating gm_solve on the same operator, call after call.

Collected after the other established tests on purpose (file name; only the tests
marked late follow it): if it fails, a stop-at-first-failure run has already run them.
"""
import ctypes

import numpy as np
import pytest

from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def test_static_solve_matches_gm_solve_on_consecutive_calls(gm):
    lib = gm.load_library()
    n, leaf, B = 64, 8, 40
    op = gm.build(*inputs.convection_fields(n), n, leaf)
    for seed in (1, 2):  # two calls in a row: the shared scratch keeps the previous data
        G = np.ascontiguousarray(inputs.gaussian_vectors(n, B, seed).T)  # vector j contiguous
        ref = op.solve(G)  # gm_solve with host buffers (allocating path)
        out = np.full_like(G, np.nan)
        rc = lib.gm_solve_static(op._h, _p(G), _p(out), B, ctypes.c_void_p(0))
        assert rc == gm.GM_OK, gm.strerror(rc)
        err = (np.linalg.norm(out - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()
        assert err < TOL


def test_static_solve_device_buffers(gm):
    import torch
    lib = gm.load_library()
    n, leaf, B = 40, 10, 7
    op = gm.build(*inputs.laplace_fields(n), n, leaf)
    G = np.ascontiguousarray(inputs.gaussian_vectors(n, B, 3).T)
    ref = op.solve(G)
    Gd = torch.from_numpy(G).cuda()
    Vd = torch.empty_like(Gd)
    for _ in range(2):
        rc = lib.gm_solve_static(op._h, ctypes.c_void_p(Gd.data_ptr()), ctypes.c_void_p(Vd.data_ptr()), B,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == gm.GM_OK
        torch.cuda.synchronize()
        out = Vd.cpu().numpy()
        assert (np.linalg.norm(out - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < TOL


def test_static_solve_rejects_oversize(gm):
    lib = gm.load_library()
    n = 64
    op = gm.build(*inputs.laplace_fields(n), n, 8)
    B = (1 << 21) // (4 * n) // 2 + 1  # host input + host output exceed 2^21 doubles
    G = np.zeros((B, 4 * n))
    out = np.zeros_like(G)
    assert lib.gm_solve_static(op._h, _p(G), _p(out), B, ctypes.c_void_p(0)) == gm.GM_ESCRATCH
    assert "scratch" in gm.strerror(gm.GM_ESCRATCH)
