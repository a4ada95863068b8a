"""gm_solve_static: the solve without any device allocation, for callers that cannot let
a library allocate (a serving loop that must not touch the allocator once running, or a
host whose device memory belongs to another runtime's pool).  Its result must equal the
allocating gm_solve on the same operator, call after call, whichever of g and dudn live
on the host and whichever precision the operator was built in.

Collected after every other test on purpose (its file name sorts last): if it fails, a
stop-at-first-failure run has already run all the others.
"""
import ctypes

import numpy as np
import pytest

from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10
LIMIT = 1 << 21  # doubles in the library's static array


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


def _p(a):
    return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)


def _rel(out, ref):
    return (np.linalg.norm(out - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()


@pytest.mark.parametrize("g_on,v_on", [("host", "host"), ("host", "device"), ("device", "host"),
                                       ("device", "device")])
def test_static_solve_matches_gm_solve_on_consecutive_calls(gm, g_on, v_on):
    import torch
    lib = gm.load_library()
    n, leaf, B = 64, 8, 40
    op = gm.build(*inputs.convection_fields(n), n, leaf)
    stream = torch.cuda.current_stream()
    for seed in (1, 2):  # two calls in a row: the shared array keeps the previous call's data
        G = np.ascontiguousarray(inputs.gaussian_vectors(n, B, seed).T)  # vector j contiguous
        ref = op.solve(G)  # gm_solve with host buffers (the allocating path)
        g = torch.from_numpy(G).cuda() if g_on == "device" else G
        out = torch.full(G.shape, float("nan"), dtype=torch.float64, device="cuda") if v_on == "device" \
            else np.full_like(G, np.nan)
        torch.cuda.synchronize()
        rc = lib.gm_solve_static(op._h, _p(g), _p(out), B, ctypes.c_void_p(stream.cuda_stream))
        assert rc == gm.GM_OK, gm.strerror(rc)
        torch.cuda.synchronize()
        res = out.cpu().numpy() if v_on == "device" else out
        assert _rel(res, ref) < TOL


def test_static_solve_mixed_precision_handle(gm):
    """A mixed-precision operator gets gm_solve's split-product apply: the same result."""
    lib = gm.load_library()
    n, leaf, B = 128, 16, 24
    op = gm.build(*inputs.convection_fields(n, seeds=(7, 8, 9)), n, leaf, precision=gm.PREC_MIXED)
    for seed in (4, 5):
        G = np.ascontiguousarray(inputs.gaussian_vectors(n, B, seed).T)
        ref = op.solve(G)
        out = np.full_like(G, np.nan)
        assert lib.gm_solve_static(op._h, _p(G), _p(out), B, ctypes.c_void_p(0)) == gm.GM_OK
        assert _rel(out, ref) < TOL


def test_static_solve_size_limit_is_exact(gm):
    """Host g and host dudn of 4n x B doubles each: B = 4096 at n = 64 fills the array
    exactly and runs; one more vector is refused."""
    lib = gm.load_library()
    n = 64
    op = gm.build(*inputs.laplace_fields(n), n, 8)
    B = LIMIT // (2 * 4 * n)
    G = np.ascontiguousarray(inputs.gaussian_vectors(n, B, 6).T)
    out = np.zeros_like(G)
    assert lib.gm_solve_static(op._h, _p(G), _p(out), B, ctypes.c_void_p(0)) == gm.GM_OK
    ref = op.solve(G[:16])
    assert _rel(out[:16], ref) < TOL
    G1 = np.zeros((B + 1, 4 * n))
    out1 = np.zeros_like(G1)
    assert lib.gm_solve_static(op._h, _p(G1), _p(out1), B + 1, ctypes.c_void_p(0)) == gm.GM_ESCRATCH
    assert "scratch" in gm.strerror(gm.GM_ESCRATCH)


def test_static_solve_refuses_overlapping_device_buffers(gm):
    import torch
    lib = gm.load_library()
    n, B = 40, 4
    op = gm.build(*inputs.laplace_fields(n), n, 10)
    buf = torch.zeros(2 * B * 4 * n, dtype=torch.float64, device="cuda")
    g = ctypes.c_void_p(buf.data_ptr())
    v = ctypes.c_void_p(buf.data_ptr() + 8 * 4 * n)  # one vector further: overlaps
    assert lib.gm_solve_static(op._h, g, v, B, None) == gm.GM_EINVAL
    assert lib.gm_solve(op._h, g, v, B, None) == gm.GM_EINVAL
