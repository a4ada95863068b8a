"""The C ABI's host-side contract, through the real libgm.so and without a GPU: every
entry point rejects bad arguments and options with GM_EINVAL (or GM_EUNSUPPORTED) before
it touches the device, NULL handles are refused, and on a machine without a GPU a valid
build fails loudly with GM_ECUDA rather than pretending to run or reporting a memory
shortage."""
import ctypes
import math

import numpy as np
import pytest

import paper_1302_5995_gb300 as gm


@pytest.fixture(scope="module")
def lib():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    return gm.load_library()


def _fields(n):
    z = np.zeros(n * n)
    return z, z.copy(), z.copy()


def _build_ex(lib, opts, b, c, d, n, leaf, tol):
    h = ctypes.c_void_p()
    rc = lib.gm_build_ex(ctypes.byref(opts) if opts is not None else None,
                         *(x.ctypes.data if x is not None else None for x in (b, c, d)), n, leaf, tol,
                         ctypes.byref(h))
    assert h.value is None  # nothing is handed out on failure
    return rc


@pytest.mark.parametrize("case", ["null_b", "n1", "leaf2", "tol_neg", "tol_nan"])
def test_build_rejects_bad_arguments(lib, case):
    n, leaf, tol = 8, 4, 0.0
    b, c, d = _fields(n)
    if case == "null_b":
        b = None
    elif case == "n1":
        n = 1
    elif case == "leaf2":
        leaf = 2
    elif case == "tol_neg":
        tol = -1e-9
    else:
        tol = math.nan
    assert _build_ex(lib, None, b, c, d, n, leaf, tol) == gm.GM_EINVAL
    assert lib.gm_build_ex(None, b.ctypes.data if b is not None else None, c.ctypes.data, d.ctypes.data, n, leaf,
                           tol, None) == gm.GM_EINVAL  # no output slot


@pytest.mark.parametrize("field,value", [("precision", 2), ("precision", -1), ("pivoting", 3), ("pivoting", -1),
                                         ("hbs_leaf", 1), ("hbs_leaf", 193), ("hbs_min_edge", 3)])
def test_build_rejects_bad_options(lib, field, value):
    o = gm.Opts()
    lib.gm_opts_default(ctypes.byref(o))
    assert o.precision == gm.PREC_FP64
    setattr(o, field, value)
    assert _build_ex(lib, o, *_fields(8), 8, 4, 0.0) == gm.GM_EINVAL


def test_batch_rejects_bad_arguments(lib):
    keep = [_fields(8), _fields(12)]
    probs = (gm.Problem * 2)(*[gm.Problem(f[0].ctypes.data, f[1].ctypes.data, f[2].ctypes.data, n, 4)
                               for f, n in zip(keep, (8, 12))])
    outs = (ctypes.c_void_p * 2)()
    assert lib.gm_build_batch(0, probs, None, 0.0, outs) == gm.GM_EINVAL
    assert lib.gm_build_batch(2, None, None, 0.0, outs) == gm.GM_EINVAL
    assert lib.gm_build_batch(2, probs, None, -1.0, outs) == gm.GM_EINVAL
    probs[1].leaf = 2
    assert lib.gm_build_batch(2, probs, None, 0.0, outs) == gm.GM_EINVAL
    probs[1].leaf = 4
    o = gm.Opts()
    lib.gm_opts_default(ctypes.byref(o))
    o.keep_levels = 1
    assert lib.gm_build_batch(2, probs, ctypes.byref(o), 0.0, outs) == gm.GM_EUNSUPPORTED
    assert list(outs) == [None, None]


def test_null_handles_are_refused(lib):
    x = np.zeros(16)
    info = gm.Info()
    assert lib.gm_solve(None, x.ctypes.data, x.ctypes.data, 1, None) == gm.GM_EINVAL
    assert lib.gm_solve_static(None, x.ctypes.data, x.ctypes.data, 1, None) == gm.GM_EINVAL
    assert lib.gm_get_dtn(None, x.ctypes.data) == gm.GM_EINVAL
    assert lib.gm_get_schur(None, 0, 0, 4, 4, x.ctypes.data) == gm.GM_EINVAL
    assert lib.gm_info(None, ctypes.byref(info)) == gm.GM_EINVAL
    h = ctypes.c_void_p()
    assert lib.gm_server_create(0, 1, ctypes.byref(h)) == gm.GM_EINVAL
    assert lib.gm_server_sync(None) == gm.GM_EINVAL
    lib.gm_server_destroy(None)
    lib.gm_free(None)
    lib.gm_opts_default(None)


def test_every_code_has_a_message(lib):
    codes = [gm.GM_OK, gm.GM_EINVAL, gm.GM_ENOMEM, gm.GM_ESINGULAR, gm.GM_ETIMEOUT, gm.GM_ECUDA,
             gm.GM_EUNSUPPORTED, gm.GM_ESCRATCH]
    msgs = [gm.strerror(c) for c in codes]
    assert len(set(msgs)) == len(codes) and "unknown" not in " ".join(msgs)
    assert gm.strerror(-99) == "unknown error"


def test_valid_build_without_a_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _build_ex(lib, None, *_fields(8), 8, 4, 0.0) == gm.GM_ECUDA
    with pytest.raises(gm.GmError):
        gm.build(*_fields(8), 8, 4)


def test_load_build_rejects_bad_arguments(lib):
    n = 8
    b, c, d = _fields(n)
    body = np.array([3, 10, 20], dtype=np.int32)
    h = ctypes.c_void_p()

    def call(opts=None, nodes=body, count=None, nn=n, leaf=4):
        return lib.gm_build_loads(ctypes.byref(opts) if opts is not None else None, b.ctypes.data, c.ctypes.data,
                                  d.ctypes.data, nn, leaf, nodes.ctypes.data if nodes is not None else None,
                                  len(nodes) if count is None else count, ctypes.byref(h))
    assert call(nodes=None, count=3) == gm.GM_EINVAL
    assert call(count=0) == gm.GM_EINVAL
    assert call(nodes=np.array([3, 64], dtype=np.int32)) == gm.GM_EINVAL  # outside the 8 x 8 grid
    assert call(nodes=np.array([-1], dtype=np.int32)) == gm.GM_EINVAL
    assert call(nodes=np.array([5, 9, 5], dtype=np.int32)) == gm.GM_EINVAL  # repeated
    assert call(leaf=2) == gm.GM_EINVAL
    o = gm.Opts()
    lib.gm_opts_default(ctypes.byref(o))
    o.precision = gm.PREC_MIXED
    assert call(opts=o) == gm.GM_EUNSUPPORTED  # FP64 only
    lib.gm_opts_default(ctypes.byref(o))
    o.keep_levels = 1
    assert call(opts=o) == gm.GM_EUNSUPPORTED
    assert h.value is None
    x = np.zeros(64)
    assert lib.gm_solve_loads(None, x.ctypes.data, x.ctypes.data, x.ctypes.data, 1, None) == gm.GM_EINVAL
    assert lib.gm_get_load_operator(None, x.ctypes.data) == gm.GM_EINVAL


def test_network_build_rejects_bad_arguments(lib):
    n = 8
    sx = np.ones(n * (n + 1))
    sy = np.ones(n * (n + 1))
    h = ctypes.c_void_p()

    def call(opts=None, a=sx, b=sy, nodes=None, count=0, nn=n, leaf=4, tol=0.0):
        return lib.gm_build_net(ctypes.byref(opts) if opts is not None else None,
                                a.ctypes.data if a is not None else None, b.ctypes.data if b is not None else None,
                                nn, leaf, tol, nodes.ctypes.data if nodes is not None else None, count,
                                ctypes.byref(h))
    assert call(a=None) == gm.GM_EINVAL
    assert call(leaf=2) == gm.GM_EINVAL
    assert call(count=-1) == gm.GM_EINVAL
    assert call(count=2) == gm.GM_EINVAL  # loads without a list
    assert call(nodes=np.array([1, 1], dtype=np.int32), count=2) == gm.GM_EINVAL
    assert call(nodes=np.array([64], dtype=np.int32), count=1) == gm.GM_EINVAL
    assert call(tol=-1.0) == gm.GM_EINVAL
    assert call(tol=1e-9, nodes=np.array([3], dtype=np.int32), count=1) == gm.GM_EUNSUPPORTED  # HBS + loads
    o = gm.Opts()
    lib.gm_opts_default(ctypes.byref(o))
    o.precision = gm.PREC_MIXED
    assert call(opts=o) == gm.GM_EUNSUPPORTED
    lib.gm_opts_default(ctypes.byref(o))
    o.keep_levels = 1
    assert call(opts=o, nodes=np.array([3], dtype=np.int32), count=1) == gm.GM_EUNSUPPORTED  # kept levels + loads
    assert h.value is None


def test_binding_checks_solve_buffers_before_the_library():
    """A wrong-sized g, f or out is refused in Python: the library would read or write
    4n * batch values through the pointers it is given."""
    op = gm.DtN(ctypes.c_void_p(1), 8, 4)  # never reaches the library
    op.nbody = 3
    N = 32
    with pytest.raises(ValueError):
        op.solve(np.zeros(N + 1))
    with pytest.raises(ValueError):
        op.solve(np.zeros(2 * N), out=np.zeros(N))
    with pytest.raises(ValueError):
        op.solve(np.zeros(2 * N), out=np.zeros(2 * N, dtype=np.float32))
    with pytest.raises(ValueError):
        op.solve(np.zeros(2 * N), out=np.zeros((2 * N, 2))[:, 0])  # not contiguous
    with pytest.raises(ValueError):
        op.solve_loads(np.zeros(2 * N), np.zeros(5))  # 2 vectors need 2 x 3 loads
    op._h = None  # nothing to free


def test_binding_checks_dtn_and_server_buffers():
    op = gm.DtN(ctypes.c_void_p(1), 8, 4)  # never reaches the library
    with pytest.raises(ValueError):
        op.dtn(out=np.zeros(32 * 32 - 1))
    op._h = None
    srv = object.__new__(gm.Server)  # the request checks run before any library call
    srv._s, srv._keep, srv._n = None, {}, {7: 8}
    with pytest.raises(ValueError):
        srv.submit(7, np.zeros((2, 32)), np.zeros((1, 32)), 2)  # out holds one vector of two
    with pytest.raises(ValueError):
        srv.submit(7, np.zeros((1, 31)), np.zeros((1, 32)), 1)
