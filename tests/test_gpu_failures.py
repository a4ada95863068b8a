"""Failure detection without faulting the GPU.

  * A bounded device wait that runs out: with gm_opts.wait_limit < 0 every bounded wait
    of the tensor-memory kernels gives up at once (as on a flag nothing sets).  The
    kernel reports GM_ETIMEOUT through the build's status, waits (bounded) for its own
    copies and products in flight, releases its tensor memory and returns; the context
    stays usable, and the next build matches the oracle.
  * A device allocation that fails: gm_debug_fail_alloc(k) makes the k-th allocation
    fail as if the device were out of memory.  The build returns GM_ENOMEM and no handle,
    at every point tried, and the library keeps working afterwards.
"""
import numpy as np
import pytest

from oracle import nd_dense
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


def rel_vec(V, Vo):
    return (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()


def solve_cols(op, G):
    B = G.shape[1]
    return op.solve(np.ascontiguousarray(G.T)).reshape(B, G.shape[0]).T


@pytest.mark.parametrize("pivoting", ["block", "auto"])
def test_wait_that_runs_out_reports_timeout_and_the_device_stays_usable(gm, pivoting):
    n, leaf = 256, 16  # large enough for the tensor-memory update and merge kernels
    b, c, d = inputs.convection_fields(n, seeds=(41, 42, 43))
    piv = gm.PIVOT_BLOCK if pivoting == "block" else gm.PIVOT_AUTO
    with pytest.raises(gm.GmError) as e:
        gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, pivoting=piv, wait_limit=-1)
    assert e.value.code == gm.GM_ETIMEOUT
    import torch
    torch.cuda.synchronize()  # no sticky error: the context is fine
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, pivoting=piv)
    G = inputs.gaussian_vectors(n, 8, 12)
    To = nd_dense.build(b, c, d, n, leaf).T
    assert rel_vec(solve_cols(op, G), To @ G) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed", "hbs"])
def test_failed_allocation_reports_enomem_at_every_point(gm, precision):
    n, leaf = 128, 16
    b, c, d = inputs.convection_fields(n, seeds=(44, 45, 46))
    kw = {"fp64": {}, "mixed": {"precision": gm.PREC_MIXED}, "hbs": {"tol": 1e-9, "hbs_leaf": 32}}[precision]
    lib = gm.load_library()
    hit = 0
    for k in (1, 2, 3, 5, 8, 13, 21, 34, 55, 89):
        lib.gm_debug_fail_alloc(k)
        try:
            gm.build(b, c, d, n, leaf, **kw)
        except gm.GmError as e:
            assert e.code == gm.GM_ENOMEM, (k, e.code)
            hit += 1
        finally:
            lib.gm_debug_fail_alloc(0)
    assert hit >= 3  # the first allocations of every build are reached
    op = gm.build(b, c, d, n, leaf, **kw)
    G = inputs.gaussian_vectors(n, 4, 13)
    To = nd_dense.build(b, c, d, n, leaf).T
    assert rel_vec(solve_cols(op, G), To @ G) < 1e-7
