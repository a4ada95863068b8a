"""Variable-wavespeed Helmholtz at 10 points per wavelength on 1024 x 1024 unknowns,
leaf 16: the HBS build (accelerated merges for shared edges >= 128, HBS root, tol 1e-9,
FP64) and the dense FP64 build, against the oracle O2 (the paper's dense nested
dissection in FP64, itself pinned against the full banded solve O1 on smaller grids).

Bounds, on 8 of the workload's plane-wave vectors: for the dense FP64 build the larger
of 1e-10 and eps kappa_1(S_root), the agreement two backward-stable FP64 eliminations of
this indefinite problem can have; for the HBS build a bound from the truncation's
measured amplification (see the test).
"""
import functools

import numpy as np
import pytest

from oracle import nd_dense
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu

N, LEAF, M, TOL = 1024, 16, 64, 1e-9


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


@functools.lru_cache(maxsize=1)
def workload():
    """The workload, O2's Neumann data on 8 of its vectors, and the FP64 bound: two
    backward-stable FP64 eliminations of this indefinite problem agree to about
    eps kappa_1(S_root) (1.6e7 at 1024^2), above the 1e-10 of the definite problems."""
    cfg = inputs.config3(N, LEAF)
    res = nd_dense.build(cfg["b"], cfg["c"], cfg["d"], N, LEAF)
    G = cfg["G"][:, :8]
    bound = max(1e-10, np.finfo(float).eps * np.linalg.cond(res.S_root, 1))
    return cfg, G, res.T @ G, bound


def rel_vec(V, Vo):
    return (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()


def solve(gm, op, G):
    import torch
    g = torch.from_numpy(np.ascontiguousarray(G.T)).cuda()
    v = torch.empty_like(g)
    op.solve(g, out=v)
    torch.cuda.synchronize()
    return v.cpu().numpy().T


def device_fields(cfg):
    import torch
    return [torch.from_numpy(cfg[k]).cuda() for k in ("b", "c", "d")]


def test_config3_hbs_build_against_oracle(gm):
    """The indefinite operator amplifies the truncation: the oracle's own accelerated
    build (Steps 1-3 on every merge with a shared edge >= 128, HBS root; pivoted QR of the
    full blocks) is 5.5e-6 off the dense operator at tol 1e-9, above the 1e-6 first
    proposed for this workload.  The bound is revised to 1e-4 (the GPU's bases come from
    Gaussian samples), and the error must follow tol: at least 10x smaller at 1e-9 than at
    1e-7."""
    cfg, G, Vo, _ = workload()
    errs = {}
    for tol in (1e-7, TOL):
        op = gm.build(*device_fields(cfg), N, LEAF, tol=tol, hbs_leaf=M, hbs_min_edge=128)
        info = op.info()
        assert info["hbs_merges"] > 0 and info["hbs_levels"] >= 5 and info["hbs_update_rank"] > 0
        errs[tol] = rel_vec(solve(gm, op, G), Vo)
    assert info["hbs_max_rank"] > 96  # beyond the sampling of a fixed 128 columns
    assert errs[TOL] < 1e-4, errs
    assert errs[TOL] < 0.1 * errs[1e-7], errs


def test_config3_dense_fp64_against_oracle(gm):
    cfg, G, Vo, bound = workload()
    op = gm.build(*device_fields(cfg), N, LEAF)
    assert rel_vec(solve(gm, op, G), Vo) < bound


def test_config3_mixed_request_falls_back_to_fp64(gm):
    """The automatic mode routes the indefinite problem to FP64 (its reaction term is
    below -2 pi^2 everywhere) and still meets the FP64 bound."""
    cfg, G, Vo, bound = workload()
    op = gm.build(*device_fields(cfg), N, LEAF, precision=gm.PREC_MIXED)
    info = op.info()
    assert info["pivot_fallback"] == 1 and info["precision"] == gm.PREC_FP64
    assert rel_vec(solve(gm, op, G), Vo) < bound
