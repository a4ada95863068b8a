"""Batched build (several independent problems, uneven n, one launch per stage across
all of them) against single builds and the FP64 oracle, in both precisions."""
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


def rel_mat(A, B):
    return np.abs(A - B).max() / np.abs(B).max()


def same_as_single(op, single):
    """Each problem of a batch takes the same path (and the same automatic fallback) as
    its single build, so the results agree to the last bits."""
    assert op.info()["pivot_fallback"] == single.info()["pivot_fallback"]
    return rel_mat(op.dtn(), single.dtn()) < 1e-13


def small_mix():
    """Five problems of uneven size, depth and leaf: one and two tree levels apart,
    ragged leaves, Laplace / convection / Helmholtz fields."""
    probs = []
    b, c, d = inputs.convection_fields(64, seeds=(7, 8, 9))
    probs.append((b, c, d, 64, 16))
    b, c, d = inputs.convection_fields(96, seeds=(10, 11, 12))
    probs.append((b, c, d, 96, 16))
    k = inputs.nudged_wavenumber(61, 8)
    b, c, d = inputs.helmholtz_fields(61, k)
    probs.append((b, c, d, 61, 8))
    b, c, d = inputs.laplace_fields(40)
    probs.append((b, c, d, 40, 8))
    b, c, d = inputs.convection_fields(128, seeds=(13, 14, 15))
    probs.append((b, c, d, 128, 16))
    return probs


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_batch_matches_oracle_and_single_builds(gm, prec, tol):
    precision = gm.PREC_FP64 if prec == "fp64" else gm.PREC_MIXED
    probs = small_mix()
    ops = gm.build_batch(probs, precision=precision)
    assert len(ops) == len(probs)
    for op, (b, c, d, n, leaf) in zip(ops, probs):
        T = op.dtn()
        assert T.shape == (4 * n, 4 * n)
        To = nd_dense.build(b, c, d, n, leaf).T
        assert rel_mat(T, To) < tol, (n, leaf)
        single = gm.build(b, c, d, n, leaf, precision=precision)
        assert same_as_single(op, single), (n, leaf)
        info = op.info()
        assert info["n"] == n and info["leaf"] == leaf


def test_batch_solve_per_problem(gm):
    probs = small_mix()
    ops = gm.build_batch(probs, precision=gm.PREC_MIXED)
    for i, (op, (b, c, d, n, leaf)) in enumerate(zip(ops, probs)):
        G = inputs.gaussian_vectors(n, 8, 50 + i)
        V = op.solve(np.ascontiguousarray(G.T)).reshape(8, 4 * n).T
        Vo = nd_dense.build(b, c, d, n, leaf).T @ G
        err = (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()
        assert err < 1e-8, (n, err)


def test_batch_of_one_equals_single(gm):
    b, c, d = inputs.convection_fields(80, seeds=(21, 22, 23))
    (op,) = gm.build_batch([(b, c, d, 80, 16)])
    single = gm.build(b, c, d, 80, 16)
    assert rel_mat(op.dtn(), single.dtn()) < 1e-14


def test_batch_device_coefficients(gm):
    import torch
    probs = small_mix()[:3]
    dev = [tuple(torch.from_numpy(x).cuda() for x in p[:3]) + p[3:] for p in probs]
    ops_d = gm.build_batch(dev, precision=gm.PREC_MIXED)
    ops_h = gm.build_batch(probs, precision=gm.PREC_MIXED)
    for a, b in zip(ops_d, ops_h):
        assert rel_mat(a.dtn(), b.dtn()) < 1e-14


def test_batch_rejects_bad_arguments(gm):
    b, c, d = inputs.laplace_fields(32)
    with pytest.raises(gm.GmError):
        gm.build_batch([])
    with pytest.raises(gm.GmError):
        gm.build_batch([(b, c, d, 32, 2)])  # leaf below 4
    lib = gm.load_library()
    o = gm.Opts()
    lib.gm_opts_default(o)
    o.keep_levels = 1
    arr = (gm.Problem * 1)(gm.Problem(b.ctypes.data, c.ctypes.data, d.ctypes.data, 32, 8))
    import ctypes
    outs = (ctypes.c_void_p * 1)()
    assert lib.gm_build_batch(1, arr, o, 0.0, outs) == -6  # GM_EUNSUPPORTED
    assert outs[0] is None


def test_config4_subset(gm):
    """Eight problems of the 64-problem batch recipe (every size, both field kinds) in
    mixed precision: each equals its single build and matches O2's dense nested
    dissection of the same problem (up to n = 512)."""
    cfg = inputs.config4()
    chosen, seen = [], set()
    for p in cfg:
        key = (p["n"], p["kind"])
        if key not in seen:
            seen.add(key)
            chosen.append(p)
    chosen = chosen[:8]
    probs = [(p["b"], p["c"], p["d"], p["n"], p["leaf"]) for p in chosen]
    ops = gm.build_batch(probs, precision=gm.PREC_MIXED, split_digits=6)
    for op, p in zip(ops, probs):
        single = gm.build(*p, precision=gm.PREC_MIXED, split_digits=6)
        assert same_as_single(op, single), p[3]
    for op, p in zip(ops, probs):
        To = nd_dense.build(*p).T
        assert rel_mat(op.dtn(), To) < 1e-8, p[3]


def test_batch_fallback_is_per_problem(gm):
    """Convection problems stay mixed precision, Helmholtz problems of the same batch are
    rebuilt in FP64; both equal their single builds."""
    probs = []
    for n in (128, 192):
        probs.append(inputs.convection_fields(n, seeds=(n, n + 1, n + 2)) + (n, 16))
        probs.append(inputs.helmholtz_fields(n, inputs.nudged_wavenumber(n, 16)) + (n, 16))
    ops = gm.build_batch(probs, precision=gm.PREC_MIXED, split_digits=6)
    for i, (op, p) in enumerate(zip(ops, probs)):
        info = op.info()
        helm = i % 2 == 1
        assert info["pivot_fallback"] == (1 if helm else 0)
        assert info["precision"] == (gm.PREC_FP64 if helm else gm.PREC_MIXED)
        assert same_as_single(op, gm.build(*p, precision=gm.PREC_MIXED, split_digits=6))
        assert rel_mat(op.dtn(), nd_dense.build(*p).T) < (1e-10 if helm else 1e-8)


def test_recorded_graph_replays_the_batch(gm):
    """With graph set, the first batched build of a plan runs as usual and records its
    launches; the next builds of that plan replay the graph on new coefficients.  Every
    replayed operator equals its eager build bit for bit (same kernels, same order), for
    two different coefficient sets, and the automatic fallback still applies per problem."""
    import torch
    sizes = (128, 192, 256, 128)
    def problems(seed):
        out = []
        for i, n in enumerate(sizes):
            f = inputs.convection_fields(n, seeds=(seed + 3 * i, seed + 3 * i + 1, seed + 3 * i + 2)) if i != 1 \
                else inputs.helmholtz_fields(n, inputs.nudged_wavenumber(n, 16) * (1 + 0.01 * (seed % 7)))
            out.append(tuple(torch.from_numpy(x).cuda() for x in f) + (n, 16))
        return out
    first = gm.build_batch(problems(300), precision=gm.PREC_MIXED, graph=True)  # records
    for seed in (400, 500):
        probs = problems(seed)
        rep = gm.build_batch(probs, precision=gm.PREC_MIXED, graph=True)  # replays
        eager = gm.build_batch(probs, precision=gm.PREC_MIXED)
        for a, b in zip(rep, eager):
            assert a.info()["pivot_fallback"] == b.info()["pivot_fallback"]
            assert np.array_equal(a.dtn(), b.dtn())
    del first


def test_autotuned_build_matches_the_oracle(gm):
    """The autotuner times a few launch shapes on the first build of a plan and keeps the
    fastest; whatever it picks, the result stays within the mixed-precision bound."""
    n, leaf = 256, 16
    b, c, d = inputs.convection_fields(n, seeds=(71, 72, 73))
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, autotune=True)
    op2 = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, autotune=True, graph=True)  # tuned, recorded
    op3 = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, autotune=True, graph=True)  # tuned, replayed
    To = nd_dense.build(b, c, d, n, leaf).T
    for o in (op, op2, op3):
        assert rel_mat(o.dtn(), To) < 1e-8
    assert np.array_equal(op2.dtn(), op3.dtn())
