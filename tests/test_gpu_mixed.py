"""Mixed precision (double-float storage, FP32 pivot search, split-product tensor-core
updates) against the FP64 oracle.  Stated bound: 1e-8 relative for the 512 x 512
convection-diffusion-reaction build and its 256 solutions (per-vector 2-norms), the
same bound for every intermediate Schur complement (max-norm relative)."""
import numpy as np
import pytest

from oracle import closed_form as cf
from oracle import nd_dense
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-8


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


def rel_mat(A, B):
    return np.abs(A - B).max() / np.abs(B).max()


def rel_vec(V, Vo):
    return (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()


def solve_cols(op, G):
    B = G.shape[1]
    return op.solve(np.ascontiguousarray(G.T)).reshape(B, G.shape[0]).T


@pytest.mark.parametrize("n,leaf", [(24, 4), (37, 5), (64, 8)])
def test_mixed_every_level(gm, n, leaf):
    b, c, d = inputs.convection_fields(n, seeds=(41, 42, 43))
    op = gm.build(b, c, d, n, leaf, keep_levels=True, precision=gm.PREC_MIXED)
    ref = nd_dense.build(b, c, d, n, leaf, keep=True)
    for box, So in ref.schur.items():
        assert rel_mat(op.schur(box.x0, box.y0, box.a, box.b), So) < TOL_MIXED, box
    assert rel_mat(op.dtn(), ref.T) < TOL_MIXED


@pytest.mark.parametrize("split", [3, 4, 5, 6])
def test_mixed_digits_control_the_error(gm, split):
    n, leaf = 128, 16
    b, c, d = inputs.convection_fields(n)
    To = nd_dense.build(b, c, d, n, leaf).T
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, split_digits=split)
    err = rel_mat(op.dtn(), To)
    # each digit carries 7 bits: the error falls by about 2^7 per added digit
    bound = {3: 1e-4, 4: 1e-7, 5: 1e-9, 6: 1e-11}[split]
    assert err < bound, err


def test_mixed_config2_full_size(gm):
    import torch
    cfg = inputs.config2()
    n = cfg["n"]
    dev = [torch.from_numpy(cfg[k]).cuda() for k in "bcd"]
    op = gm.build(*dev, n, cfg["leaf"], precision=gm.PREC_MIXED)
    To = nd_dense.build(cfg["b"], cfg["c"], cfg["d"], n, cfg["leaf"]).T
    assert rel_mat(op.dtn(), To) < TOL_MIXED
    G = torch.from_numpy(np.ascontiguousarray(cfg["G"].T)).cuda()
    V = op.solve(G)
    torch.cuda.synchronize()
    V = V.cpu().numpy().reshape(256, 4 * n).T
    assert rel_vec(V, To @ cfg["G"]) < TOL_MIXED


def test_mixed_laplace_harmonic(gm):
    cfg = inputs.config1()
    n = cfg["n"]
    op = gm.build(cfg["b"], cfg["c"], cfg["d"], n, cfg["leaf"], precision=gm.PREC_MIXED)
    T = op.dtn()
    G5, V5 = cf.harmonic_pairs(n)
    assert np.abs(T @ G5 - V5).max() < TOL_MIXED * np.abs(T).max()
    V = solve_cols(op, G5)
    assert np.abs(V - V5).max() < TOL_MIXED * np.abs(T).max()


@pytest.mark.parametrize("n,leaf", [(2, 4), (5, 4), (9, 4), (61, 16)])
def test_mixed_small_and_ragged(gm, n, leaf):
    b, c, d = inputs.convection_fields(n, seeds=(3, 4, 5))
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED)
    assert rel_mat(op.dtn(), nd_dense.build(b, c, d, n, leaf).T) < TOL_MIXED


def test_mixed_singular_box_reported(gm):
    n = 6
    b, c, d = inputs.laplace_fields(n)
    d = d.copy()
    # exactly minus the centre weight 4/h^2, which the library forms as 4 (n+1)^2
    d[1 + n * 1] = -4.0 * (n + 1) ** 2
    with pytest.raises(gm.GmError) as e:
        gm.build(b, c, d, n, 4, precision=gm.PREC_MIXED)
    assert e.value.code == gm.GM_ESINGULAR


@pytest.mark.parametrize("piv", ["block", "partial"])
def test_mixed_pivoting_modes_agree_with_oracle(gm, piv):
    n, leaf = 100, 13
    b, c, d = inputs.convection_fields(n, seeds=(71, 72, 73))
    mode = gm.PIVOT_BLOCK if piv == "block" else gm.PIVOT_PARTIAL
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, pivoting=mode)
    assert op.info()["pivoting"] == mode
    assert rel_mat(op.dtn(), nd_dense.build(b, c, d, n, leaf).T) < TOL_MIXED


def test_auto_meets_bound_on_mild_helmholtz(gm):
    """Variable-wavespeed Helmholtz (indefinite) at n = 96: its block solves refine fast
    enough to stay in mixed precision, or the automatic mode rebuilds it in FP64; either
    way the result meets the bound."""
    n, leaf = 96, 12
    k = inputs.nudged_wavenumber(n, leaf)
    b, c, d = inputs.helmholtz_fields(n, k)
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED)
    info = op.info()
    assert info["precision"] == (gm.PREC_FP64 if info["pivot_fallback"] else gm.PREC_MIXED)
    To = nd_dense.build(b, c, d, n, leaf).T
    assert rel_mat(op.dtn(), To) < TOL_MIXED


def test_auto_fallback_matches_fp64_build_at_384(gm):
    """At n = 384 mixed precision with partial pivoting would miss the bound (its digit
    products lose what the indefinite problem amplifies); the fallback is the FP64 build."""
    n, leaf = 384, 16
    b, c, d = inputs.helmholtz_fields(n, inputs.nudged_wavenumber(n, leaf))
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, split_digits=6)
    info = op.info()
    assert info["pivot_fallback"] == 1 and info["refine_ratio"] == 0.0  # the FP64 rebuild's info
    assert rel_mat(op.dtn(), gm.build(b, c, d, n, leaf).dtn()) < 1e-14


def test_convection_stays_mixed_block_pivoted(gm):
    n, leaf = 256, 16
    b, c, d = inputs.convection_fields(n, seeds=(8, 9, 10))
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, split_digits=6)
    info = op.info()
    assert info["pivot_fallback"] == 0 and info["precision"] == gm.PREC_MIXED
    assert info["pivoting"] == gm.PIVOT_BLOCK
    assert rel_mat(op.dtn(), gm.build(b, c, d, n, leaf).dtn()) < TOL_MIXED


def test_mixed_long_interface_matches_oracle_at_1100(gm):
    """n = 1100: the top merge's interface gives K = 2196, so the tensor-memory merge
    update accumulates its levels in five K chunks of at most 512 (each later chunk adds
    into the parent entries the first wrote).  The whole 4400 x 4400 T against O2's dense
    nested dissection of the same problem, and against the FP64 build."""
    n, leaf = 1100, 16
    b, c, d = inputs.convection_fields(n, seeds=(21, 22, 23))
    op = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED, split_digits=6)
    assert op.info()["pivot_fallback"] == 0
    T = op.dtn()
    op.free()
    To = nd_dense.build(b, c, d, n, leaf).T
    assert rel_mat(T, To) < TOL_MIXED
    ref = gm.build(b, c, d, n, leaf)
    assert rel_mat(ref.dtn(), To) < 1e-9


def test_non_finite_mixed_result_is_caught(gm):
    """Diffusion-Convection II (b = 1000) at 512 x 512: the mixed build's block-local
    elimination leaves the double-float range on the way and its T is not finite.  The
    root reports that like a non-finite pivot: the automatic mode rebuilds the problem in
    FP64 (and matches the FP64 build), a build with block pivoting forced returns
    GM_ESINGULAR instead of NaN."""
    import numpy as np
    n, leaf = 512, 16
    f = inputs.paper_problem("diffconv2", n)
    op = gm.build(*f, n, leaf, precision=gm.PREC_MIXED)
    T = op.dtn()
    assert np.isfinite(T).all()
    assert op.info()["pivot_fallback"] == 1
    assert rel_mat(T, gm.build(*f, n, leaf).dtn()) < 1e-13
    with pytest.raises(gm.GmError) as e:
        gm.build(*f, n, leaf, precision=gm.PREC_MIXED, pivoting=gm.PIVOT_BLOCK)
    assert e.value.code == gm.GM_ESINGULAR


@pytest.fixture(scope="module")
def oracle_256():
    n, leaf = 256, 16
    b, c, d = inputs.convection_fields(n, seeds=(41, 42, 43))
    return (b, c, d, n, leaf), nd_dense.build(b, c, d, n, leaf).T


@pytest.mark.parametrize("tune", ["", "early=1", "a11=1", "upd_tiles=-1", "upd_tiles=2", "upd_tiles=4",
                                  "rtile32_max=0", "rtile32_max=1073741824", "tc_min_k=448",
                                  "tc_min_k=1073741824", "early=1,upd_tiles=-1"])
def test_every_schedule_the_autotuner_may_choose(gm, oracle_256, monkeypatch, tune):
    """The autotuner picks, per plan, among launch shapes and schedules of the blocked
    sweep (R tile width, tiles per CTA of the pipelined update or the one-tile kernel, the
    early-factor and A11-first schedules, the tcgen05 threshold of the merge update).
    Each, forced through GM_TUNE, builds the 256 x 256 convection problem to the mixed
    bound against O2."""
    monkeypatch.setenv("GM_TUNE", tune)
    args, To = oracle_256
    op = gm.build(*args, precision=gm.PREC_MIXED)
    assert op.info()["pivot_fallback"] == 0
    assert rel_mat(op.dtn(), To) < TOL_MIXED
