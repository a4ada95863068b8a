"""GPU parity: the CUDA build and solve, called through the C ABI, against the FP64
oracle (O2: the paper's nested dissection step by step; O1: full banded solve).

Tolerance: the all-FP64 path must match to 1e-10 relative (max-norm of the error over
max-norm of the oracle for matrices; per-vector 2-norms for Neumann data).
"""
import numpy as np
import pytest

from oracle import closed_form as cf
from oracle import nd_dense, o1
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


def rel_mat(A, B):
    return np.abs(A - B).max() / np.abs(B).max()


def solve_cols(op, G):
    """Solve for the columns of G (4n x B); the library stores vector j contiguously."""
    B = G.shape[1]
    return op.solve(np.ascontiguousarray(G.T)).reshape(B, G.shape[0]).T


def rel_vec(V, Vo):
    return (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()


def rel_vec_T(V, Vo, T, G):
    """Per-vector error relative to max(|v_o|, |T| |g|): the constant vector of a
    Laplace problem has zero Neumann data, so |v_o| alone is no scale there."""
    scale = np.maximum(np.linalg.norm(Vo, axis=0), np.linalg.norm(T, 2) * np.linalg.norm(G, axis=0) * 1e-3)
    return (np.linalg.norm(V - Vo, axis=0) / scale).max()


def test_config1_laplace_64(gm):
    cfg = inputs.config1()
    n = cfg["n"]
    op = gm.build(cfg["b"], cfg["c"], cfg["d"], n, cfg["leaf"])
    T = op.dtn()
    To = nd_dense.build(cfg["b"], cfg["c"], cfg["d"], n, cfg["leaf"]).T
    assert T.shape == (256, 256)
    assert rel_mat(T, To) < TOL
    V = solve_cols(op, cfg["G"])
    assert rel_vec_T(V, To @ cfg["G"], To, cfg["G"]) < TOL
    assert rel_vec(V[:, 1:], (To @ cfg["G"])[:, 1:]) < TOL  # all but the constant vector
    # closed form: harmonic polynomials give the exact discrete normal derivative
    G5, V5 = cf.harmonic_pairs(n)
    assert np.abs(T @ G5 - V5).max() < 1e-10 * np.abs(T).max()
    assert np.abs(T @ np.ones(4 * n)).max() < 1e-10 * np.abs(T).max()
    assert rel_mat(T, T.T) < 1e-10


@pytest.mark.parametrize("n,leaf", [(24, 4), (37, 5), (16, 8)])
def test_every_level_matches_oracle(gm, n, leaf):
    """Leaf, half-box and box Schur complements of every level (rows a1-a4)."""
    b, c, d = inputs.convection_fields(n, seeds=(41, 42, 43))
    op = gm.build(b, c, d, n, leaf, keep_levels=True)
    ref = nd_dense.build(b, c, d, n, leaf, keep=True)
    # leaves are kept by the GPU path too; the oracle keeps leaves, halves and boxes
    for box, So in ref.schur.items():
        S = op.schur(box.x0, box.y0, box.a, box.b)
        assert rel_mat(S, So) < TOL, box
    assert rel_mat(op.dtn(), ref.T) < TOL


@pytest.mark.parametrize("n,leaf", [(33, 5), (100, 7), (128, 16), (61, 16)])
def test_convection_fields_match_oracle(gm, n, leaf):
    b, c, d = inputs.convection_fields(n)
    op = gm.build(b, c, d, n, leaf)
    To = nd_dense.build(b, c, d, n, leaf).T
    T = op.dtn()
    assert rel_mat(T, To) < TOL
    G = inputs.gaussian_vectors(n, 7, 2)
    V = solve_cols(op, G)
    assert rel_vec(V, To @ G) < TOL


def test_config2_full_size_fp64(gm):
    """512 x 512 convection-diffusion-reaction, leaf 16, 256 Gaussian vectors, FP64."""
    import torch
    cfg = inputs.config2()
    n = cfg["n"]
    dev = torch.device("cuda")
    b, c, d = (torch.from_numpy(cfg[k]).to(dev) for k in "bcd")
    op = gm.build(b, c, d, n, cfg["leaf"])
    To = nd_dense.build(cfg["b"], cfg["c"], cfg["d"], n, cfg["leaf"]).T
    T = op.dtn()
    assert rel_mat(T, To) < TOL
    G = torch.from_numpy(np.ascontiguousarray(cfg["G"].T)).to(dev)  # 256 vectors, each contiguous
    V = op.solve(G)
    torch.cuda.synchronize()
    V = V.cpu().numpy().reshape(256, 4 * n).T
    assert rel_vec(V, To @ cfg["G"]) < TOL


def test_o1_full_solve_agrees_on_gpu_result(gm):
    """Independent of O2: the GPU result against the banded full-system solve."""
    n, leaf = 45, 6
    b, c, d = inputs.convection_fields(n, seeds=(7, 8, 9))
    op = gm.build(b, c, d, n, leaf)
    G = inputs.gaussian_vectors(n, 5, 11)
    V = solve_cols(op, G)
    assert rel_vec(V, o1.dtn_apply(b, c, d, n, G)) < TOL


@pytest.mark.parametrize("n,leaf", [(2, 4), (3, 4), (4, 4), (5, 4), (9, 4), (17, 17), (18, 17)])
def test_small_and_degenerate_grids(gm, n, leaf):
    """L = 0 (the whole grid is one leaf), 2 x 2 and 3 x 3 leaves, ragged splits."""
    b, c, d = inputs.convection_fields(n, seeds=(3, 4, 5))
    op = gm.build(b, c, d, n, leaf)
    To = o1.dtn_matrix(b, c, d, n)
    assert rel_mat(op.dtn(), To) < TOL


def test_host_and_device_pointers_agree(gm):
    import torch
    n, leaf = 40, 10
    b, c, d = inputs.convection_fields(n, seeds=(1, 5, 9))
    op_h = gm.build(b, c, d, n, leaf)
    dev = [torch.from_numpy(x).cuda() for x in (b, c, d)]
    op_d = gm.build(*dev, n, leaf)
    assert np.array_equal(op_h.dtn(), op_d.dtn())
    G = inputs.gaussian_vectors(n, 3, 1)
    gh = np.ascontiguousarray(G.T)
    vh = op_d.solve(gh)
    vd = op_d.solve(torch.from_numpy(gh).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(vh, vd)


def test_solve_batch_edges(gm):
    n = 20
    b, c, d = inputs.laplace_fields(n)
    op = gm.build(b, c, d, n, 5)
    T = op.dtn()
    g = inputs.gaussian_vectors(n, 1, 3)[:, 0]
    v = op.solve(g.copy())
    assert rel_vec(v[:, None], (T @ g)[:, None]) < 1e-13
    empty = np.zeros(0)
    assert op.solve(empty).size == 0


def test_errors_are_reported(gm):
    n = 8
    b, c, d = inputs.laplace_fields(n)
    with pytest.raises(gm.GmError) as e:
        gm.build(b, c, d, n, 2)
    assert e.value.code == gm.GM_EINVAL
    with pytest.raises(gm.GmError) as e:  # n = 7, leaf 3: the tree would hold 1-wide boxes (no ring)
        gm.build(*inputs.laplace_fields(7), 7, 3)
    assert e.value.code == gm.GM_EINVAL
    with pytest.raises(gm.GmError) as e:  # a 28-node root ring is one HBS node: nothing to compress
        gm.build(b, c, d, n, 4, tol=1e-9)
    assert e.value.code == gm.GM_EUNSUPPORTED
    with pytest.raises(gm.GmError) as e:
        gm.build(b, c, d, n, 4, tol=-1.0)
    assert e.value.code == gm.GM_EINVAL
    with pytest.raises(gm.GmError) as e:
        gm.build(b[:1], c[:1], d[:1], 1, 4)
    assert e.value.code == gm.GM_EINVAL


def test_singular_box_is_reported_not_faulted(gm):
    """A 3 x 3 leaf whose single interior node has a zero diagonal: an exactly singular
    Dirichlet problem -> GM_ESINGULAR, and the context stays usable."""
    n = 6  # leaf 4 -> four 3 x 3 leaves; interior node of the south-west leaf is (1, 1)
    b, c, d = inputs.laplace_fields(n)
    d = d.copy()
    # exactly minus the centre weight 4/h^2, which the library forms as 4 (n+1)^2
    d[1 + n * 1] = -4.0 * (n + 1) ** 2
    with pytest.raises(gm.GmError) as e:
        gm.build(b, c, d, n, 4)
    assert e.value.code == gm.GM_ESINGULAR
    op = gm.build(*inputs.laplace_fields(n), n, 4)  # the device still works
    assert np.isfinite(op.dtn()).all()


def test_info_reports_the_build(gm):
    n, leaf = 64, 8
    op = gm.build(*inputs.laplace_fields(n), n, leaf)
    info = op.info()
    assert info["n"] == n and info["leaf"] == leaf and info["levels"] == 3
    assert info["dtn_bytes"] == 16 * n * n * 8
    assert 0 < info["min_pivot_ratio"] <= 1.5
    assert info["bad_stage"] == -1
    assert info["launches"] > 0


@pytest.mark.parametrize("n,leaf", [(12, 3), (48, 3), (96, 32), (128, 64), (100, 64), (40, 200)])
def test_every_leaf_size_of_the_boundary(gm, n, leaf):
    """3 <= leaf <= n (and beyond): against O1, the plain definition.  Leaves wider than
    17 are eliminated in nested-dissection order inside the leaf; the reported levels are
    the requested tree's."""
    b, c, d = inputs.convection_fields(n, seeds=(n, n + 1, n + 2))
    op = gm.build(b, c, d, n, leaf)
    assert op.info()["levels"] == nd_dense.num_levels(n, leaf)
    To = o1.dtn_matrix(b, c, d, n)
    assert rel_mat(op.dtn(), To) < TOL
    if leaf >= 32:
        mx = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED)
        assert rel_mat(mx.dtn(), To) < 1e-8


def test_wide_leaf_schur_complement_is_the_leaf_elimination(gm):
    """A 64 x 64 leaf (the paper's default N_leaf = 4096 points): its Schur complement,
    kept by the build, against the oracle's dense elimination of the leaf's interior
    (eq. def_schur_nd)."""
    n, leaf = 128, 64
    b, c, d = inputs.convection_fields(n, seeds=(61, 62, 63))
    op = gm.build(b, c, d, n, leaf, keep_levels=True)
    prob = nd_dense.Problem(b, c, d, n)
    box = nd_dense.quad_tree(n, leaf)[-1][3]  # the north-east leaf
    assert (box.a, box.b) == (64, 64)
    S = op.schur(box.x0, box.y0, box.a, box.b)
    So = nd_dense.leaf_schur(prob, box)
    assert rel_mat(S, So) < TOL
