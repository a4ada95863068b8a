"""Body loads (Section 6.3: dudn = T g + F f_hat) and conductance networks (Section 6.1,
Random Laplacian I and II) on the GPU, through the C ABI, against the oracle.  Loads: F element by element against O1's one-solve-per-load definition on ragged
trees with loads on the outer ring, the merge interfaces and leaf rings; T unchanged by
the loads; the combined solve with host and device buffers; and at 512 x 512 with 1000
loads (the paper's largest N_body) the conservation and maximum-principle properties of
a Laplace problem, which hold at any size.  Networks: T and F against O1's network
solve, unit conductivities against the Laplace build, and the paper's body-load workload
(Random Laplacian I, 512 x 512, 1000 loads) against symmetry, T 1 = 0 and conservation."""
import numpy as np
import pytest

import paper_1302_5995_gb300 as gm
from oracle import o1
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def placed_loads(n, count, seed):
    body = [int(g) for g in inputs.body_nodes(n, count, seed)]
    for g in (0, n - 1, (n // 2) * n + 3, (n // 2 - 1) * n + n // 2, n * n - 1):
        if g not in body:
            body.append(g)
    return np.array(body, dtype=np.int32)


@pytest.mark.parametrize("n,leaf,count", [(9, 4, 6), (23, 6, 12), (37, 5, 30), (64, 16, 100)])
def test_load_operator_matches_o1(n, leaf, count):
    b, c, d = inputs.convection_fields(n, seeds=(91, 92, 93))
    body = placed_loads(n, count, n)
    op = gm.build_loads(b, c, d, n, leaf, body)
    F = op.load_operator()
    assert F.shape == (4 * n, body.size)
    assert rel(F, o1.load_matrix(b, c, d, n, body)) < 1e-10
    T_plain = gm.build(b, c, d, n, leaf).dtn()
    assert rel(op.dtn(), T_plain) < 1e-13
    info = op.info()
    assert info["resident_bytes"] == (16 * n * n + 4 * n * body.size) * 8


def test_solve_with_loads_host_and_device():
    torch = pytest.importorskip("torch")
    n, leaf = 48, 8
    b, c, d = inputs.convection_fields(n, seeds=(94, 95, 96))
    body = placed_loads(n, 40, 7)
    op = gm.build_loads(b, c, d, n, leaf, body)
    G = inputs.gaussian_vectors(n, 5, 8)
    Fl = inputs.body_load_vectors(body.size, 5, 9)
    ref = o1.apply_loads(b, c, d, n, G, body, Fl)
    g_cols = np.ascontiguousarray(G.T)   # vector j contiguous
    f_cols = np.ascontiguousarray(Fl.T)
    host = op.solve_loads(g_cols, f_cols).T
    assert rel(host, ref) < 1e-10
    dev = op.solve_loads(torch.from_numpy(g_cols).cuda(), torch.from_numpy(f_cols).cuda())
    torch.cuda.synchronize()
    assert rel(dev.cpu().numpy().T, ref) < 1e-10
    # the plain solve of the same handle is the T g term alone
    assert rel(op.solve(g_cols).T, o1.dtn_apply(b, c, d, n, G)) < 1e-10


def test_load_operator_at_512_conserves_and_stays_in_bounds():
    n, leaf = 512, 16
    h = 1.0 / (n + 1)
    b, c, d = inputs.laplace_fields(n)
    body = inputs.body_nodes(n, 1000, 11).astype(np.int32)
    F = gm.build_loads(b, c, d, n, leaf, body).load_operator()
    np.testing.assert_allclose(F.sum(axis=0), -h, rtol=1e-9)  # every load leaves by the boundary
    # F = -h times a harmonic measure, which is positive everywhere in the square
    assert F.max() < 0.0 and F.min() >= -h * (1 + 1e-9)


def test_plain_handle_has_no_load_operator():
    n = 16
    b, c, d = inputs.laplace_fields(n)
    op = gm.build(b, c, d, n, 8)
    with pytest.raises(gm.GmError) as e:
        op.load_operator()
    assert e.value.code == gm.GM_EUNSUPPORTED


@pytest.mark.parametrize("make", [inputs.random_laplacian_1, inputs.random_laplacian_2])
@pytest.mark.parametrize("n,leaf", [(23, 6), (40, 8)])
def test_network_dtn_and_loads_match_o1(make, n, leaf):
    sx, sy = make(n)
    T = gm.build_network(sx, sy, n, leaf).dtn()
    T_ref = o1.net_dtn_matrix(sx, sy, n)
    assert rel(T, T_ref) < 1e-10
    body = placed_loads(n, 10, n + 1)
    op = gm.build_network(sx, sy, n, leaf, body)
    assert rel(op.load_operator(), o1.net_load_matrix(sx, sy, n, body)) < 1e-10
    assert rel(op.dtn(), T_ref) < 1e-10


def test_unit_network_is_the_laplace_build():
    n, leaf = 32, 8
    ones = np.ones(n * (n + 1))
    T_net = gm.build_network(ones, ones, n, leaf).dtn()
    T_lap = gm.build(*inputs.laplace_fields(n), n, leaf).dtn()
    assert rel(T_net, T_lap) < 1e-13


def test_random_laplacian_512_with_1000_loads():
    n, leaf = 512, 16
    h = 1.0 / (n + 1)
    sx, sy = inputs.random_laplacian_1(n)
    body = inputs.body_nodes(n, 1000, 12).astype(np.int32)
    op = gm.build_network(sx, sy, n, leaf, body)
    T, F = op.dtn(), op.load_operator()
    scale = np.abs(T).max()
    assert np.abs(T - T.T).max() < 1e-10 * scale  # reciprocity of the network
    assert np.abs(T.sum(axis=1)).max() < 1e-10 * scale  # constants carry no current
    np.testing.assert_allclose(F.sum(axis=0), -h, rtol=1e-9)
    assert F.max() < 0.0 and F.min() >= -h * (1 + 1e-9)


def test_network_keeps_every_level_schur_complement():
    """Per-level parity for a network: every kept box's Schur complement (leaves, half
    boxes, boxes) against the oracle's direct elimination of that box."""
    from oracle import nd_dense
    n, leaf = 24, 6
    sx, sy = inputs.random_laplacian_2(n)
    op = gm.build_network(sx, sy, n, leaf, keep_levels=True)
    prob = nd_dense.Problem.network(sx, sy, n)
    levels = nd_dense.quad_tree(n, leaf)
    boxes = list(levels[-1])
    for lev in range(len(levels) - 1, 0, -1):
        for p in levels[lev - 1]:
            sw, se, nw, ne = p.children()
            boxes += [nd_dense.Box(p.x0, p.y0, p.a, sw.b), nd_dense.Box(p.x0, p.y0 + sw.b, p.a, nw.b), p]
    for bx in boxes:
        S = op.schur(bx.x0, bx.y0, bx.a, bx.b)
        ref = nd_dense.direct_schur(prob, bx)
        assert rel(S, ref) < 1e-11, bx


@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_low_rank_load_operator_against_o1(tol):
    """Section 6.3's low-rank form of F: L R from a Gaussian sample of F, truncated at tol.
    It stays within 100 tol of O1's F, its rank is far below the number of loads and
    falls as tol grows, and the load solve through L (R f) matches O1 within the same
    bound; the handle's footprint shrinks accordingly."""
    n, leaf, count = 96, 12, 300
    b, c, d = inputs.convection_fields(n, seeds=(97, 98, 99))
    body = placed_loads(n, count, 12)
    op = gm.build_loads(b, c, d, n, leaf, body)
    dense_bytes = op.info()["resident_bytes"]
    assert op.info()["load_rank"] == -1
    Fo = o1.load_matrix(b, c, d, n, body)
    k = op.compress_loads(tol)
    assert 0 < k < body.size // 2
    assert op.info()["load_rank"] == k
    assert op.info()["resident_bytes"] == (16 * n * n + (4 * n + body.size) * k) * 8 < dense_bytes
    assert rel(op.load_operator(), Fo) < 100 * tol
    G = inputs.gaussian_vectors(n, 4, 13)
    Fl = inputs.body_load_vectors(body.size, 4, 14)
    ref = o1.apply_loads(b, c, d, n, G, body, Fl)
    got = op.solve_loads(np.ascontiguousarray(G.T), np.ascontiguousarray(Fl.T)).T
    assert rel(got, ref) < 100 * tol
    with pytest.raises(gm.GmError) as e:  # already compressed
        op.compress_loads(tol)
    assert e.value.code == gm.GM_EUNSUPPORTED
    if tol == 1e-9:
        k6 = gm.build_loads(b, c, d, n, leaf, body).compress_loads(1e-6)
        assert k6 < k
