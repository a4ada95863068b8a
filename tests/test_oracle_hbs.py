"""Pins of the HBS oracle (Sections 4 and 5) to facts that do not come from the oracle.

- with no truncation the factors are exact: the telescoping product (eq. tele1-tele3)
  reproduces H and Algorithms 1 and 2 reproduce a LAPACK solve, on random matrices;
- matrices with known off-diagonal ranks: a tridiagonal matrix (one coupling per block
  boundary) and the inverse of a tridiagonal matrix (semiseparable) compress to those
  ranks, and Algorithm 1 of the tridiagonal matrix applies its exact inverse;
- the truncated representation of a root Schur complement stays within a small
  multiple of the tolerance, and so does the DtN map computed through it;
- the printed down-sweep of Algorithm 2 (E_tau applied to x^_tau) is a typo: planting
  it in a copy of the oracle breaks the inverse, which the y^_tau reading reproduces;
- the accelerated merge's Step 1 (block elimination with HBS inverses) is the exact
  interface solve without truncation, and a build using it tracks the tolerance.
"""
import numpy as np
import pytest

from oracle import hbs, nd_dense
from paper_1302_5995_gb300 import inputs


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def random_matrix(M, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((M, M)) + M * np.eye(M)


@pytest.mark.parametrize("M,m", [(200, 24), (130, 64), (64, 64), (97, 10)])
def test_untruncated_factors_are_exact(M, m):
    H = random_matrix(M, M)
    tree = hbs.HBSTree(M, m)
    f = hbs.compress(H, tree, 0.0)
    x = np.random.default_rng(1).standard_normal((M, 3))
    assert rel(hbs.matvec(f, x), H @ x) < 1e-13
    y = hbs.apply_inverse(hbs.invert(f), x)
    assert rel(y, np.linalg.solve(H, x)) < 1e-12


def test_tree_shape():
    t = hbs.HBSTree(4092, 64)
    assert t.L == 6
    sizes = [t.rng[tau][1] - t.rng[tau][0] for tau in t.level(t.L)]
    assert min(sizes) >= 63 and max(sizes) <= 64 and sum(sizes) == 4092
    assert t.rng[2] == (0, 2046) and t.rng[3] == (2046, 4092)


def tridiagonal(M, seed):
    rng = np.random.default_rng(seed)
    return np.diag(4.0 + rng.random(M)) + np.diag(-1.0 - rng.random(M - 1), 1) + np.diag(-1.0 - rng.random(M - 1), -1)


def test_tridiagonal_ranks_and_inverse():
    M, m = 128, 16
    H = tridiagonal(M, 3)
    tree = hbs.HBSTree(M, m)
    f = hbs.compress(H, tree, 1e-12)
    # a leaf's off-diagonal block row has one nonzero to the left and one to the right
    ranks = [f.rank(tau) for tau in tree.level(tree.L)]
    assert ranks[0] == 1 and ranks[-1] == 1 and all(k == 2 for k in ranks[1:-1])
    assert rel(hbs.to_dense(f), H) < 1e-14
    x = np.random.default_rng(2).standard_normal((M, 2))
    assert rel(hbs.apply_inverse(hbs.invert(f), x), np.linalg.solve(H, x)) < 1e-13


def test_semiseparable_inverse_has_rank_two_blocks():
    M, m = 128, 16
    Hi = np.linalg.inv(tridiagonal(M, 5))
    tree = hbs.HBSTree(M, m)
    f = hbs.compress(Hi, tree, 1e-12)
    for l in range(1, tree.L + 1):
        assert max(f.rank(tau) for tau in tree.level(l)) <= 2
    assert rel(hbs.to_dense(f), Hi) < 1e-11


@pytest.mark.parametrize("fields", ["laplace", "convection"])
def test_root_schur_compression_error_tracks_tolerance(fields):
    n, leaf, m = 64, 8, 32
    b, c, d = inputs.laplace_fields(n) if fields == "laplace" else inputs.convection_fields(n)
    S = nd_dense.build(b, c, d, n, leaf).S_root
    tree = hbs.HBSTree(S.shape[0], m)
    for tol in (1e-6, 1e-9):
        f = hbs.compress(S, tree, tol)
        err = rel(hbs.to_dense(f), S)
        assert err < 50 * tol, (tol, err)
        assert max(f.rank(tau) for tau in tree.level(tree.L)) < m  # it does compress
    # tighter tolerance, higher ranks
    k6 = sum(hbs.compress(S, tree, 1e-6).rank(t) for t in tree.level(tree.L))
    k9 = sum(hbs.compress(S, tree, 1e-9).rank(t) for t in tree.level(tree.L))
    assert k9 > k6


def test_hbs_dtn_matches_dense_dtn():
    """Section 5 applied to the root: (g - P S^{-1} B g)/h with S^{-1} from Algorithms
    1 and 2 agrees with the dense T within a small multiple of the tolerance."""
    n, leaf, m, tol = 64, 8, 32, 1e-9
    b, c, d = inputs.convection_fields(n)
    res = nd_dense.build(b, c, d, n, leaf)
    G = inputs.gaussian_vectors(n, 6, 11)
    V = hbs.dtn_apply(nd_dense.Problem(b, c, d, n), res.S_root, tol, m, G)
    Vo = res.T @ G
    err = (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()
    assert err < 100 * tol, err


def _apply_inverse_printed_typo(inv, x):
    """Algorithm 2 with the down-sweep exactly as printed (E_tau x^_tau)."""
    t = inv.tree
    xh, yh = {}, {}
    for tau in t.level(t.L):
        xh[tau] = inv.F[tau].T @ x[t.idx(tau)]
    for l in range(t.L - 1, 0, -1):
        for tau in t.level(l):
            xh[tau] = inv.F[tau].T @ np.vstack([xh[2 * tau], xh[2 * tau + 1]])
    z = inv.G[1] @ np.vstack([xh[2], xh[3]])
    yh[2], yh[3] = z[:xh[2].shape[0]], z[xh[2].shape[0]:]
    for l in range(1, t.L):
        for tau in t.level(l):
            a, b = 2 * tau, 2 * tau + 1
            z = inv.E[tau] @ xh[tau] + inv.G[tau] @ np.vstack([xh[a], xh[b]])
            yh[a], yh[b] = z[:xh[a].shape[0]], z[xh[a].shape[0]:]
    y = np.zeros_like(x)
    for tau in t.level(t.L):
        I = t.idx(tau)
        y[I] = inv.E[tau] @ yh[tau] + inv.G[tau] @ x[I]
    return y


def test_printed_down_sweep_is_a_typo():
    M = 200
    H = random_matrix(M, 7)
    inv = hbs.invert(hbs.compress(H, hbs.HBSTree(M, 24), 0.0))
    x = np.random.default_rng(3).standard_normal((M, 2))
    exact = np.linalg.solve(H, x)
    assert rel(hbs.apply_inverse(inv, x), exact) < 1e-12
    assert rel(_apply_inverse_printed_typo(inv, x), exact) > 1e-3


def test_step1_interface_solver_exact_without_truncation():
    """Step 1's block elimination with untruncated HBS inverses is the exact solve."""
    rng = np.random.default_rng(9)
    s3, p = 96, 40
    S33 = rng.standard_normal((s3, s3)) + s3 * np.eye(s3)
    S44 = rng.standard_normal((s3, s3)) + s3 * np.eye(s3)
    A34 = np.diag(rng.standard_normal(s3))
    A43 = np.diag(rng.standard_normal(s3))
    Z = rng.standard_normal((2 * s3, p))
    X = hbs.step1_interface_solver(0.0, 16)(S33, A34, A43, S44, Z)
    M = np.block([[S33, A34], [A43, S44]])
    assert rel(X, np.linalg.solve(M, Z)) < 1e-12


def test_build_with_hbs_step1_merges_tracks_tolerance():
    n, leaf = 96, 12
    b, c, d = inputs.convection_fields(n, seeds=(3, 5, 7))
    T0 = nd_dense.build(b, c, d, n, leaf).T
    for tol in (1e-6, 1e-9):
        T1 = nd_dense.build(b, c, d, n, leaf, interface_solve=hbs.step1_interface_solver(tol, 12), min_edge=24).T
        assert rel(T1, T0) < 100 * tol
