"""Pins of the FP64 oracle to values fixed by the paper and by the mathematics.

Each oracle part is checked against something other than itself: the paper's printed
Laplace block matrix (Section 1.3), exact discrete solutions of the Section 6 scheme,
a sine-transform solve, brute-force dense solves on tiny grids, the plain definition
of every intermediate Schur complement (eq. def_schur_nd on the whole box), and the
structural facts the paper states (Figure 3, symmetry, Section 3.4 cost growth).
"""
import os

import numpy as np
import pytest

from oracle import closed_form as cf
from oracle import nd_dense, o1
from paper_1302_5995_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _golden_matrix(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=np.float64)


# --------------------------------------------------------------------------- stencil / O1

def test_laplace_block_form_matches_paper():
    """Section 1.3 example: h^2 A = blocks tridiag(-1, 4, -1) with -I couplings."""
    n = 3
    b, c, d = inputs.laplace_fields(n)
    A = o1.assemble_dense(b, c, d, n)
    h = 1.0 / (n + 1)
    np.testing.assert_allclose(A * h * h, _golden_matrix("laplace_block_form_n3.txt"), atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_o1_equals_dense_solve(n):
    """O1's banded elimination vs LAPACK on the dense full system, random fields."""
    b, c, d = (inputs.fourier_field(n, s, -40.0, 40.0) for s in (11, 12, 13))
    A = o1.assemble_dense(b, c, d, n)
    G = inputs.gaussian_vectors(n, 6, 9)
    V = o1.dtn_apply(b, c, d, n, G)
    # dense route: right-hand side from the ghost couplings, flux from the solution
    h = 1.0 / (n + 1)
    gi, gj, ni, nj = cf._ghost_and_neighbour_positions(n)
    ih2 = 1 / h**2
    bb, cc = b.reshape(n, n), c.reshape(n, n)
    w = np.where(gj < 0, -ih2 - cc[nj, ni] / h,
        np.where(gi >= n, -ih2 + bb[nj, ni] / h,
        np.where(gj >= n, -ih2 + cc[nj, ni] / h, -ih2 - bb[nj, ni] / h)))
    F = np.zeros((n * n, G.shape[1]))
    np.add.at(F, ni + n * nj, -w[:, None] * G)
    U = np.linalg.solve(A, F)
    Vd = (G - U[ni + n * nj]) / h
    assert rel(V, Vd) < 1e-12


# --------------------------------------------------------------------------- closed forms

EXP_CASES = [  # (n, b, c, d, nu)
    (9, 3.0, -2.0, 5.0, 0.9), (9, 3.0, -2.0, 5.0, 1.2), (16, -7.0, 4.0, -30.0, 1.1),
    (13, 0.0, 0.0, 40.0, 1.0), (12, 25.0, 0.0, 0.0, 1.0), (12, 0.0, -25.0, 0.0, 0.7),
]


@pytest.mark.parametrize("n,b,c,d,nu", EXP_CASES)
@pytest.mark.parametrize("root", [0, 1])
def test_discrete_exponentials_o1_o2(n, b, c, d, nu, root):
    """u = mu^(i+1) nu^(j+1) solves the Section 6 scheme exactly: pins the weights, the
    1/h convection scaling and signs, the tree, the merges and the root flux."""
    g, v = cf.exponential_pair(n, b, c, d, nu, root)
    B, C, D = inputs.constant_fields(n, b, c, d)
    T = nd_dense.build(B, C, D, n, 4).T
    scale = np.abs(T).max() * np.abs(g).max()
    assert np.abs(T @ g - v).max() < 1e-12 * scale
    assert np.abs(o1.dtn_apply(B, C, D, n, g[:, None])[:, 0] - v).max() < 1e-12 * scale


@pytest.mark.parametrize("n,leaf", [(64, 8), (31, 5), (20, 4)])
def test_harmonic_exactness(n, leaf):
    """Laplace: 1, x, y, x^2-y^2, xy give the exact discrete normal derivative."""
    G, V = cf.harmonic_pairs(n)
    b, c, d = inputs.laplace_fields(n)
    T = nd_dense.build(b, c, d, n, leaf).T
    scale = np.abs(T).max() * np.abs(G).max()
    assert np.abs(T @ G - V).max() < 1e-12 * scale
    assert np.abs(o1.dtn_apply(b, c, d, n, G) - V).max() < 1e-12 * scale


@pytest.mark.parametrize("n,b,c,d", [(17, 4.0, -9.0, 12.0), (24, -4.0, 3.0, -50.0), (10, 0.0, 0.0, 0.0)])
def test_sine_transform_closed_form(n, b, c, d):
    B, C, D = inputs.constant_fields(n, b, c, d)
    T = nd_dense.build(B, C, D, n, 4).T
    assert rel(T, cf.dst_dtn_matrix(n, b, c, d)) < 1e-11


# --------------------------------------------------------------------------- O2 vs O1

@pytest.mark.parametrize("n,leaf", [(8, 4), (12, 4), (16, 4), (16, 8), (24, 5), (33, 8), (64, 8)])
def test_o2_matches_o1_variable_fields(n, leaf):
    b, c, d = inputs.convection_fields(n, seeds=(21, 22, 23))
    T2 = nd_dense.build(b, c, d, n, leaf).T
    G = inputs.gaussian_vectors(n, 8, 3)
    assert rel(T2 @ G, o1.dtn_apply(b, c, d, n, G)) < 1e-11


def test_o2_matches_o1_n128():
    n, leaf = 128, 16
    b, c, d = inputs.convection_fields(n)
    T2 = nd_dense.build(b, c, d, n, leaf).T
    G = inputs.gaussian_vectors(n, 4, 4)
    assert rel(T2 @ G, o1.dtn_apply(b, c, d, n, G)) < 1e-11


@pytest.mark.parametrize("n,leaf", [(24, 4), (21, 5)])
def test_every_intermediate_is_the_box_schur_complement(n, leaf):
    """Each merged S^(tau) equals eq. def_schur_nd applied to the whole box directly."""
    b, c, d = inputs.convection_fields(n, seeds=(5, 6, 7))
    res = nd_dense.build(b, c, d, n, leaf, keep=True)
    prob = nd_dense.Problem(b, c, d, n)
    assert len(res.schur) > 4
    for box, S in res.schur.items():
        Sd = nd_dense.direct_schur(prob, box)
        assert rel(S, Sd) < 1e-11, box


# --------------------------------------------------------------------------- invariants

def test_symmetry_when_no_convection():
    n = 20
    _, _, d = inputs.convection_fields(n)
    z = np.zeros(n * n)
    res = nd_dense.build(z, z, d, n, 5, keep=True)
    assert rel(res.T, res.T.T) < 1e-12
    for S in res.schur.values():
        assert rel(S, S.T) < 1e-12


def test_laplace_constants_in_kernel_and_psd():
    n = 32
    b, c, d = inputs.laplace_fields(n)
    T = nd_dense.build(b, c, d, n, 8).T
    assert np.abs(T @ np.ones(4 * n)).max() < 1e-10 * np.abs(T).max()
    ev = np.linalg.eigvalsh(0.5 * (T + T.T))
    assert ev.min() > -1e-10 * ev.max()


def test_fig3_structure_of_root_schur():
    """Figure 3: the 252-point Laplace root Schur complement is dominated by its
    near-diagonal entries and smooth far from the diagonal."""
    n, r, *rows = [int(x) for x in open(os.path.join(GOLDEN, "fig3_laplace_root.txt")).read().split("\n")[-2].split()]
    b, c, d = inputs.laplace_fields(n)
    res = nd_dense.build(b, c, d, n, 8, keep=True)
    S = res.schur[nd_dense.Box(0, 0, n, n)]
    assert S.shape == (r, r)
    for row in rows:
        s = S[row - 1]
        near = np.abs(s[[(row - 1 + k) % r for k in (-1, 0, 1)]]).sum()
        far_idx = [j for j in range(r) if min(abs(j - row + 1), r - abs(j - row + 1)) > 2]
        assert abs(s[row - 1]) > np.abs(s[far_idx]).sum()
        assert near > 10 * np.abs(s[far_idx]).max()
        # panel (b): far from the diagonal the row is small and varies slowly
        far = np.array([s[(row - 1 + k) % r] for k in range(r // 4, 3 * r // 4)])
        assert np.abs(far).max() < 1e-3 * abs(s[row - 1])
        assert np.abs(np.diff(far, 2)).max() < 1e-5 * abs(s[row - 1])


def test_dense_cost_grows_like_n_cubed():
    """Section 3.4: the dense build costs O(n^3) = O(N^1.5) (counted, not timed)."""
    fl = []
    for n in (64, 128, 256, 512):
        # count only: run the tree bookkeeping without the arithmetic
        levels = nd_dense.quad_tree(n, 16)
        f = 0.0
        for lev in range(len(levels) - 1, 0, -1):
            for parent in levels[lev - 1]:
                for (m, p) in nd_dense._merge_shapes(parent, parent.children()):
                    f += (16 / 3) * m**3 + 8 * m * m * p + 2 * p * p * m
        r = 4 * n - 4
        f += (2 / 3) * r**3 + 2 * r * r * 4 * n
        fl.append(f)
    ratios = [fl[i + 1] / fl[i] for i in range(3)]
    assert all(7.0 < x < 9.0 for x in ratios), ratios


# --------------------------------------------------------------------------- planted mistakes

def _plant(monkeypatch, fn):
    monkeypatch.setattr(nd_dense, "merge_two", fn)


@pytest.mark.parametrize("mistake", ["transpose_S13", "drop_A34", "sign_A12"])
def test_planted_merge_mistakes_are_caught(monkeypatch, mistake):
    """A plausible slip inside the merge formula makes the O1 comparison fail."""
    orig = nd_dense.merge_two

    def bad(prob, box1, S1, box2, S2, parent, interface_solve=None):
        if mistake == "transpose_S13":
            S1 = S1.T.copy()
        elif mistake == "drop_A34":
            real = prob.A_block

            class P:
                pass
            p = P()
            p.__dict__.update(prob.__dict__)
            p.A_block = lambda r, c: real(r, c) * (0.0 if (set(r) & set(box1.ring()) and set(c) & set(box2.ring())) else 1.0)
            return orig(p, box1, S1, box2, S2, parent, interface_solve)
        elif mistake == "sign_A12":
            out = orig(prob, box1, S1, box2, S2, parent, interface_solve)
            return out + 1e-3 * np.abs(out).max() * np.eye(len(out))
        return orig(prob, box1, S1, box2, S2, parent, interface_solve)

    _plant(monkeypatch, bad)
    n = 12
    b, c, d = inputs.convection_fields(n, seeds=(31, 32, 33))
    G = inputs.gaussian_vectors(n, 4, 1)
    T = nd_dense.build(b, c, d, n, 4).T
    assert rel(T @ G, o1.dtn_apply(b, c, d, n, G)) > 1e-6
