"""The mixed build's interface solve is a blocked Gauss-Jordan sweep on [M | Z] with
block-local pivoting (the pivot block inverted in FP32, X0 ~ A11^{-1}) and one step of
iterative refinement per block:

    R0 = X0 A12,   E = A12 - A11 R0,   R = R0 + X0 E,   W(i, :) -= W(i, J) R  (i not in J),

after which the right block of W holds M^{-1} Z.  Checked here in numpy (FP32 inverse,
FP64 elsewhere) on a merge's interface system from the oracle: with the refinement the
result is accurate far beyond FP32; without it, it is not.  The last test restates the
in-place panel form in which the block factor forms X0 (rows never move, each panel's
transform takes the place of the panel's columns) and checks it against A^{-1}.
"""
import functools

import numpy as np
import pytest

from oracle import nd_dense
from paper_1302_5995_gb300 import inputs


def blocked_gj(M, Z, nb, refine=True):
    m = M.shape[0]
    W = np.hstack([M, Z]).astype(np.float64)
    for k in range(0, m, nb):
        J = slice(k, min(k + nb, m))
        A11 = W[J, J]
        X0 = np.linalg.inv(A11.astype(np.float32)).astype(np.float64)  # FP32 block inverse
        A12 = W[J, k + A11.shape[0]:]
        R = X0 @ A12
        if refine:
            R = R + X0 @ (A12 - A11 @ R)
        F = W[:, J].copy()
        F[J, :] = 0.0
        W[:, k + A11.shape[0]:] -= F @ R
        W[J, k + A11.shape[0]:] = R
    return W[:, m:]


@functools.lru_cache(maxsize=None)
def interface_system(n=40, leaf=10, seeds=(11, 12, 13)):
    """[M | Z] of the top vertical merge of an n x n convection problem (oracle O2)."""
    b, c, d = inputs.convection_fields(n, seeds=seeds)
    prob = nd_dense.Problem(b, c, d, n)
    root = nd_dense.Box(0, 0, n, n)
    sw, se, nw, ne = root.children()
    south, north = nd_dense.Box(0, 0, n, sw.b), nd_dense.Box(0, sw.b, n, nw.b)
    # the two halves' Schur complements by direct elimination, then the merge's blocks
    S1, S2 = nd_dense.direct_schur(prob, south), nd_dense.direct_schur(prob, north)
    r1, r2 = south.ring(), north.ring()
    p3 = [q for q in r1 if q[1] == south.y0 + south.b - 1 and 0 < q[0] < n - 1]
    p4 = [q for q in r2 if q[1] == north.y0 and 0 < q[0] < n - 1]
    i3 = [r1.index(q) for q in p3]
    i4 = [r2.index(q) for q in p4]
    S33, S44 = S1[np.ix_(i3, i3)], S2[np.ix_(i4, i4)]
    A34, A43 = prob.A_block(p3, p4), prob.A_block(p4, p3)
    M = np.block([[S33, A34], [A43, S44]])
    o1 = [j for j in range(len(r1)) if j not in i3]
    o2 = [j for j in range(len(r2)) if j not in i4]
    Z = np.block([[S1[np.ix_(i3, o1)], np.zeros((len(i3), len(o2)))],
                  [np.zeros((len(i4), len(o1))), S2[np.ix_(i4, o2)]]])
    return M, Z


@pytest.mark.parametrize("nb", [8, 16])
def test_blocked_gauss_jordan_with_refinement(nb):
    M, Z = interface_system()
    X = np.linalg.solve(M, Z)
    ok = blocked_gj(M, Z, nb)
    bad = blocked_gj(M, Z, nb, refine=False)
    err = lambda Y: np.abs(Y - X).max() / np.abs(X).max()
    assert err(ok) < 1e-11
    assert err(bad) > 1e-9  # FP32 block inverses alone stay near FP32 accuracy


@pytest.mark.parametrize("nb", [64, 128, 256])
def test_larger_blocks_keep_the_accuracy(nb):
    """The 128 x 128 workload's top merge (m = 252) swept with the block width of the
    kernels (64) and wider ones: one refinement step reaches 1e-14 for each, and the FP32
    block inverses alone stay near FP32 accuracy."""
    M, Z = interface_system(n=128, leaf=16, seeds=(1, 2, 3))
    X = np.linalg.solve(M, Z)
    err = lambda Y: np.abs(Y - X).max() / np.abs(X).max()
    assert err(blocked_gj(M, Z, nb)) < 1e-13
    assert err(blocked_gj(M, Z, nb, refine=False)) > 1e-9


def panel_gauss_jordan_in_place(A, panel=8, mistake=None):
    """X0 = A^{-1} the way the block factor forms it: Gauss-Jordan with partial pivoting
    among the unused rows (rows never move), panels of `panel` pivots, in place on the
    n x n slots.  Panel q's transform T (n x panel) maps the slots S to [r not in P] S[r] +
    T[r] S[P] on every slot outside the panel; the panel's own slots become T's columns
    (on [A | I] these are the right-hand columns of the pivot rows, which start as unit
    columns).  At the end slot (r, t) is entry (r, p_t) of the right half, so
    X0[t, i] = S[p_t, step[i]].  `mistake` plants one error, for the test below."""
    n = A.shape[0]
    S = A.astype(np.float64).copy()
    used = np.zeros(n, bool)
    step = np.zeros(n, int)
    prow = np.zeros(n, int)
    for t0 in range(0, n, panel):
        w = min(panel, n - t0)
        pv = S[:, t0:t0 + w].copy()
        T = np.zeros((n, w))
        P = []
        for u in range(w):
            p = int(np.argmax(np.where(used, -1.0, np.abs(pv[:, u]))))
            used[p] = True
            P.append(p)
            T[p, u] = 1.0
            prv, prt, ip = pv[p].copy(), T[p].copy(), 1.0 / pv[p, u]
            g = pv[:, u] * ip
            pv -= np.outer(g, prv)
            T -= np.outer(g, prt)
            pv[p], T[p] = prv * ip, prt * ip
            step[p], prow[t0 + u] = t0 + u, p
        new = S.copy()
        if mistake != "keep pivot rows":
            new[P] = 0.0
        new += T @ S[P]
        if mistake != "no slot swap":
            new[:, t0:t0 + w] = T
        S = new
    if mistake == "transposed map":
        return S[np.ix_(step, prow)]
    return S[np.ix_(prow, step)]


@pytest.mark.parametrize("n,panel", [(64, 8), (64, 64), (40, 8), (17, 8)])
def test_in_place_panel_inverse(n, panel):
    """The factor's in-place reading gives A^{-1} (the identity padding beyond nbe
    included); each planted mistake in it does not."""
    rng = np.random.default_rng(n + panel)
    A = np.eye(n)
    m = n - 5 if n > 20 else n
    A[:m, :m] = rng.standard_normal((m, m))
    ref = np.linalg.inv(A)
    scale = np.abs(ref).max()
    assert np.abs(panel_gauss_jordan_in_place(A, panel) - ref).max() < 1e-10 * scale
    # (with one panel there is no slot outside it for the pivot-row mistake to spoil)
    for mistake in ("no slot swap", "transposed map") + (("keep pivot rows",) if n > panel else ()):
        bad = panel_gauss_jordan_in_place(A, panel, mistake)
        assert not np.abs(bad - ref).max() < 1e-6 * scale, mistake
