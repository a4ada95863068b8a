"""The mixed build eliminates a leaf's interior one grid line at a time (block
tridiagonal elimination; a reading of eq. def_schur_nd, Section 3.1): eliminating line
jj with the lines below already gone is

    [P | Q] = T^{-1} [C' | N],   S -= C P,
    T' = D - S_next Q,   C_next = direct - C Q,   C'_next = direct - S_next P,

which must give the leaf Schur complement A_bb - A_bi A_ii^{-1} A_ib exactly (up to
rounding).  Checked here in numpy against the oracle's dense leaf Schur complement, on a
square and a rectangular leaf of a convection-diffusion problem; a recursion that forgets
the C' update must fail the same check.
"""
import numpy as np
import pytest

from oracle import nd_dense
from paper_1302_5995_gb300 import inputs


def line_schur(prob, box, keep_cprime_update=True):
    """Leaf Schur complement by eliminating the interior lines bottom to top."""
    K = box.ring()
    lines = [[(box.x0 + 1 + i, box.y0 + 1 + j) for i in range(box.a - 2)] for j in range(box.b - 2)]
    A = prob.A_block
    S = A(K, K)
    C, Cp, T = A(K, lines[0]), A(lines[0], K), A(lines[0], lines[0])
    for jj, line in enumerate(lines):
        P = np.linalg.solve(T, Cp)
        S = S - C @ P
        if jj + 1 == len(lines):
            break
        nxt = lines[jj + 1]
        N, Sn = A(line, nxt), A(nxt, line)
        Q = np.linalg.solve(T, N)
        T = A(nxt, nxt) - Sn @ Q
        C = A(K, nxt) - C @ Q
        Cp = A(nxt, K) - Sn @ P if keep_cprime_update else A(nxt, K)
    return S


@pytest.mark.parametrize("box", [nd_dense.Box(3, 5, 16, 16), nd_dense.Box(10, 2, 9, 12)])
def test_line_elimination_is_the_leaf_schur_complement(box):
    n = 32
    b, c, d = inputs.convection_fields(n, seeds=(2, 3, 4))
    prob = nd_dense.Problem(b, c, d, n)
    ref = nd_dense.leaf_schur(prob, box)
    S = line_schur(prob, box)
    assert np.abs(S - ref).max() / np.abs(ref).max() < 1e-12


def test_dropping_the_cprime_update_is_caught():
    n = 32
    b, c, d = inputs.convection_fields(n, seeds=(2, 3, 4))
    prob = nd_dense.Problem(b, c, d, n)
    box = nd_dense.Box(3, 5, 16, 16)
    ref = nd_dense.leaf_schur(prob, box)
    S = line_schur(prob, box, keep_cprime_update=False)
    assert np.abs(S - ref).max() / np.abs(ref).max() > 1e-6
