"""Oracle for the HBS part of the method -- Sections 4 and 5 of the paper.

TEST INFRASTRUCTURE ONLY: the library never imports this module.  The tests, the
smoke check and the benchmark's CPU-baseline leg are its only users.

Follows, in the paper's notation:
  Section 4 (tree)        binary tree over the index vector [0, M): node 1 is the root,
                          node tau has children 2 tau and 2 tau + 1; every node is split
                          in two halves (the first half takes floor) down to level L,
                          the smallest L with ceil(M / 2^L) <= m.
  Section 4 (HBS factors) D_tau for leaves, U_tau / V_tau for every non-root node (m x k
                          at leaves, (k1 + k2) x k at parents), B_tau for every parent,
                          B_tau = [0, Ht_{s1 s2}; Ht_{s2 s1}, 0]           (eq. def6)
  Section 4 (telescoping) H = U^(L) Ht^(L) V^(L)* + D^(L), Ht^(l+1) = U^(l) Ht^(l) V^(l)*
                          + B^(l), Ht^(1) = B^(0)                     (eq. tele1-tele3)
  Section 5, Algorithm 1  inversion: factors {E, F, G} of H^{-1}
  Section 5, Algorithm 2  y = H^{-1} x from those factors
  Section 5, Steps 1-3    the accelerated merge: block solve with HBS inverses, low-rank
                          S13 / S24 and the factored update, parent recompressed to HBS

Readings (the paper defers construction to its references):
  * compression: U_tau is an orthonormal basis of the columns of tau's off-diagonal
    block row (at a parent: the children's bases applied to it), V_tau the same for the
    block column, from a column-pivoted QR truncated at the first |R_jj| <= tol |R_11|
    -- "local tolerance" read as relative per node.  U_tau and V_tau keep the same
    number of columns (the larger of the two truncation points): Algorithm 1 inverts
    V_tau* D~_tau^{-1} U_tau, which must be square.  With orthonormal bases,
    Ht_{s t} = U_s* H(I_s, I_t) V_t (full bases).
  * Algorithm 2's down-sweep applies E_tau to y^_tau (the printed x^_tau and q^_tau are
    typos for y^_tau).
Precision: FP64.
"""
from __future__ import annotations

import numpy as np


class HBSTree:
    """Perfect binary tree of depth L over [0, M); node ids 1 .. 2^(L+1) - 1."""

    def __init__(self, M: int, m: int):
        L = 0
        while -(-M // (1 << L)) > m:
            L += 1
        self.M, self.m, self.L = M, m, L
        self.rng = {1: (0, M)}
        for tau in range(1, 1 << L):
            lo, hi = self.rng[tau]
            mid = lo + (hi - lo) // 2
            self.rng[2 * tau] = (lo, mid)
            self.rng[2 * tau + 1] = (mid, hi)

    def level(self, l):
        return range(1 << l, 1 << (l + 1))

    def is_leaf(self, tau):
        return tau >= (1 << self.L)

    def idx(self, tau):
        lo, hi = self.rng[tau]
        return np.arange(lo, hi)


def _pivoted_qr(A, tol):
    """Column-pivoted QR of A (a LAPACK library step): the orthonormal Q and the number
    of its columns before the first |R_jj| <= tol |R_11|."""
    from scipy.linalg import qr
    if A.shape[1] == 0 or A.shape[0] == 0:
        return np.zeros((A.shape[0], 0)), 0
    Q, R, _ = qr(A, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    if d.size == 0 or d[0] == 0.0:
        return Q, 0
    small = np.nonzero(d <= tol * d[0])[0]
    return Q, (int(small[0]) if small.size else d.size)


class HBS:
    """HBS factors of an M x M matrix (Section 4)."""

    def __init__(self, tree: HBSTree):
        self.tree = tree
        self.U, self.V, self.D, self.B = {}, {}, {}, {}
        self.Ufull, self.Vfull = {}, {}

    def rank(self, tau):
        return self.U[tau].shape[1]


def compress(H, tree: HBSTree, tol: float) -> HBS:
    """HBS factors of the dense matrix H at local tolerance tol (finest level first)."""
    H = np.asarray(H, dtype=np.float64)
    M = tree.M
    f = HBS(tree)
    for l in range(tree.L, 0, -1):
        for tau in tree.level(l):
            I = tree.idx(tau)
            J = np.setdiff1d(np.arange(M), I)
            if tree.is_leaf(tau):
                rows = H[np.ix_(I, J)]
                cols = H[np.ix_(J, I)]
            else:
                a, b = 2 * tau, 2 * tau + 1
                Ia, Ib = tree.idx(a), tree.idx(b)
                rows = np.vstack([f.Ufull[a].T @ H[np.ix_(Ia, J)], f.Ufull[b].T @ H[np.ix_(Ib, J)]])
                cols = np.hstack([H[np.ix_(J, Ia)] @ f.Vfull[a], H[np.ix_(J, Ib)] @ f.Vfull[b]])
            Qu, ku = _pivoted_qr(rows, tol)
            Qv, kv = _pivoted_qr(cols.T, tol)
            # one rank for both bases: Algorithm 1 inverts the k x k matrix V* D^{-1} U
            k = min(max(ku, kv), Qu.shape[1], Qv.shape[1])
            f.U[tau] = Qu[:, :k]
            f.V[tau] = Qv[:, :k]
            if tree.is_leaf(tau):
                f.D[tau] = H[np.ix_(I, I)].copy()
                f.Ufull[tau] = f.U[tau]
                f.Vfull[tau] = f.V[tau]
            else:
                a, b = 2 * tau, 2 * tau + 1
                f.Ufull[tau] = _blkdiag(f.Ufull[a], f.Ufull[b]) @ f.U[tau]
                f.Vfull[tau] = _blkdiag(f.Vfull[a], f.Vfull[b]) @ f.V[tau]
    # B_tau for every parent (eq. def6): interactions of its two children
    for l in range(tree.L - 1, -1, -1):
        for tau in tree.level(l):
            a, b = 2 * tau, 2 * tau + 1
            Ia, Ib = tree.idx(a), tree.idx(b)
            Hab = f.Ufull[a].T @ H[np.ix_(Ia, Ib)] @ f.Vfull[b]
            Hba = f.Ufull[b].T @ H[np.ix_(Ib, Ia)] @ f.Vfull[a]
            ka, kb = Hab.shape
            f.B[tau] = np.block([[np.zeros((ka, ka)), Hab], [Hba, np.zeros((kb, kb))]])
    if tree.L == 0:
        f.D[1] = H.copy()
    return f


def _blkdiag(A, B):
    out = np.zeros((A.shape[0] + B.shape[0], A.shape[1] + B.shape[1]))
    out[:A.shape[0], :A.shape[1]] = A
    out[A.shape[0]:, A.shape[1]:] = B
    return out


def matvec(f: HBS, x):
    """y = H x through the telescoping factorisation (eq. tele1-tele3); x is M x B."""
    t = f.tree
    x = np.asarray(x, dtype=np.float64).reshape(t.M, -1)
    if t.L == 0:
        return f.D[1] @ x
    xh, yh = {}, {}
    for l in range(t.L, 0, -1):  # up: x^_tau = V_tau* (x on I_tau, or the children's x^)
        for tau in t.level(l):
            src = x[t.idx(tau)] if t.is_leaf(tau) else np.vstack([xh[2 * tau], xh[2 * tau + 1]])
            xh[tau] = f.V[tau].T @ src
    for l in range(0, t.L):  # down: children's y^ = U_tau y^_tau + B_tau [x^_a; x^_b]
        for tau in t.level(l):
            a, b = 2 * tau, 2 * tau + 1
            z = f.B[tau] @ np.vstack([xh[a], xh[b]])
            if l > 0:
                z = z + f.U[tau] @ yh[tau]
            ka = f.rank(a)
            yh[a], yh[b] = z[:ka], z[ka:]
    y = np.zeros_like(x)
    for tau in t.level(t.L):
        I = t.idx(tau)
        y[I] = f.U[tau] @ yh[tau] + f.D[tau] @ x[I]
    return y


class HBSInverse:
    def __init__(self, tree):
        self.tree = tree
        self.E, self.F, self.G, self.Dhat = {}, {}, {}, {}


def invert(f: HBS) -> HBSInverse:
    """Algorithm 1: factors {E_tau, F_tau, G_tau} representing H^{-1}."""
    t = f.tree
    inv = HBSInverse(t)
    if t.L == 0:
        inv.G[1] = np.linalg.inv(f.D[1])
        return inv
    for l in range(t.L, 0, -1):
        for tau in t.level(l):
            if t.is_leaf(tau):
                Dt = f.D[tau]
            else:
                a, b = 2 * tau, 2 * tau + 1
                ka = f.rank(a)
                Bt = f.B[tau]
                Dt = np.block([[inv.Dhat[a], Bt[:ka, ka:]], [Bt[ka:, :ka], inv.Dhat[b]]])
            Dti = np.linalg.inv(Dt)
            U, V = f.U[tau], f.V[tau]
            Dhat = np.linalg.inv(V.T @ Dti @ U)
            inv.Dhat[tau] = Dhat
            inv.E[tau] = Dti @ U @ Dhat
            inv.F[tau] = (Dhat @ V.T @ Dti).T
            inv.G[tau] = Dti - Dti @ U @ Dhat @ V.T @ Dti
    k2 = f.rank(2)
    B1 = f.B[1]
    inv.G[1] = np.linalg.inv(np.block([[inv.Dhat[2], B1[:k2, k2:]], [B1[k2:, :k2], inv.Dhat[3]]]))
    return inv


def apply_inverse(inv: HBSInverse, x):
    """Algorithm 2: y = H^{-1} x; x is M x B."""
    t = inv.tree
    x = np.asarray(x, dtype=np.float64).reshape(t.M, -1)
    if t.L == 0:
        return inv.G[1] @ x
    xh, yh = {}, {}
    for tau in t.level(t.L):
        xh[tau] = inv.F[tau].T @ x[t.idx(tau)]
    for l in range(t.L - 1, 0, -1):
        for tau in t.level(l):
            xh[tau] = inv.F[tau].T @ np.vstack([xh[2 * tau], xh[2 * tau + 1]])
    k2 = inv.E[2].shape[1] if 2 in inv.E else 0
    z = inv.G[1] @ np.vstack([xh[2], xh[3]])
    yh[2], yh[3] = z[:xh[2].shape[0]], z[xh[2].shape[0]:]
    for l in range(1, t.L):
        for tau in t.level(l):
            a, b = 2 * tau, 2 * tau + 1
            z = inv.E[tau] @ yh[tau] + inv.G[tau] @ np.vstack([xh[a], xh[b]])
            na = xh[a].shape[0]
            yh[a], yh[b] = z[:na], z[na:]
    y = np.zeros_like(x)
    for tau in t.level(t.L):
        I = t.idx(tau)
        y[I] = inv.E[tau] @ yh[tau] + inv.G[tau] @ x[I]
    return y


def to_dense(f: HBS):
    """The matrix an HBS representation stands for (telescoping applied to I)."""
    return matvec(f, np.eye(f.tree.M))


def dtn_apply(prob, S_root, tol, m, G):
    """Solve stage with an HBS root (Section 5 applied to Section 3.3 step 4):
    Neumann data (g - P S_root^{-1} B g)/h, S_root^{-1} by Algorithms 1 and 2."""
    from oracle.nd_dense import Box, ghost_map
    n, h = prob.n, prob.h
    rp = Box(0, 0, n, n).ring()
    where = {q: k for k, q in enumerate(rp)}
    Bm = np.zeros((len(rp), 4 * n))
    Pm = np.zeros((4 * n, len(rp)))
    for k, (q, wgt) in enumerate(ghost_map(prob)):
        Bm[where[q], k] = -wgt
        Pm[k, where[q]] = 1.0
    tree = HBSTree(len(rp), m)
    inv = invert(compress(S_root, tree, tol))
    G = np.asarray(G, dtype=np.float64).reshape(4 * n, -1)
    return (G - Pm @ apply_inverse(inv, Bm @ G)) / h


def step1_interface_solver(tol: float, m: int):
    """The accelerated merge's Step 1 (Section 5, "Accelerating the nested dissection
    algorithm"): [S33 A34; A43 S44]^{-1} Z by block elimination, S33 and the Schur
    complement S44 - A43 S33^{-1} A34 each compressed at tol and inverted by Algorithms
    1 and 2:
        X4 = (S44 - A43 S33^{-1} A34)^{-1} (Z4 - A43 S33^{-1} Z3),
        X3 = S33^{-1} Z3 - S33^{-1} A34 X4.
    The Schur complement is formed densely and recompressed (the paper's fast HBS
    addition is deferred to a reference; dense recompression is the reading here)."""

    def inv_apply(A):
        t = HBSTree(A.shape[0], m)
        if t.L == 0:
            return lambda X: np.linalg.solve(A, X)
        inv = invert(compress(A, t, tol))
        return lambda X: apply_inverse(inv, X)

    def solve(S33, A34, A43, S44, Z):
        s3 = S33.shape[0]
        Z3, Z4 = Z[:s3], Z[s3:]
        i33 = inv_apply(S33)
        W3 = i33(Z3)
        V3 = i33(A34)
        i44 = inv_apply(S44 - A43 @ V3)
        X4 = i44(Z4 - A43 @ W3)
        X3 = W3 - V3 @ X4
        return np.vstack([X3, X4])

    return solve


def low_rank(A, tol):
    """A ~ L R from a column-pivoted QR of A truncated at the first |R_jj| <= tol |R_11|
    (the local-tolerance reading of the compression): L = Q_k orthonormal, R = L^T A."""
    Q, k = _pivoted_qr(A, tol)
    L = Q[:, :k]
    return L, L.T @ A


def accelerated_merge(prob, box1, S1, box2, S2, parent, tol, m):
    """The accelerated merge of two siblings (Section 5, Steps 1-3), from their dense
    Schur complements S1, S2 (eq. partition_we for P1..P4):
      Step 1  X = [S33 A34; A43 S44]^{-1} [S31 A32; A41 S42] by the block solve with HBS
              inverses (step1_interface_solver);
      Step 2  S13 = L13 R13 and S24 = L24 R24 truncated at tol, and the update in factored
              form (A14 = A23 = 0 for the five-point stencil):
                  [L13 (R13 X31)  L13 (R13 X32); L24 (R24 X41)  L24 (R24 X42)];
      Step 3  S = [S11 A12; A21 S22] minus that update, placed in the parent's ring order
              and compressed to HBS form at tol.  The paper's HBS + low-rank addition and
              recompression algorithms are not in its text: the sum is formed and
              recompressed densely here (the reading).
    Returns (S dense, its HBS form, (rank of L13, rank of L24))."""
    from oracle.nd_dense import partition_we
    i1, i3, i2, i4, P1, P3, P2, P4 = partition_we(box1, box2, parent)
    A = prob.A_block
    S11, S13, S31, S33 = (S1[np.ix_(r, c)] for r, c in ((i1, i1), (i1, i3), (i3, i1), (i3, i3)))
    S22, S24, S42, S44 = (S2[np.ix_(r, c)] for r, c in ((i2, i2), (i2, i4), (i4, i2), (i4, i4)))
    A12, A21, A32, A41 = A(P1, P2), A(P2, P1), A(P3, P2), A(P4, P1)
    A34, A43 = A(P3, P4), A(P4, P3)
    n1, s3 = len(P1), len(P3)
    # Step 1
    Z = np.block([[S31, A32], [A41, S42]])
    X = step1_interface_solver(tol, m)(S33, A34, A43, S44, Z) if s3 else np.zeros((0, Z.shape[1]))
    X31, X32 = X[:s3, :n1], X[:s3, n1:]
    X41, X42 = X[s3:, :n1], X[s3:, n1:]
    # Step 2
    L13, R13 = low_rank(S13, tol)
    L24, R24 = low_rank(S24, tol)
    upd = np.block([[L13 @ (R13 @ X31), L13 @ (R13 @ X32)], [L24 @ (R24 @ X41), L24 @ (R24 @ X42)]])
    # Step 3
    S = np.block([[S11, A12], [A21, S22]]) - upd
    rp = parent.ring()
    where = {q: k for k, q in enumerate(rp)}
    perm = np.array([where[q] for q in P1 + P2])
    out = np.empty_like(S)
    out[np.ix_(perm, perm)] = S
    return out, compress(out, HBSTree(out.shape[0], m), tol), (L13.shape[1], L24.shape[1])
