"""Oracle O2 -- the paper's dense nested-dissection build and solve, step by step.

TEST INFRASTRUCTURE ONLY: the library never imports this module.  The tests, the
smoke check and the benchmark's CPU-baseline leg are its only users.

Follows, in the paper's order and notation:
  Section 2        quad-tree of boxes; L = smallest level count whose boxes have
                   edge <= leaf; levels 0 (root) .. L (leaves)
  Section 3.1      leaf Schur complement S = A_bb - A_bi A_ii^{-1} A_ib   (eq. def_schur_nd)
  Section 3.2      merge of two siblings, P^(w) = P1 u P3, P^(e) = P2 u P4 (eq. partition_we),
                   S = [S11 A12; A21 S22] - [S13 A14; A23 S24] [S33 A34; A43 S44]^{-1}
                       [S31 A32; A41 S42]                                  (eq. S_fromtwo_nd)
  Section 3.3      four-child merge as three pairwise merges; level-by-level sweep
  Section 3.3 (4)  root: invert the root Schur complement to get the solution operator
  Section 6        five-point stencil with (1/h) convection terms
  Section 6.1      Random Laplacian problems: a conductance network on the same grid
  Section 6.3      body loads at listed nodes: every box carries a load map beside S
                   (leaf: f_b - A_bi A_ii^{-1} f_i; merge: the updated right-hand side of
                   Section 3.2), and the root gives the second operator F of v = T g + F f

Readings where the paper is silent (each one is listed with its reason in the design
notes of the repository):
  * n x n UNKNOWN nodes, h = 1/(n+1); the 4n non-corner ghost nodes carry g.
  * a box's "ring" P_b is its outermost layer of unknowns, ordered counter-clockwise
    from its south-west corner; a tree split gives the west/south child floor(a/2).
  * four-child merge order: (SW + SE), (NW + NE), then (S-half + N-half).
  * a network's equation is (1/h^2) sum over links of sigma (u_k - u_l) = f_k and its
    datum at ghost k the link current sigma_k (g_k - u_{k'})/h (unit conductivities
    give Laplace); a body load f_k enters the equation at its node as written.
  * the Neumann datum at ghost k is the outward one-sided flux (g_k - u_{k'})/h,
    k' the only unknown next to k; hence T = (I - P S_root^{-1} B)/h, where B holds
    every ring node's stencil weight on its ghosts (negated, moved to the right-hand
    side) and P picks each ghost's ring neighbour.

Precision: FP64 throughout.  The dense solves call LAPACK through numpy, a library
primitive used as one step; nothing is blocked, fused or reordered beyond the
paper's formulas.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EAST, WEST, NORTH, SOUTH = 1, 2, 3, 4
_STEP = {EAST: (1, 0), WEST: (-1, 0), NORTH: (0, 1), SOUTH: (0, -1)}


class Problem:
    """Five-point stencil of Section 6 on an n x n grid of unknowns."""

    def __init__(self, b, c, d, n):
        self.n = n
        self.h = 1.0 / (n + 1)
        h = self.h
        B = np.asarray(b, dtype=np.float64).reshape(n, n)  # [j, i]
        C = np.asarray(c, dtype=np.float64).reshape(n, n)
        D = np.asarray(d, dtype=np.float64).reshape(n, n)
        # weight of the equation at (i, j) on itself and on each neighbour
        self.w = {
            0: 4.0 / h**2 + D,
            EAST: -1.0 / h**2 + B / h,
            WEST: -1.0 / h**2 - B / h,
            NORTH: -1.0 / h**2 + C / h,
            SOUTH: -1.0 / h**2 - C / h,
        }

    @classmethod
    def network(cls, sx, sy, n):
        """Random Laplacian problems (Section 6.1): a square-grid network whose links carry
        conductivities; the equation at node k is (1/h^2) sum_l sigma_l (u_k - u_l) = f_k
        (scaled like the five-point Laplacian, so unit conductivities give Laplace).
        sx: n rows of n + 1 x-links, [j, i] joins (i-1, j) and (i, j); sy: n + 1 rows of n
        y-links, [j, i] joins (i, j-1) and (i, j); the outermost links reach the ghosts."""
        self = cls.__new__(cls)
        self.n = n
        self.h = 1.0 / (n + 1)
        ih2 = 1.0 / self.h**2
        SX = np.asarray(sx, dtype=np.float64).reshape(n, n + 1)
        SY = np.asarray(sy, dtype=np.float64).reshape(n + 1, n)
        east, west, north, south = SX[:, 1:], SX[:, :-1], SY[1:, :], SY[:-1, :]
        self.w = {
            0: (east + west + north + south) * ih2,
            EAST: -east * ih2,
            WEST: -west * ih2,
            NORTH: -north * ih2,
            SOUTH: -south * ih2,
        }
        t = np.arange(n)
        # conductivity of each ghost's link, in ghost order (south, east, north, west)
        self.ghost_sigma = np.concatenate([SY[0, t], SX[t, n], SY[n, n - 1 - t], SX[n - 1 - t, 0]])
        return self

    def datum_weights(self):
        """Weight of each ghost's datum: 1 for the PDE flux (g_k - u_k')/h, the link's
        conductivity for a network (the current through the link, over h)."""
        sig = getattr(self, "ghost_sigma", None)
        return np.ones(4 * self.n) if sig is None else sig

    def A_block(self, rows, cols):
        """Dense sub-matrix A(rows, cols) of the global stencil matrix.

        rows, cols: sequences of (i, j) unknown nodes."""
        pos = {tuple(q): k for k, q in enumerate(cols)}
        out = np.zeros((len(rows), len(cols)))
        for r, (i, j) in enumerate(rows):
            k = pos.get((i, j))
            if k is not None:
                out[r, k] = self.w[0][j, i]
            for dirn, (di, dj) in _STEP.items():
                k = pos.get((i + di, j + dj))
                if k is not None:
                    out[r, k] = self.w[dirn][j, i]
        return out


@dataclass(frozen=True)
class Box:
    """Rectangle of unknowns [x0, x0+a) x [y0, y0+b)."""
    x0: int
    y0: int
    a: int
    b: int

    def nodes(self):
        return [(self.x0 + i, self.y0 + j) for j in range(self.b) for i in range(self.a)]

    def ring(self):
        """Outermost layer P_b, counter-clockwise from the south-west corner."""
        a, b, x0, y0 = self.a, self.b, self.x0, self.y0
        if a == 1 or b == 1:
            raise ValueError("boxes must be at least 2 x 2")
        out = [(x0 + i, y0) for i in range(a)]
        out += [(x0 + a - 1, y0 + j) for j in range(1, b)]
        out += [(x0 + i, y0 + b - 1) for i in range(a - 2, -1, -1)]
        out += [(x0, y0 + j) for j in range(b - 2, 0, -1)]
        return out

    def contains(self, q):
        return self.x0 <= q[0] < self.x0 + self.a and self.y0 <= q[1] < self.y0 + self.b

    def interior(self):
        ring = set(self.ring())
        return [q for q in self.nodes() if q not in ring]

    def children(self):
        """SW, SE, NW, NE; the west and south halves take the floor."""
        a0, b0 = self.a // 2, self.b // 2
        return (Box(self.x0, self.y0, a0, b0),
                Box(self.x0 + a0, self.y0, self.a - a0, b0),
                Box(self.x0, self.y0 + b0, a0, self.b - b0),
                Box(self.x0 + a0, self.y0 + b0, self.a - a0, self.b - b0))


def num_levels(n, leaf):
    """Section 2: the smallest L whose 4^L boxes have edge ceil(n / 2^L) <= leaf."""
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    return L


def quad_tree(n, leaf):
    """levels[l] lists the boxes of level l (0 = root, L = leaves), children in
    SW, SE, NW, NE order under each parent."""
    L = num_levels(n, leaf)
    levels = [[Box(0, 0, n, n)]]
    for _ in range(L):
        levels.append([c for p in levels[-1] for c in p.children()])
    return levels


def leaf_schur(prob: Problem, box: Box):
    """Eq. def_schur_nd: S = A_bb - A_bi A_ii^{-1} A_ib on the box's ring."""
    Pb, Pi = box.ring(), box.interior()
    A_bb = prob.A_block(Pb, Pb)
    if not Pi:
        return A_bb
    A_bi = prob.A_block(Pb, Pi)
    A_ii = prob.A_block(Pi, Pi)
    A_ib = prob.A_block(Pi, Pb)
    return A_bb - A_bi @ np.linalg.solve(A_ii, A_ib)


def partition_we(box1: Box, box2: Box, parent: Box):
    """Eq. partition_we: positions (in each child's ring) of P1, P3 (child 1) and P2, P4
    (child 2) -- the nodes that stay on the parent's ring and the ones that become
    interior -- and the node lists themselves."""
    r1, r2 = box1.ring(), box2.ring()
    on_parent = set(parent.ring())
    i1 = [k for k, q in enumerate(r1) if q in on_parent]
    i3 = [k for k, q in enumerate(r1) if q not in on_parent]
    i2 = [k for k, q in enumerate(r2) if q in on_parent]
    i4 = [k for k, q in enumerate(r2) if q not in on_parent]
    return (i1, i3, i2, i4, [r1[k] for k in i1], [r1[k] for k in i3],
            [r2[k] for k in i2], [r2[k] for k in i4])


def merge_two(prob: Problem, box1: Box, S1, box2: Box, S2, parent: Box, interface_solve=None):
    """Eq. S_fromtwo_nd for two sibling rectangles whose union is `parent`.

    box1 is the west (or south) sibling and box2 the east (or north) one.  P1/P2 are
    the nodes of each child's ring that lie on the parent's ring, P3/P4 the ones that
    become interior (eq. partition_we).  Returns the parent's S in its ring order.
    interface_solve(S33, A34, A43, S44, Z) -> [S33 A34; A43 S44]^{-1} Z replaces the
    dense solve when given (the HBS Step 1 of the accelerated method).
    """
    rp = parent.ring()
    i1, i3, i2, i4, P1, P3, P2, P4 = partition_we(box1, box2, parent)

    S11, S13 = S1[np.ix_(i1, i1)], S1[np.ix_(i1, i3)]
    S31, S33 = S1[np.ix_(i3, i1)], S1[np.ix_(i3, i3)]
    S22, S24 = S2[np.ix_(i2, i2)], S2[np.ix_(i2, i4)]
    S42, S44 = S2[np.ix_(i4, i2)], S2[np.ix_(i4, i4)]
    A = prob.A_block
    A12, A14 = A(P1, P2), A(P1, P4)
    A21, A23 = A(P2, P1), A(P2, P3)
    A32, A34 = A(P3, P2), A(P3, P4)
    A41, A43 = A(P4, P1), A(P4, P3)

    outer = np.block([[S11, A12], [A21, S22]])
    left = np.block([[S13, A14], [A23, S24]])
    mid = np.block([[S33, A34], [A43, S44]])
    right = np.block([[S31, A32], [A41, S42]])
    if mid.shape[0] and interface_solve is not None:
        S = outer - left @ interface_solve(S33, A34, A43, S44, right)
    elif mid.shape[0]:
        S = outer - left @ np.linalg.solve(mid, right)
    else:
        S = outer
    # rows/columns of S follow [P1; P2]; place them in the parent's ring order
    where = {q: k for k, q in enumerate(rp)}
    perm = np.array([where[q] for q in P1 + P2])
    out = np.empty_like(S)
    out[np.ix_(perm, perm)] = S
    return out


def merge_four(prob: Problem, parent: Box, S_children, interface_solve=None, min_edge=None):
    """Section 3.3 step 3: a four-child merge as three pairwise merges.  With
    interface_solve, merges whose shared edge has >= min_edge nodes use it."""
    sw, se, nw, ne = parent.children()
    S_sw, S_se, S_nw, S_ne = S_children
    south = Box(parent.x0, parent.y0, parent.a, sw.b)
    north = Box(parent.x0, parent.y0 + sw.b, parent.a, nw.b)

    def pick(edge):
        return interface_solve if interface_solve is not None and edge >= min_edge else None

    S_south = merge_two(prob, sw, S_sw, se, S_se, south, pick(sw.b))
    S_north = merge_two(prob, nw, S_nw, ne, S_ne, north, pick(nw.b))
    S = merge_two(prob, south, S_south, north, S_north, parent, pick(parent.a))
    return S, (south, S_south, north, S_north)


def ghost_map(prob: Problem):
    """For ghost k: its ring neighbour (i, j) and that node's stencil weight on k."""
    n = prob.n
    out = []
    for k in range(4 * n):
        side, t = divmod(k, n)
        if side == 0:
            q, dirn = (t, 0), SOUTH
        elif side == 1:
            q, dirn = (n - 1, t), EAST
        elif side == 2:
            q, dirn = (n - 1 - t, n - 1), NORTH
        else:
            q, dirn = (0, n - 1 - t), WEST
        out.append((q, prob.w[dirn][q[1], q[0]]))
    return out


def root_dtn(prob: Problem, S_root):
    """Section 3.3 step 4 with the flux reading: T = (I - P S_root^{-1} B)/h."""
    n, h = prob.n, prob.h
    rp = Box(0, 0, n, n).ring()
    where = {q: k for k, q in enumerate(rp)}
    Bm = np.zeros((len(rp), 4 * n))
    Pm = np.zeros((4 * n, len(rp)))
    for k, (q, wgt) in enumerate(ghost_map(prob)):
        Bm[where[q], k] = -wgt
        Pm[k, where[q]] = 1.0
    return prob.datum_weights()[:, None] * (np.eye(4 * n) - Pm @ np.linalg.solve(S_root, Bm)) / h


@dataclass
class BuildResult:
    T: np.ndarray
    L: int
    schur: dict  # Box -> S on its ring (leaves, half-boxes and boxes), if kept
    flops: float
    S_root: np.ndarray = None  # the root Schur complement (ring of the whole grid)


def build(b, c, d, n, leaf, keep=False, interface_solve=None, min_edge=None):
    """Full dense build (Section 3.3 steps 1-4).  Returns the 4n x 4n DtN matrix T.
    interface_solve / min_edge: the merges whose shared edge has >= min_edge nodes solve
    their interface system with interface_solve (see merge_two)."""
    prob = Problem(b, c, d, n)
    levels = quad_tree(n, leaf)
    L = len(levels) - 1
    flops = 0.0
    S = {}
    for box in levels[L]:
        S[box] = leaf_schur(prob, box)
        # nominal banded cost (Section 3.4): A_ii has bandwidth a-2
        ni = max(box.a - 2, 0) * max(box.b - 2, 0)
        bw = max(box.a - 2, 0)
        flops += 2.0 * ni * bw * bw + 4.0 * ni * bw * len(box.ring())
    kept = dict(S) if keep else {}
    for lev in range(L, 0, -1):
        nxt = {}
        for parent in levels[lev - 1]:
            kids = parent.children()
            Sp, halves = merge_four(prob, parent, [S[k] for k in kids], interface_solve, min_edge)
            nxt[parent] = Sp
            if keep:
                kept[halves[0]] = halves[1]
                kept[halves[2]] = halves[3]
                kept[parent] = Sp
            for (m_s, p_s) in _merge_shapes(parent, kids):
                flops += (16.0 / 3.0) * m_s**3 + 8.0 * m_s**2 * p_s + 2.0 * p_s**2 * m_s
        S = nxt
    root = levels[0][0]
    r = len(root.ring())
    flops += (2.0 / 3.0) * r**3 + 2.0 * r**2 * 4 * n
    T = root_dtn(prob, S[root])
    return BuildResult(T=T, L=L, schur=kept, flops=flops, S_root=S[root])


def _merge_shapes(parent, kids):
    """(s', p) of the three pairwise merges of a four-child merge (for flop counting)."""
    sw, se, nw, ne = kids
    shapes = []
    for (b1, b2) in ((sw, se), (nw, ne)):
        shapes.append((max(b1.b - 2, 0), 2 * (b1.a + b2.a) + 2 * b1.b - 4))
    shapes.append((max(parent.a - 2, 0), len(parent.ring())))
    return shapes


def solve(T, G):
    """Solve stage (Section 1.1): Neumann data V = T G for Dirichlet vectors G (4n x B)."""
    return T @ G


def direct_schur(prob: Problem, box: Box):
    """Plain definition of a box's Schur complement (eq. def_schur_nd applied to the
    whole box at once, no tree) -- used to pin every intermediate of the merge."""
    return leaf_schur(prob, box)


# ----------------------------------------------------------------------------- body loads

def _inject(nodes, cols):
    """0/1 matrix placing load column c at the row of node cols[c] in `nodes`."""
    where = {q: k for k, q in enumerate(nodes)}
    E = np.zeros((len(nodes), len(cols)))
    for c, q in enumerate(cols):
        if q in where:
            E[where[q], c] = 1.0
    return E


def leaf_load_map(prob: Problem, box: Box, body):
    """Section 3.1 with a body load: eliminating u_i leaves S u_b = f_b - A_bi A_ii^{-1} f_i.
    Returns (Lmap, cols): cols are the body nodes inside the box (in the order of `body`),
    and Lmap (ring x len(cols)) takes their loads to that right-hand side."""
    cols = [q for q in body if box.contains(q)]
    Pb, Pi = box.ring(), box.interior()
    E_b = _inject(Pb, cols)
    if not Pi:
        return E_b, cols
    E_i = _inject(Pi, cols)
    return E_b - prob.A_block(Pb, Pi) @ np.linalg.solve(prob.A_block(Pi, Pi), E_i), cols


def merge_loads(prob: Problem, box1: Box, S1, L1, box2: Box, S2, L2, parent: Box):
    """Section 3.2, the updated right-hand side of a merge:
        [f1; f2] - [S13 A14; A23 S24] [S33 A34; A43 S44]^{-1} [f3; f4],
    as a map of the children's loads: f1..f4 are the rows P1..P4 of the children's load
    maps (child 1's columns first, then child 2's).  Rows in the parent's ring order."""
    rp = parent.ring()
    i1, i3, i2, i4, P1, P3, P2, P4 = partition_we(box1, box2, parent)
    m1, m2 = L1.shape[1], L2.shape[1]

    def two(L1rows, L2rows):
        return np.vstack([np.hstack([L1rows, np.zeros((L1rows.shape[0], m2))]),
                          np.hstack([np.zeros((L2rows.shape[0], m1)), L2rows])])

    f12 = two(L1[i1], L2[i2])
    f34 = two(L1[i3], L2[i4])
    if f34.shape[0]:
        A = prob.A_block
        left = np.block([[S1[np.ix_(i1, i3)], A(P1, P4)], [A(P2, P3), S2[np.ix_(i2, i4)]]])
        mid = np.block([[S1[np.ix_(i3, i3)], A(P3, P4)], [A(P4, P3), S2[np.ix_(i4, i4)]]])
        f12 = f12 - left @ np.linalg.solve(mid, f34)
    where = {q: k for k, q in enumerate(rp)}
    perm = np.array([where[q] for q in P1 + P2])
    out = np.empty_like(f12)
    out[perm] = f12
    return out


def root_load_operator(prob: Problem, S_root, L_root):
    """Section 6.3's second term: the root ring solves S_root u = B g + L_root f_hat, so the
    ghost data take F = -D P S_root^{-1} L_root / h (D the datum weights)."""
    n, h = prob.n, prob.h
    rp = Box(0, 0, n, n).ring()
    where = {q: k for k, q in enumerate(rp)}
    Pm = np.zeros((4 * n, len(rp)))
    for k, (q, _) in enumerate(ghost_map(prob)):
        Pm[k, where[q]] = 1.0
    return -prob.datum_weights()[:, None] * (Pm @ np.linalg.solve(S_root, L_root)) / h


def build_loads(prob: Problem, leaf, body):
    """Section 6.3: the two operators of v = T g + F f_hat for loads at the listed body
    nodes ((i, j) pairs or flat indices i + n j; F's columns follow that order).  The tree,
    leaf and merge steps are those of `build`; every box carries its load map beside S."""
    n = prob.n
    body = [tuple(divmod(int(k), n)[::-1]) if np.isscalar(k) else tuple(k) for k in body]
    if len(set(body)) != len(body):
        raise ValueError("body nodes must be distinct")
    levels = quad_tree(n, leaf)
    S, Lm, cols = {}, {}, {}
    for box in levels[-1]:
        S[box] = leaf_schur(prob, box)
        Lm[box], cols[box] = leaf_load_map(prob, box, body)
    for lev in range(len(levels) - 1, 0, -1):
        for parent in levels[lev - 1]:
            sw, se, nw, ne = parent.children()
            south = Box(parent.x0, parent.y0, parent.a, sw.b)
            north = Box(parent.x0, parent.y0 + sw.b, parent.a, nw.b)
            for (b1, b2, half) in ((sw, se, south), (nw, ne, north), (south, north, parent)):
                Lm[half] = merge_loads(prob, b1, S[b1], Lm[b1], b2, S[b2], Lm[b2], half)
                cols[half] = cols[b1] + cols[b2]
                S[half] = merge_two(prob, b1, S[b1], b2, S[b2], half)
    root = levels[0][0]
    T = root_dtn(prob, S[root])
    Fr = root_load_operator(prob, S[root], Lm[root])
    order = {q: c for c, q in enumerate(cols[root])}
    F = Fr[:, [order[q] for q in body]]
    return T, F
