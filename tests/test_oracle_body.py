"""Pins of the oracle's body-load operator (Section 6.3: v = T g + F f_hat) and of its
conductance-network problems (Section 6.1, Random Laplacian I and II).

Each is checked against something other than the oracle itself:
  * a manufactured solution: for a quadratic u the five-point scheme is exact, so the
    load it needs at every node and its Neumann data are closed forms in x, y, b, c, d;
  * the sine-transform solve for constant coefficients (unit loads, zero data);
  * a network whose vertical links are cut: every grid row is a chain of resistors in
    series, so its Dirichlet-to-Neumann map and its response to a load follow from
    the series and current-divider rules;
  * conservation and the maximum principle for divergence-form problems (Laplace and
    any network): F's columns sum to -h and F lies in [-h, 0]; T is symmetric, positive
    semi-definite, with T 1 = 0;
  * unit conductivities give the Laplace operator;
  * O2 (the tree with a load map per box) against O1 (one full solve per load), on
    ragged trees with loads on leaf rings, merge interfaces and the outer ring;
  * planted mistakes in the load-map steps are caught.
"""
import numpy as np
import pytest

from oracle import closed_form as cf
from oracle import nd_dense, o1
from paper_1302_5995_gb300 import inputs


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def quadratic(x, y):
    return x * x + x * y - 2.0 * y * y + 0.3 * x - 0.7 * y + 0.1


def quadratic_load(x, y, b, c, d):
    """-Lap u + (1/h) b (u_e - u_w) + (1/h) c (u_n - u_s) + d u for the quadratic above:
    centred differences are exact for quadratics, and the literal 1/h convection scaling
    doubles the derivative (u_e - u_w = 2 h u_x)."""
    ux = 2.0 * x + y + 0.3
    uy = x - 4.0 * y - 0.7
    return 2.0 + 2.0 * b * ux + 2.0 * c * uy + d * quadratic(x, y)


def quadratic_data(n):
    """(g, v): the quadratic on the ghosts and its exact one-sided flux."""
    h = 1.0 / (n + 1)
    xs, ys = inputs.ghost_xy(n)
    xn, yn = np.clip(xs, h, n * h), np.clip(ys, h, n * h)  # each ghost's unknown neighbour
    g = quadratic(xs, ys)
    return g, (g - quadratic(xn, yn)) / h


# --------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n,leaf", [(11, 3), (14, 4)])
def test_manufactured_quadratic_with_loads_everywhere(n, leaf):
    b, c, d = inputs.convection_fields(n, seeds=(41, 42, 43))
    X, Y = inputs.node_xy(n)
    f = quadratic_load(X, Y, b, c, d)
    g, v = quadratic_data(n)
    every = np.arange(n * n)
    assert rel(o1.apply_loads(b, c, d, n, g[:, None], every, f[:, None])[:, 0], v) < 1e-12
    T, F = nd_dense.build_loads(nd_dense.Problem(b, c, d, n), leaf, every)
    assert rel(T @ g + F @ f, v) < 1e-11


def test_sine_transform_load_operator():
    n, b0, c0, d0 = 13, 1.5, -2.5, 3.0
    b, c, d = inputs.constant_fields(n, b0, c0, d0)
    idx = np.array([0, n - 1, n * n - 1, 5 + n * 6, 6 + n * 6, 3 + n * 9])
    F_cf = cf.dst_load_matrix(n, b0, c0, d0, idx)
    assert rel(o1.load_matrix(b, c, d, n, idx), F_cf) < 1e-12
    _, F = nd_dense.build_loads(nd_dense.Problem(b, c, d, n), 4, idx)
    assert rel(F, F_cf) < 1e-12


def _series_network(n, seed):
    sx, _ = inputs.network_conductivities(n, 1.0, 2.0, seed)
    return sx, np.zeros(n * (n + 1))  # every vertical link cut


def test_series_chains_dtn_closed_form():
    n, h = 10, 1.0 / 11
    sx, sy = _series_network(n, 51)
    SX = sx.reshape(n, n + 1)
    T_cf = np.zeros((4 * n, 4 * n))
    for j in range(n):
        R = np.sum(1.0 / SX[j])  # resistors in series
        kw, ke = 3 * n + (n - 1 - j), n + j
        T_cf[np.ix_([kw, ke], [kw, ke])] = np.array([[1.0, -1.0], [-1.0, 1.0]]) / (R * h)
    assert rel(o1.net_dtn_matrix(sx, sy, n), T_cf) < 1e-12
    T, _ = nd_dense.build_loads(nd_dense.Problem.network(sx, sy, n), 3, [])
    assert rel(T, T_cf) < 1e-12


def test_series_chains_load_closed_form():
    n, h = 10, 1.0 / 11
    sx, sy = _series_network(n, 52)
    SX = sx.reshape(n, n + 1)
    idx = np.array([0, 9, 4 + 3 * n, 5 + 3 * n, 7 + 8 * n, 2 + 9 * n])
    F_cf = np.zeros((4 * n, idx.size))
    for m, k in enumerate(idx):
        i, j = int(k) % n, int(k) // n
        RW, RE = np.sum(1.0 / SX[j, : i + 1]), np.sum(1.0 / SX[j, i + 1:])
        # the injected current h^2 f splits between the two ends like a current divider
        F_cf[3 * n + (n - 1 - j), m] = -h * RE / (RW + RE)
        F_cf[n + j, m] = -h * RW / (RW + RE)
    assert rel(o1.net_load_matrix(sx, sy, n, idx), F_cf) < 1e-12
    _, F = nd_dense.build_loads(nd_dense.Problem.network(sx, sy, n), 3, idx)
    assert rel(F, F_cf) < 1e-12


@pytest.mark.parametrize("which", ["laplace", "random1", "random2"])
def test_conservation_and_maximum_principle(which):
    n, leaf = 17, 5
    h = 1.0 / (n + 1)
    if which == "laplace":
        prob = nd_dense.Problem(*inputs.laplace_fields(n), n)
    else:
        sx, sy = (inputs.random_laplacian_1 if which == "random1" else inputs.random_laplacian_2)(n)
        prob = nd_dense.Problem.network(sx, sy, n)
    idx = inputs.body_nodes(n, 25, 7)
    T, F = nd_dense.build_loads(prob, leaf, idx)
    scale = np.abs(T).max()
    assert np.abs(T - T.T).max() < 1e-12 * scale  # reciprocity
    assert np.abs(T.sum(axis=1)).max() < 1e-12 * scale  # constants carry no current
    assert np.linalg.eigvalsh(0.5 * (T + T.T)).min() > -1e-12 * scale
    np.testing.assert_allclose(F.sum(axis=0), -h, rtol=1e-12)  # every load leaves by the boundary
    assert F.max() <= 1e-15 and F.min() >= -h * (1 + 1e-12)


def test_unit_network_is_laplace_and_scales():
    n, leaf = 12, 4
    idx = inputs.body_nodes(n, 9, 3)
    ones = np.ones(n * (n + 1))
    T_lap, F_lap = nd_dense.build_loads(nd_dense.Problem(*inputs.laplace_fields(n), n), leaf, idx)
    T_net, F_net = nd_dense.build_loads(nd_dense.Problem.network(ones, ones, n), leaf, idx)
    assert rel(T_net, T_lap) < 1e-13 and rel(F_net, F_lap) < 1e-13
    assert rel(o1.net_dtn_matrix(ones, ones, n), o1.dtn_matrix(*inputs.laplace_fields(n), n)) < 1e-13
    # conductivities s: the currents scale by s, the load response does not
    T_s, F_s = nd_dense.build_loads(nd_dense.Problem.network(7 * ones, 7 * ones, n), leaf, idx)
    assert rel(T_s, 7 * T_lap) < 1e-13 and rel(F_s, F_lap) < 1e-13


# --------------------------------------------------------------------------- O2 against O1

def _placed_loads(n):
    """Loads on the outer ring (a corner, two edges), on both sides of the root's two
    merge interfaces, plus a localized random set (flat indices, distinct)."""
    half = n // 2
    fixed = [(0, 0), (5, 0), (n - 1, half - 1), (7, half - 1), (8, half), (half - 1, 4),
             (half, 5), (3, n - 1)]
    idx = [i + n * j for (i, j) in fixed]
    idx += [int(k) for k in inputs.body_nodes(n, 20, 13) if int(k) not in idx]
    return np.array(idx)


@pytest.mark.parametrize("n,leaf", [(23, 4), (30, 5)])
def test_o2_loads_match_o1_convection(n, leaf):
    b, c, d = inputs.convection_fields(n, seeds=(61, 62, 63))
    idx = _placed_loads(n)
    T, F = nd_dense.build_loads(nd_dense.Problem(b, c, d, n), leaf, idx)
    assert rel(F, o1.load_matrix(b, c, d, n, idx)) < 1e-11
    assert rel(T, nd_dense.build(b, c, d, n, leaf).T) < 1e-13  # loads leave T alone


@pytest.mark.parametrize("make", [inputs.random_laplacian_1, inputs.random_laplacian_2])
def test_o2_loads_match_o1_network(make):
    n, leaf = 26, 4
    sx, sy = make(n)
    idx = _placed_loads(n)
    T, F = nd_dense.build_loads(nd_dense.Problem.network(sx, sy, n), leaf, idx)
    assert rel(F, o1.net_load_matrix(sx, sy, n, idx)) < 1e-11
    assert rel(T, o1.net_dtn_matrix(sx, sy, n)) < 1e-11
    # the two terms together, for Gaussian data and loads
    G = inputs.gaussian_vectors(n, 3, 71)
    Fl = inputs.body_load_vectors(idx.size, 3, 72)
    assert rel(T @ G + F @ Fl, o1.net_apply(sx, sy, n, G, idx, Fl)) < 1e-11


def test_body_nodes_are_distinct_localized_and_seeded():
    n = 64
    for count in (1, 10, 100, 1000):
        idx = inputs.body_nodes(n, count, 5)
        assert idx.size == count and len(set(idx.tolist())) == count
        i, j = idx % n, idx // n
        w = min(n, max(4, int(np.ceil(2 * np.sqrt(count)))))
        assert i.max() - i.min() < w and j.max() - j.min() < w
        assert np.array_equal(idx, inputs.body_nodes(n, count, 5))
    with pytest.raises(ValueError):
        inputs.body_nodes(4, 17, 0)


# --------------------------------------------------------------------------- planted mistakes

@pytest.mark.parametrize("mistake", ["drop_correction", "leaf_without_ring_rows", "child_columns_swapped"])
def test_planted_load_mistakes_are_caught(monkeypatch, mistake):
    orig_merge, orig_leaf = nd_dense.merge_loads, nd_dense.leaf_load_map

    def bad_merge(prob, box1, S1, L1, box2, S2, L2, parent):
        if mistake == "drop_correction":
            # identities for S1, S2 make S13 = S24 = 0 (and A14 = A23 = 0 already), so the
            # correction term vanishes: only the gathered P1/P2 rows remain
            return orig_merge(prob, box1, np.eye(len(S1)), L1, box2, np.eye(len(S2)), L2, parent)
        if mistake == "child_columns_swapped":
            out = orig_merge(prob, box1, S1, L1, box2, S2, L2, parent)
            return np.hstack([out[:, L1.shape[1]:], out[:, :L1.shape[1]]])
        return orig_merge(prob, box1, S1, L1, box2, S2, L2, parent)

    def bad_leaf(prob, box, body):
        Lm, cols = orig_leaf(prob, box, body)
        if mistake == "leaf_without_ring_rows":
            ring = box.ring()
            for cidx, q in enumerate(cols):
                if q in ring:
                    Lm[ring.index(q), cidx] -= 1.0  # forgets f_b, keeps only -A_bi A_ii^-1 f_i
        return Lm, cols

    monkeypatch.setattr(nd_dense, "merge_loads", bad_merge)
    monkeypatch.setattr(nd_dense, "leaf_load_map", bad_leaf)
    n, leaf = 23, 4
    b, c, d = inputs.convection_fields(n, seeds=(81, 82, 83))
    idx = _placed_loads(n)
    _, F = nd_dense.build_loads(nd_dense.Problem(b, c, d, n), leaf, idx)
    assert rel(F, o1.load_matrix(b, c, d, n, idx)) > 1e-4
