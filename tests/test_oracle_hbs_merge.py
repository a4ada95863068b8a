"""The oracle's accelerated merge (Section 5, Steps 1-3: block solve with HBS inverses,
low-rank factors of S13 and S24, the parent recompressed to HBS form) against the dense
merge of eq. S_fromtwo_nd on the top merge of a grid: the parent within 100 tol at two
tolerances, error tracking the tolerance, the low-rank claim for S13 / S24 (ranks well
below the interface length, growing slowly with it), and a planted mistake caught."""
import functools

import numpy as np
import pytest

from oracle import hbs, nd_dense as nd
from paper_1302_5995_gb300 import inputs


@functools.lru_cache(maxsize=None)
def top_merge(n, kind):
    b, c, d = inputs.laplace_fields(n) if kind == "laplace" else inputs.convection_fields(n, seeds=(1, 2, 3))
    prob = nd.Problem(b, c, d, n)
    root = nd.Box(0, 0, n, n)
    sw, se, nw, ne = root.children()
    south, north = nd.Box(0, 0, n, sw.b), nd.Box(0, sw.b, n, nw.b)
    S1, S2 = nd.direct_schur(prob, south), nd.direct_schur(prob, north)
    return prob, south, S1, north, S2, root, nd.merge_two(prob, south, S1, north, S2, root)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("kind", ["laplace", "convection"])
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_accelerated_merge_matches_the_dense_merge(kind, tol):
    prob, s, S1, nrt, S2, root, ref = top_merge(48, kind)
    S, f, ranks = hbs.accelerated_merge(prob, s, S1, nrt, S2, root, tol, 16)
    assert rel(S, ref) < 100 * tol
    assert rel(hbs.to_dense(f), ref) < 100 * tol
    assert f.tree.L >= 2


def test_error_tracks_the_tolerance():
    prob, s, S1, nrt, S2, root, ref = top_merge(48, "convection")
    e6 = rel(hbs.accelerated_merge(prob, s, S1, nrt, S2, root, 1e-6, 16)[0], ref)
    e10 = rel(hbs.accelerated_merge(prob, s, S1, nrt, S2, root, 1e-10, 16)[0], ref)
    assert e10 < 1e-3 * e6


def test_interface_couplings_are_low_rank():
    sp = {}
    rk = {}
    for n in (48, 96):
        prob, s, S1, nrt, S2, root, ref = top_merge(n, "laplace")
        _, _, ranks = hbs.accelerated_merge(prob, s, S1, nrt, S2, root, 1e-10, 16)
        sp[n] = len(nd.partition_we(s, nrt, root)[1])
        rk[n] = max(ranks)
    assert rk[48] < sp[48] and rk[96] < 0.45 * sp[96]  # S13, S24: well below the interface length
    assert rk[96] < 1.5 * rk[48]                        # and growing slowly while it doubles


def test_planted_dropped_off_diagonal_update_is_caught(monkeypatch):
    prob, s, S1, nrt, S2, root, ref = top_merge(48, "laplace")
    real = hbs.low_rank
    calls = []

    def bad(A, tol):  # S24 (factored second) forgotten: the north half loses its update
        calls.append(1)
        L, R = real(A, tol)
        return (L, R) if len(calls) == 1 else (L, 0 * R)

    monkeypatch.setattr(hbs, "low_rank", bad)
    S, _, _ = hbs.accelerated_merge(prob, s, S1, nrt, S2, root, 1e-10, 16)
    assert rel(S, ref) > 1e-3
