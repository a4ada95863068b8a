"""Exact discrete solutions used to pin the oracle (test infrastructure only).

None of these routines performs nested dissection; each one is an independent
route to values the five-point scheme of Section 6 fixes exactly.

1. Discrete exponentials.  With constant b, c, d the grid function
       u(i, j) = mu^(i+1) nu^(j+1)
   satisfies the scheme at every unknown node iff
       (1/h^2)(4 - mu - 1/mu - nu - 1/nu) + (b/h)(mu - 1/mu) + (c/h)(nu - 1/nu) + d = 0.
   For a chosen nu this is a quadratic in mu.  Sampling u at the ghosts gives Dirichlet
   data whose exact Neumann data is (u(ghost) - u(neighbour))/h.
2. Harmonic polynomials.  For b = c = d = 0 the five-point Laplacian annihilates
   1, x, y, x^2 - y^2 and x y exactly, so the same formula holds for them.
3. Sine transform.  With constant b, c (|bh|, |ch| < 1) and d, the diagonal similarity
   u = rho_x^i rho_y^j w, rho = sqrt((1 + bh)/(1 - bh)), makes the operator symmetric
   with eigenvectors sin(p pi (i+1)/(n+1)) sin(q pi (j+1)/(n+1)); the system is then
   solved exactly by two type-I discrete sine transforms (scipy.fft).  The same solve
   with a unit body load and zero Dirichlet data gives the load operator's columns.
"""
from __future__ import annotations

import numpy as np


def _ghost_and_neighbour_positions(n):
    """Integer positions (i, j) of ghost k and of its unknown neighbour."""
    t = np.arange(n)
    gi = np.concatenate([t, np.full(n, n), t[::-1], np.full(n, -1)])
    gj = np.concatenate([np.full(n, -1), t, np.full(n, n), t[::-1]])
    ni = np.clip(gi, 0, n - 1)
    nj = np.clip(gj, 0, n - 1)
    return gi, gj, ni, nj


def exponential_mu(n, b, c, d, nu):
    """Both roots mu of the quadratic above for the given nu (real roots only)."""
    h = 1.0 / (n + 1)
    # multiply the condition by mu h^2:
    # (b h - 1) mu^2 + (4 - nu - 1/nu + c h (nu - 1/nu) + d h^2) mu - (1 + b h) = 0
    A = b * h - 1.0
    B = 4.0 - nu - 1.0 / nu + c * h * (nu - 1.0 / nu) + d * h * h
    C = -(1.0 + b * h)
    disc = B * B - 4 * A * C
    if disc < 0:
        raise ValueError("complex roots")
    s = np.sqrt(disc)
    return ((-B + s) / (2 * A), (-B - s) / (2 * A))


def exponential_pair(n, b, c, d, nu, root=0):
    """(g, v): Dirichlet data of u = mu^(i+1) nu^(j+1) and its exact Neumann data."""
    h = 1.0 / (n + 1)
    mu = exponential_mu(n, b, c, d, nu)[root]
    gi, gj, ni, nj = _ghost_and_neighbour_positions(n)
    ug = mu ** (gi + 1.0) * nu ** (gj + 1.0)
    un = mu ** (ni + 1.0) * nu ** (nj + 1.0)
    return ug, (ug - un) / h


def harmonic_pairs(n):
    """(G, V) for the five harmonic polynomials of the Laplace case."""
    h = 1.0 / (n + 1)
    gi, gj, ni, nj = _ghost_and_neighbour_positions(n)
    polys = [lambda x, y: np.ones_like(x), lambda x, y: x, lambda x, y: y,
             lambda x, y: x * x - y * y, lambda x, y: x * y]
    xg, yg = (gi + 1) * h, (gj + 1) * h
    xn, yn = (ni + 1) * h, (nj + 1) * h
    G = np.stack([p(xg, yg) for p in polys], axis=1)
    V = np.stack([(p(xg, yg) - p(xn, yn)) / h for p in polys], axis=1)
    return G, V


def _dst_solver(n, b, c, d):
    """Exact solve of the constant-coefficient scheme (zero Dirichlet data) by the sine
    transform: returns (solve, weights), solve(F) -> U for right-hand sides F[k, j, i]."""
    from scipy.fft import dstn

    h = 1.0 / (n + 1)
    ih2 = 1.0 / (h * h)
    wC = 4 * ih2 + d
    wE, wW = -ih2 + b / h, -ih2 - b / h
    wN, wS = -ih2 + c / h, -ih2 - c / h
    if not (abs(b * h) < 1 and abs(c * h) < 1):
        raise ValueError("need |bh|, |ch| < 1")
    rx, ry = np.sqrt(wW / wE), np.sqrt(wS / wN)
    sx, sy = np.sqrt(wE * wW), np.sqrt(wN * wS)
    p = np.arange(1, n + 1)
    lam = (wC - 2 * sx * np.cos(p * np.pi / (n + 1)))[None, :] \
        - 2 * sy * np.cos(p * np.pi / (n + 1))[:, None]  # [q, p]
    i = np.arange(n)
    scale = (rx ** i)[None, :] * (ry ** i)[:, None]  # u = scale * w

    def solve(F):
        Fw = F / scale[None]
        # exact inverse of the symmetric operator: orthonormal DST-I diagonalises it
        W = dstn(dstn(Fw, type=1, axes=(1, 2), norm="ortho") / lam[None], type=1, axes=(1, 2),
                 norm="ortho")
        return W * scale[None]

    return solve, dict(E=wE, W=wW, N=wN, S=wS)


def dst_dtn_matrix(n, b, c, d):
    """Full 4n x 4n DtN matrix for constant coefficients by the sine transform."""
    h = 1.0 / (n + 1)
    solve, w = _dst_solver(n, b, c, d)
    gi, gj, ni, nj = _ghost_and_neighbour_positions(n)
    wdir = np.select([gj < 0, gi >= n, gj >= n, gi < 0], [w["S"], w["E"], w["N"], w["W"]])
    F = np.zeros((4 * n, n, n))  # right-hand side of each unit ghost vector, [k, j, i]
    F[np.arange(4 * n), nj, ni] = -wdir
    U = solve(F)
    T = np.zeros((4 * n, 4 * n))
    T[:, :] = -U[:, nj, ni].T / h  # row = ghost whose flux we read, column = data vector
    T += np.eye(4 * n) / h
    return T


def dst_load_matrix(n, b, c, d, idx):
    """Body-load operator F (4n x len(idx)) for constant coefficients: column m is the
    flux -u_{k'}/h of the solution with a unit load at node idx[m] (flat i + n j) and zero
    Dirichlet data, the solution taken exactly by the sine transform."""
    h = 1.0 / (n + 1)
    solve, _ = _dst_solver(n, b, c, d)
    idx = np.asarray(idx).reshape(-1)
    F = np.zeros((idx.size, n, n))
    F[np.arange(idx.size), idx // n, idx % n] = 1.0
    U = solve(F)
    gi, gj, ni, nj = _ghost_and_neighbour_positions(n)
    return -U[:, nj, ni].T / h
