"""Seeded synthetic inputs: coefficient fields b, c, d and boundary-data vectors.

This module holds no arithmetic of the solver.  It only draws numbers and samples
analytic functions at grid positions, so that the oracle and the CUDA path can be
fed byte-identical inputs.

Grid convention (the paper's Section 6 stencil on the unit square): n x n unknown
nodes, h = 1/(n+1), node (i, j) sits at ((i+1)h, (j+1)h), flat index i + n*j.
The 4n Dirichlet ("ghost") nodes are the non-corner nodes one step outside the grid,
ordered counter-clockwise from the south-west corner: south (x increasing), east
(y increasing), north (x decreasing), west (y decreasing), n nodes per side.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a 64-bit
counter advanced by the golden-gamma constant, then two xor-shift-multiply rounds.
Uniform doubles use the top 53 bits; normals use the Box-Muller transform.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream; draw(k) returns the next k raw 64-bit outputs."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def draw(self, k: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            ctr = self.state + _GOLDEN_GAMMA * np.arange(1, k + 1, dtype=np.uint64)
            self.state = self.state + _GOLDEN_GAMMA * np.uint64(k)
            z = ctr
            z = (z ^ (z >> np.uint64(30))) * _MIX1
            z = (z ^ (z >> np.uint64(27))) * _MIX2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int) -> np.ndarray:
        """k doubles in [0, 1): top 53 bits times 2^-53."""
        return (self.draw(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, k: int) -> np.ndarray:
        """k standard normals by Box-Muller on pairs of uniforms (u1 mapped to (0, 1])."""
        m = (k + 1) // 2
        u = self.uniform(2 * m)
        u1 = 1.0 - u[0::2]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m)
        z[0::2] = r * np.cos(2.0 * math.pi * u2)
        z[1::2] = r * np.sin(2.0 * math.pi * u2)
        return z[:k]


# ----------------------------------------------------------------------------- geometry

def node_xy(n: int):
    """Coordinates of the n*n unknown nodes, flat order i + n*j."""
    h = 1.0 / (n + 1)
    t = (np.arange(n) + 1) * h
    X, Y = np.meshgrid(t, t, indexing="xy")  # [j, i]
    return X.reshape(-1), Y.reshape(-1)


def ghost_xy(n: int):
    """Coordinates of the 4n ghost (Dirichlet) nodes in counter-clockwise order."""
    h = 1.0 / (n + 1)
    t = (np.arange(n) + 1) * h
    xs = np.concatenate([t, np.ones(n), t[::-1], np.zeros(n)])
    ys = np.concatenate([np.zeros(n), t, np.ones(n), t[::-1]])
    return xs, ys


# ----------------------------------------------------------------------------- fields

def fourier_field(n: int, seed: int, lo: float, hi: float, modes: int = 8) -> np.ndarray:
    """Smooth random field: sum of `modes` terms a * f(2 pi (kx x + ky y)).

    Per mode, in draw order: f in {sin, cos} by a fair coin, kx and ky uniform on
    {0..4}, amplitude a uniform on [lo, hi).
    """
    rng = SplitMix64(seed)
    X, Y = node_xy(n)
    out = np.zeros(n * n)
    for _ in range(modes):
        u = rng.uniform(4)
        f = np.sin if u[0] < 0.5 else np.cos
        kx = int(u[1] * 5.0)
        ky = int(u[2] * 5.0)
        a = lo + (hi - lo) * u[3]
        out += a * f(2.0 * math.pi * (kx * X + ky * Y))
    return out


def convection_fields(n: int, seeds=(1, 2, 3)):
    """Convection-diffusion-reaction fields: b, c with amplitudes U(-5, 5), d with U(0, 10)."""
    b = fourier_field(n, seeds[0], -5.0, 5.0)
    c = fourier_field(n, seeds[1], -5.0, 5.0)
    d = fourier_field(n, seeds[2], 0.0, 10.0)
    return b, c, d


def laplace_fields(n: int):
    z = np.zeros(n * n)
    return z, z.copy(), z.copy()


def constant_fields(n: int, b0: float, c0: float, d0: float):
    return np.full(n * n, b0), np.full(n * n, c0), np.full(n * n, d0)


def box_interior_sizes(n: int, leaf: int):
    """Every (width, height) of a box or half-box rectangle that the quad-tree creates.

    The tree splits a box of width a into floor(a/2) (west) and ceil(a/2) (east), and
    likewise in y; the merge of two siblings forms a half-box rectangle first.
    """
    L = 0
    while -(-n // (1 << L)) > leaf:
        L += 1
    sizes = set()
    boxes = [(n, n)]
    for _ in range(L):
        nxt = []
        for (a, b) in boxes:
            sizes.add((a, b))
            for bb in (b // 2, b - b // 2):
                sizes.add((a, bb))  # half-box rectangles after the horizontal merges
            for aa in (a // 2, a - a // 2):
                for bb in (b // 2, b - b // 2):
                    nxt.append((aa, bb))
        boxes = sorted(set(nxt))
    for s in boxes:
        sizes.add(s)
    return sorted(sizes)


def nudged_wavenumber(n: int, leaf: int, ppw: float = 10.0, margin: float = 0.25,
                      step: float = 1e-4, max_steps: int = 200000) -> float:
    """Wavenumber k = 2 pi (n+1)/ppw, multiplied by (1 + delta) with the smallest scanned
    delta >= 0 that keeps k^2 at least `margin` times the local eigenvalue spacing away
    from every Dirichlet eigenvalue of the 5-point Laplacian on every box interior of
    the tree and on the whole grid (constant-coefficient proxy).

    Eigenvalues of an (a-2) x (b-2) interior with spacing h:
    (4/h^2)(sin^2(p pi / (2(a-1))) + sin^2(q pi / (2(b-1)))).
    """
    h = 1.0 / (n + 1)
    k0 = 2.0 * math.pi * (n + 1) / ppw
    spectra = []
    shapes = [(a - 2, b - 2) for (a, b) in box_interior_sizes(n, leaf) if a > 2 and b > 2]
    shapes.append((n, n))
    for (ia, ib) in set(shapes):
        p = np.arange(1, ia + 1)
        q = np.arange(1, ib + 1)
        ev = (4.0 / h**2) * (np.sin(p * math.pi / (2 * (ia + 1)))[:, None] ** 2
                             + np.sin(q * math.pi / (2 * (ib + 1)))[None, :] ** 2)
        spectra.append(np.unique(ev.reshape(-1)))
    for s in range(max_steps):
        k = k0 * (1.0 + s * step)
        k2 = k * k
        ok = True
        for ev in spectra:
            idx = np.searchsorted(ev, k2)
            lo_i = max(idx - 1, 0)
            hi_i = min(idx, len(ev) - 1)
            gap = ev[hi_i] - ev[lo_i] if hi_i > lo_i else (ev[1] - ev[0] if len(ev) > 1 else ev[0])
            dist = min(abs(k2 - ev[lo_i]), abs(k2 - ev[hi_i]))
            if dist < margin * gap:
                ok = False
                break
        if ok:
            return k
    raise RuntimeError("no non-resonant wavenumber found")


def helmholtz_fields(n: int, k: float):
    """Variable wave speed: b = c = 0, d = -k^2 (1 - 0.5 exp(-|x - (0.5, 0.5)|^2 / 0.02))."""
    X, Y = node_xy(n)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
    d = -(k * k) * (1.0 - 0.5 * np.exp(-r2 / 0.02))
    z = np.zeros(n * n)
    return z, z.copy(), d


# ----------------------------------------------------------------------------- the paper's problem set

def discrete_laplace_eigenvalue(n: int, index: int) -> float:
    """The index-th smallest eigenvalue (1-based, repeated eigenvalues counted) of the
    five-point Dirichlet Laplacian on the n x n unknowns: (4/h^2)(sin^2(p pi h/2) +
    sin^2(q pi h/2)), p, q = 1..n."""
    h = 1.0 / (n + 1)
    s2 = np.sin(np.arange(1, n + 1) * math.pi * h / 2.0) ** 2
    ev = np.sort(((4.0 / h**2) * (s2[:, None] + s2[None, :])).reshape(-1))
    return float(ev[index - 1])


PAPER_PROBLEMS = ("laplace", "diffconv1", "diffconv2", "diffconv3", "diffconv4",
                  "helmholtz1", "helmholtz2", "helmholtz3", "helmholtz4")


def paper_problem(name: str, n: int):
    """Fields (b, c, d) of the PDE problems of Section 6.1, sampled at the unknowns:
    Laplace; Diffusion-Convection I/II (b = 100 / 1000); III (b = 125 cos 4 pi y,
    c = 125 sin 4 pi x, divergence free); IV (b = 125 cos 4 pi x, c = 125 sin 4 pi y);
    Helmholtz I/II (d = -100 / -4005); III (d = -lambda_10 + 1e-5, lambda_10 the tenth
    eigenvalue of the discrete Laplacian: near resonance); IV (d = -(2 pi (n+1)/40)^2,
    40 points per wavelength at h = 1/(n+1))."""
    X, Y = node_xy(n)
    z = np.zeros(n * n)
    b, c, d = z.copy(), z.copy(), z.copy()
    if name == "laplace":
        pass
    elif name == "diffconv1":
        b[:] = 100.0
    elif name == "diffconv2":
        b[:] = 1000.0
    elif name == "diffconv3":
        b, c = 125.0 * np.cos(4.0 * math.pi * Y), 125.0 * np.sin(4.0 * math.pi * X)
    elif name == "diffconv4":
        b, c = 125.0 * np.cos(4.0 * math.pi * X), 125.0 * np.sin(4.0 * math.pi * Y)
    elif name == "helmholtz1":
        d[:] = -100.0
    elif name == "helmholtz2":
        d[:] = -4005.0
    elif name == "helmholtz3":
        d[:] = -discrete_laplace_eigenvalue(n, 10) + 1e-5
    elif name == "helmholtz4":
        d[:] = -(2.0 * math.pi * (n + 1) / 40.0) ** 2
    else:
        raise ValueError(f"unknown problem {name}")
    return b, c, d


def error_vectors(n: int, seed: int):
    """The two boundary vectors of the paper's error measures (Section 6.1): a unit
    vector of random direction (normalised N(0,1) draw) and a smooth one, the trace of
    cos(2 pi x) exp(y) + x y on the ghost ring, normalised.  Shape (4n, 2)."""
    r = SplitMix64(seed).normal(4 * n)
    x, y = ghost_xy(n)
    sm = np.cos(2.0 * math.pi * x) * np.exp(y) + x * y
    return np.stack([r / np.linalg.norm(r), sm / np.linalg.norm(sm)], axis=1)


# ----------------------------------------------------------------------------- networks and body loads

def network_conductivities(n: int, lo: float, hi: float, seed: int):
    """Random link conductivities of the square-grid network (the Random Laplacian
    problems of Section 6.1): every link, including the 4n links from the grid to its
    ghost nodes, gets a conductivity uniform on [lo, hi).

    Returns (sx, sy).  sx has n rows of n + 1 x-links, flat index i + (n+1) j: the link
    between (i-1, j) and (i, j) for i = 0..n (i = 0 and i = n reach the west and east
    ghosts).  sy has n + 1 rows of n y-links, flat index i + n j: the link between
    (i, j-1) and (i, j) for j = 0..n (j = 0 and j = n reach the south and north ghosts).
    Draw order: sx, then sy.
    """
    rng = SplitMix64(seed)
    sx = lo + (hi - lo) * rng.uniform(n * (n + 1))
    sy = lo + (hi - lo) * rng.uniform((n + 1) * n)
    return sx, sy


def random_laplacian_1(n: int, seed: int = 21):
    """Random Laplacian I: conductivities uniform on [1, 2)."""
    return network_conductivities(n, 1.0, 2.0, seed)


def random_laplacian_2(n: int, seed: int = 22):
    """Random Laplacian II: conductivities uniform on [1, 1000)."""
    return network_conductivities(n, 1.0, 1000.0, seed)


def body_nodes(n: int, count: int, seed: int) -> np.ndarray:
    """count distinct unknown nodes in a localized square window (Section 6.3 places the
    loads in a small area): window edge w = min(n, max(4, ceil(2 sqrt(count)))), its
    south-west corner uniform among the positions that keep it inside the grid, then
    `count` distinct nodes of the window in the order of a random permutation (argsort
    of uniforms).  Returns flat indices i + n j, in load-column order."""
    if count > n * n:
        raise ValueError("more body nodes than unknowns")
    w = min(n, max(4, math.ceil(2.0 * math.sqrt(count))))
    while w * w < count:
        w += 1
    rng = SplitMix64(seed)
    u = rng.uniform(2)
    x0 = int(u[0] * (n - w + 1))
    y0 = int(u[1] * (n - w + 1))
    order = np.argsort(rng.uniform(w * w), kind="stable")[:count]
    return ((x0 + order % w) + n * (y0 + order // w)).astype(np.int64)


def body_load_vectors(count: int, nvec: int, seed: int) -> np.ndarray:
    """nvec i.i.d. N(0,1) load vectors on `count` body nodes, shape (count, nvec)."""
    z = SplitMix64(seed).normal(count * nvec)
    return z.reshape(nvec, count).T.copy()


# ----------------------------------------------------------------------------- boundary data

def harmonic_vectors(n: int) -> np.ndarray:
    """Columns 1, x, y, x^2 - y^2, x y sampled at the ghost nodes; shape (4n, 5)."""
    x, y = ghost_xy(n)
    return np.stack([np.ones_like(x), x, y, x * x - y * y, x * y], axis=1)


def gaussian_vectors(n: int, count: int, seed: int) -> np.ndarray:
    """count i.i.d. N(0,1) boundary vectors, shape (4n, count), vector j = column j."""
    z = SplitMix64(seed).normal(4 * n * count)
    return z.reshape(count, 4 * n).T.copy()


def plane_wave_vectors(n: int, k: float, count_angles: int, seed: int) -> np.ndarray:
    """Real and imaginary parts of exp(i k (x cos t + y sin t)) on the ghost ring for
    count_angles angles t ~ U(0, 2 pi); shape (4n, 2 * count_angles)."""
    x, y = ghost_xy(n)
    th = 2.0 * math.pi * SplitMix64(seed).uniform(count_angles)
    ph = k * (x[:, None] * np.cos(th)[None, :] + y[:, None] * np.sin(th)[None, :])
    out = np.empty((4 * n, 2 * count_angles))
    out[:, 0::2] = np.cos(ph)
    out[:, 1::2] = np.sin(ph)
    return out


def config1(n: int = 64):
    """Laplace on 64 x 64, 16 vectors: the five harmonic columns then 11 N(0,1) (seed 0)."""
    b, c, d = laplace_fields(n)
    G = np.concatenate([harmonic_vectors(n), gaussian_vectors(n, 11, 0)], axis=1)
    return dict(n=n, leaf=8, b=b, c=c, d=d, G=G)


def config2(n: int = 512, nvec: int = 256):
    """Convection-diffusion-reaction on 512 x 512, leaf 16, 256 Gaussian vectors (seed 4)."""
    b, c, d = convection_fields(n)
    return dict(n=n, leaf=16, b=b, c=c, d=d, G=gaussian_vectors(n, nvec, 4))


def config3(n: int = 1024, leaf: int = 16, angles: int = 32):
    """Variable-wavespeed Helmholtz at 10 points per wavelength, plane-wave data (seed 5)."""
    k = nudged_wavenumber(n, leaf)
    b, c, d = helmholtz_fields(n, k)
    return dict(n=n, leaf=leaf, k=k, b=b, c=c, d=d, G=plane_wave_vectors(n, k, angles, 5))


def config4(count: int = 64, sizes=(128, 192, 256, 384, 512), leaf: int = 16, seed: int = 6):
    """Batch of independent problems: n drawn uniformly from `sizes` (seeded); the even
    positions carry convection-diffusion-reaction fields (Fourier seeds 100 + 3p ...),
    the odd ones variable-wavespeed Helmholtz at 10 points per wavelength for their own n.
    Returns a list of dicts with n, leaf, kind, b, c, d."""
    pick = (SplitMix64(seed).draw(count) % np.uint64(len(sizes))).astype(np.int64)
    ks = {}
    out = []
    for p in range(count):
        n = int(sizes[pick[p]])
        if p % 2 == 0:
            b, c, d = convection_fields(n, seeds=(100 + 3 * p, 101 + 3 * p, 102 + 3 * p))
            out.append(dict(n=n, leaf=leaf, kind="convection", b=b, c=c, d=d))
        else:
            if n not in ks:
                ks[n] = nudged_wavenumber(n, leaf)
            b, c, d = helmholtz_fields(n, ks[n])
            out.append(dict(n=n, leaf=leaf, kind="helmholtz", k=ks[n], b=b, c=c, d=d))
    return out
