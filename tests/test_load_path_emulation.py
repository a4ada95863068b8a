"""The body-load build's device steps emulated on the CPU, index for index, before they
run on a GPU: the loop bodies of k_leaf_load_assemble, k_leaf_load_finalize,
k_merge_assemble, k_merge_load_assemble, k_merge_load_update, the root assembly and
k_load_finalize (csrc/loads.cu, csrc/kernels_fp64.cu) are written out here over the
offsets and index tables of the library's own plan and load plan (compiled from
csrc/plan.cpp and csrc/loads_plan.cpp), every buffer starts as NaN, every write is
bounds-checked, and the load operator F that comes out must equal the oracle's.  The
dense sweeps are LAPACK solves here and the parents' Schur complements the oracle's
(those device steps are the plain build's, checked by the GPU parity tests).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import nd_dense as nd
from oracle import o1
from paper_1302_5995_gb300 import inputs

from test_load_plan_host import dump as load_dump
from test_plan_host import parse as plan_parse
from test_server_host import _cuda_include

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C, E, W, N, S = 0, 1, 2, 3, 4
DIRS = [(E, 1, 0), (W, -1, 0), (N, 0, 1), (S, 0, -1)]


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("no CUDA headers")
    out = str(tmp_path_factory.mktemp("emul") / "shims.so")
    csrc = os.path.join(ROOT, "paper_1302_5995_gb300", "csrc")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", inc, "-o", out,
                           os.path.join(ROOT, "tests", "plan_shim.cpp"),
                           os.path.join(ROOT, "tests", "load_plan_shim.cpp"),
                           os.path.join(csrc, "loads_plan.cpp"), os.path.join(csrc, "plan.cpp")])
    lib = ctypes.CDLL(out)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.plan_dump.argtypes = [ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int64]
    lib.plan_dump.restype = ctypes.c_int64
    lib.load_plan_dump.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, i64p,
                                   ctypes.c_int64]
    lib.load_plan_dump.restype = ctypes.c_int64
    return lib


def plain_plan(lib, n, leaf):
    cap = 1 << 18
    buf = np.zeros(cap, dtype=np.int64)
    got = lib.plan_dump(n, leaf, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
    assert got > 0
    return plan_parse(buf[:got].tolist())


class Buf:
    """A device buffer stand-in: NaN-filled, every access bounds-checked."""

    def __init__(self, size):
        self.a = np.full(max(int(size), 1), np.nan)

    def __getitem__(self, i):
        assert 0 <= i < self.a.size, i
        return self.a[i]

    def __setitem__(self, i, v):
        assert 0 <= i < self.a.size, i
        self.a[i] = v

    def block(self, off, rows, cols):
        assert off >= 0 and off + rows * cols <= self.a.size
        return self.a[off: off + rows * cols].reshape((rows, cols), order="F")


def emulate_F(prob, n, leaf, body, plan, lp):
    w = lambda g, d: prob.w[d][g // n, g % n]  # the stencil weight of equation g towards d
    A = Buf(plan["arena"])  # every box's Schur complement, by its plain definition
    for l in plan["leaves"]:
        bx = nd.Box(l["x0"], l["y0"], l["a"], l["b"])
        r = len(bx.ring())
        A.block(l["off"], r, r)[:] = nd.direct_schur(prob, bx)
    for st in plan["stages"]:
        for m in st["merges"]:
            A.block(m["out"], m["rp"], m["rp"])[:] = nd.direct_schur(prob, m["par"])
    LA = Buf(lp["arena"])
    # leaves: k_leaf_load_assemble, the sweep, k_leaf_load_finalize
    lws = Buf(lp["leaf_ws"])
    nodes = [g for d in lp["leaves"] for g in d["nodes"]]
    for d in lp["leaves"]:
        ni, ia, m = d["ni"], d["a"] - 2, d["m"]
        if d["sys"] >= 0:
            for e in range(ni * (ni + m)):
                p, col = e % ni, e // ni
                i, j = 1 + p % ia, 1 + p // ia
                g = (d["x0"] + i) + n * (d["y0"] + j)
                v = 0.0
                if col < ni:
                    iq, jq = 1 + col % ia, 1 + col // ia
                    if col == p:
                        v = w(g, C)
                    else:
                        for (dr, di, dj) in DIRS:
                            if iq == i + di and jq == j + dj:
                                v = w(g, dr)
                else:
                    v = 1.0 if nodes[d["col0"] + col - ni] == g else 0.0
                lws[d["sys"] + e] = v
            Wl = lws.block(d["sys"], ni, ni + m)
            Wl[:, ni:] = np.linalg.solve(Wl[:, :ni], Wl[:, ni:])
        a, b = d["a"], d["b"]
        r = 2 * a + 2 * b - 4
        ring = nd.Box(0, 0, a, b).ring()
        for e in range(r * m):
            rb, col = e % r, e // r
            i, j = ring[rb]
            g = (d["x0"] + i) + n * (d["y0"] + j)
            v = 1.0 if nodes[d["col0"] + col] == g else 0.0
            if d["sys"] >= 0:
                for (dr, di, dj) in DIRS:
                    i2, j2 = i + di, j + dj
                    if 1 <= i2 <= a - 2 and 1 <= j2 <= b - 2:
                        v -= w(g, dr) * lws[d["sys"] + ni * ni + (i2 - 1) + ia * (j2 - 1) + ni * col]
            LA[d["lout"] + e] = v
    # merges: k_merge_assemble, k_merge_load_assemble, the sweep, k_merge_load_update
    for st, lst in zip(plan["stages"], lp["stages"]):
        ws = Buf(lst["ws"])
        for M, D in zip(st["merges"], lst["merges"]):
            sp, rp, n1 = M["sp"], M["rp"], M["n1"]
            mm, mL = 2 * sp, D["m1"] + D["m2"]
            d34, d43 = (N, S) if M["orient"] else (E, W)
            for e in range(mm * (mm + rp)):
                t, c = e % mm, e // mm
                if c < mm:
                    if t < sp and c < sp:
                        v = A[M["s1"] + M["p3"][t] + M["r1"] * M["p3"][c]]
                    elif t >= sp and c >= sp:
                        v = A[M["s2"] + M["p4"][t - sp] + M["r2"] * M["p4"][c - sp]]
                    elif t < sp:
                        v = w(M["g3"][t], d34) if c - sp == t else 0.0
                    else:
                        v = w(M["g4"][t - sp], d43) if c == t - sp else 0.0
                else:
                    cc = c - mm
                    if cc < n1:
                        v = A[M["s1"] + M["p3"][t] + M["r1"] * M["p1"][cc]] if t < sp else 0.0
                    else:
                        v = A[M["s2"] + M["p4"][t - sp] + M["r2"] * M["p2"][cc - n1]] if t >= sp else 0.0
                ws[D["ws"] + e] = v
            if mL and mm:
                base = D["ws"] + mm * (mm + rp)
                for e in range(mm * mL):
                    t, col = e % mm, e // mm
                    v = 0.0
                    if t < sp and col < D["m1"]:
                        v = LA[D["l1"] + M["p3"][t] + M["r1"] * col]
                    elif t >= sp and col >= D["m1"]:
                        v = LA[D["l2"] + M["p4"][t - sp] + M["r2"] * (col - D["m1"])]
                    ws[base + e] = v
            ncol = mm + rp + mL
            assert D["sncol"] == ncol
            if mm:
                Wm = ws.block(D["ws"], mm, ncol)
                Wm[:, mm:] = np.linalg.solve(Wm[:, :mm], Wm[:, mm:])
            if mL:
                XL = D["ws"] + mm * (mm + rp)
                for e in range(rp * mL):
                    a, col = e % rp, e // rp
                    g = acc = 0.0
                    if a < n1:
                        if col < D["m1"]:
                            g = LA[D["l1"] + M["p1"][a] + M["r1"] * col]
                        for t in range(sp):
                            acc += A[M["s1"] + M["p1"][a] + M["r1"] * M["p3"][t]] * ws[XL + t + mm * col]
                        qa = M["q1"][a]
                    else:
                        a2 = a - n1
                        if col >= D["m1"]:
                            g = LA[D["l2"] + M["p2"][a2] + M["r2"] * (col - D["m1"])]
                        for t in range(sp):
                            acc += A[M["s2"] + M["p2"][a2] + M["r2"] * M["p4"][t]] * ws[XL + sp + t + mm * col]
                        qa = M["q2"][a2]
                    LA[D["lout"] + qa + rp * col] = g - acc
    # root: [S_root | B | L_root], the sweep, k_load_finalize
    (root,) = plan["roots"]
    r, nb4, m = root["r"], 4 * n, len(body)
    Wr = Buf(r * (r + nb4 + m))
    Wr.block(0, r, r)[:] = A.block(root["off"], r, r)
    ring = nd.Box(0, 0, n, n).ring()
    for k, (q, wgt) in enumerate(nd.ghost_map(prob)):
        col = Wr.block(r * (r + k), r, 1)
        col[:] = 0.0
        p = k - k // n
        p = p - r if p >= r else p  # the device's ghost -> root ring position
        assert ring[p] == q
        col[p, 0] = -wgt
    for e in range(r * m):
        Wr[r * (r + nb4) + e] = LA[lp["root_l"] + e]
    Wm = Wr.block(0, r, r + nb4 + m)
    Wm[:, r:] = np.linalg.solve(Wm[:, :r], Wm[:, r:])
    F = Buf(nb4 * m)
    ih = n + 1.0
    for e in range(nb4 * m):
        k, col = e % nb4, e // nb4
        p = k - k // n
        p = p - r if p >= r else p
        F[k + nb4 * lp["root_order"][col]] = -Wr[r * (r + nb4) + p + r * col] * ih
    return F.a.reshape((m, nb4)).T


@pytest.mark.parametrize("n,leaf,count,seed", [(9, 4, 6, 1), (23, 6, 12, 3), (30, 8, 20, 4)])
def test_emulated_load_path_gives_the_oracle_F(shim, n, leaf, count, seed):
    b, c, d = inputs.convection_fields(n, seeds=(91, 92, 93))
    prob = nd.Problem(b, c, d, n)
    body = [int(g) for g in inputs.body_nodes(n, count, seed)]
    for g in (0, n - 1, (n // 2) * n + 3, (n // 2 - 1) * n + n // 2, n * n - 1):  # ring, interfaces, corner
        if g not in body:
            body.append(g)
    plan = plain_plan(shim, n, leaf)
    lp = load_dump(shim, n, leaf, body)
    assert plan["rc"] == 0 and lp["rc"] == 0
    F = emulate_F(prob, n, leaf, body, plan, lp)
    assert np.isfinite(F).all()
    F_ref = o1.load_matrix(b, c, d, n, body)
    assert np.abs(F - F_ref).max() / np.abs(F_ref).max() < 1e-10


def emulate_net_weights(sx, sy, n):
    """k_net_weights (csrc/network.cu), index for index: the weight table W (5 per node)
    and the ghosts' link conductivities."""
    ih2 = (n + 1.0) ** 2
    Wt, sig = Buf(5 * n * n), Buf(4 * n)
    for g in range(n * n + 4 * n):
        if g < n * n:
            i, j = g % n, g // n
            e, w_ = sx[(i + 1) + (n + 1) * j], sx[i + (n + 1) * j]
            no, so = sy[i + n * (j + 1)], sy[i + n * j]
            Wt[5 * g + C] = (e + w_ + no + so) * ih2
            Wt[5 * g + E] = -e * ih2
            Wt[5 * g + W] = -w_ * ih2
            Wt[5 * g + N] = -no * ih2
            Wt[5 * g + S] = -so * ih2
        else:
            k = g - n * n
            side, t = divmod(k, n)
            sig[k] = [sy[t], sx[n + (n + 1) * t], sy[(n - 1 - t) + n * n], sx[(n + 1) * (n - 1 - t)]][side]
    return Wt.a, sig.a


@pytest.mark.parametrize("make", [inputs.random_laplacian_1, inputs.random_laplacian_2])
def test_emulated_network_path_gives_the_oracle_F(shim, make):
    n, leaf = 23, 6
    sx, sy = make(n)
    prob = nd.Problem.network(sx, sy, n)
    Wt, sig = emulate_net_weights(sx, sy, n)
    for dr in (C, E, W, N, S):  # the table the FP64 kernels read is the oracle's stencil
        np.testing.assert_array_equal(Wt[dr::5], prob.w[dr].reshape(-1))
    np.testing.assert_array_equal(sig, prob.datum_weights())
    body = [int(g) for g in inputs.body_nodes(n, 10, 6)] + [0, n * n - 1]
    plan = plain_plan(shim, n, leaf)
    lp = load_dump(shim, n, leaf, body)
    F = emulate_F(prob, n, leaf, body, plan, lp) * sig[:, None]  # k_scale_rows
    F_ref = o1.net_load_matrix(sx, sy, n, body)
    assert np.abs(F - F_ref).max() / np.abs(F_ref).max() < 1e-10


def test_emulated_apply_add_tiles():
    """k_apply_add (csrc/loads.cu): 16 x 16 output tiles, the k loop in steps of 16 through
    shared tiles Ft[k][row] and Lt[col][k], with the kernel's bounds on every load."""
    N, m, B = 37, 21, 19  # ragged in every dimension
    rng = np.random.default_rng(3)
    Fm, Lm, V0 = rng.standard_normal((N, m)), rng.standard_normal((m, B)), rng.standard_normal((N, B))
    F = Fm.reshape(-1, order="F")
    Fl = Lm.reshape(-1, order="F")
    V = V0.reshape(-1, order="F").copy()
    for bx in range((N + 15) // 16):
        for by in range((B + 15) // 16):
            acc = np.zeros((16, 16))  # acc[ty][tx]
            for k0 in range(0, m, 16):
                Ft = np.zeros((16, 16))
                Lt = np.zeros((16, 16))
                for ty in range(16):
                    for tx in range(16):
                        fr, fk = bx * 16 + tx, k0 + ty
                        Ft[ty, tx] = F[fr + N * fk] if (fr < N and fk < m) else 0.0
                        lk, lc = k0 + tx, by * 16 + ty
                        Lt[ty, tx] = Fl[lk + m * lc] if (lk < m and lc < B) else 0.0
                for ty in range(16):
                    for tx in range(16):
                        acc[ty, tx] += sum(Ft[q, tx] * Lt[ty, q] for q in range(16))
            for ty in range(16):
                for tx in range(16):
                    row, col = bx * 16 + tx, by * 16 + ty
                    if row < N and col < B:
                        V[row + N * col] += acc[ty, tx]
    np.testing.assert_allclose(V.reshape((N, B), order="F"), V0 + Fm @ Lm, rtol=1e-12, atol=1e-12)
