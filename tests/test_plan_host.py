"""The library's host plan (csrc/plan.cpp: Section 2's quad-tree, the ring orders, the
P1..P4 index tables of eq. partition_we, the stage order of Section 3.3 and the arena
layout) checked on the CPU against the oracle's tree and partition.

plan.cpp is compiled here with g++ beside a test-only shim (tests/plan_shim.cpp) that
writes the plan out as integers; nothing runs on a GPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import nd_dense

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GM_EINVAL = -1


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("plan") / "plan_shim.so")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-o", out,
                           os.path.join(ROOT, "tests", "plan_shim.cpp"),
                           os.path.join(ROOT, "paper_1302_5995_gb300", "csrc", "plan.cpp")])
    lib = ctypes.CDLL(out)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.plan_dump.argtypes = [ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int64]
    lib.plan_dump.restype = ctypes.c_int64
    lib.plan_dump_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    i64p, i64p, ctypes.c_int64]
    lib.plan_dump_batch.restype = ctypes.c_int64
    return lib


def _call(fn, *args):
    cap = 1 << 16
    while True:
        buf = np.zeros(cap, dtype=np.int64)
        got = fn(*args, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
        if got >= 0:
            return buf[:got].tolist()
        cap = -got


def parse(rec):
    it = iter(rec)
    nxt = lambda k: [next(it) for _ in range(k)]
    rc, L, leaf_doubles, arena, coef_total, nleaves, nstages, nroots = nxt(8)
    P = dict(rc=rc, L=L, leaf_doubles=leaf_doubles, arena=arena, coef_total=coef_total,
             roots=[], leaves=[], stages=[])
    if rc:
        return P
    for _ in range(nroots):
        P["roots"].append(dict(zip(["n", "r", "off", "coef", "problem"], nxt(5))))
    for _ in range(nleaves):
        P["leaves"].append(dict(zip(["x0", "y0", "a", "b", "off", "n", "prob", "coef"], nxt(8))))
    for _ in range(nstages):
        st = dict(zip(["orient", "nmerges", "out_base", "out_doubles", "ws_doubles", "dig_elems",
                       "exp_elems", "max_m", "max_ncol", "max_rp"], nxt(10)))
        st["merges"] = []
        for _ in range(st["nmerges"]):
            m = dict(zip(["s1", "s2", "out", "ws", "r1", "r2", "rp", "sp", "n1", "n2", "orient", "n",
                          "kpad", "eoff", "doff", "prob"], nxt(16)))
            m["c1"], m["c2"], m["par"] = (nd_dense.Box(*nxt(4)) for _ in range(3))
            sp, n1, n2 = m["sp"], m["n1"], m["n2"]
            for name, k in (("p3", sp), ("p4", sp), ("g3", sp), ("g4", sp), ("p1", n1), ("q1", n1),
                            ("p2", n2), ("q2", n2), ("x12", 8)):
                m[name] = nxt(k)
            st["merges"].append(m)
        P["stages"].append(st)
    assert next(it, None) is None
    return P


def plan(shim, n, leaf):
    return parse(_call(shim.plan_dump, n, leaf))


def expected_merges(n, leaf):
    """Stage by stage (finest level first; horizontal merges, then vertical), the
    (child1, child2, parent) triples of the oracle's tree in its merge order."""
    levels = nd_dense.quad_tree(n, leaf)
    L = len(levels) - 1
    out = []
    for lev in range(L, 0, -1):
        H, V = [], []
        for p in levels[lev - 1]:
            sw, se, nw, ne = p.children()
            south = nd_dense.Box(p.x0, p.y0, p.a, sw.b)
            north = nd_dense.Box(p.x0, p.y0 + sw.b, p.a, nw.b)
            H += [(sw, se, south), (nw, ne, north)]
            V.append((south, north, p))
        out += [H, V]
    return levels, out


def node(n, g, co=0):
    g -= co
    return (g % n, g // n)


def check_merge(m, n, co=0):
    c1, c2, par = m["c1"], m["c2"], m["par"]
    r1, r2, rp = c1.ring(), c2.ring(), par.ring()
    i1, i3, i2, i4, P1, P3, P2, P4 = nd_dense.partition_we(c1, c2, par)
    assert (m["r1"], m["r2"], m["rp"]) == (len(r1), len(r2), len(rp))
    assert (m["sp"], m["n1"], m["n2"]) == (len(i3), len(i1), len(i2)) and len(i3) == len(i4)
    # P3 / P4: the same node sets, paired across the shared edge, with matching globals
    assert sorted(m["p3"]) == sorted(i3) and sorted(m["p4"]) == sorted(i4)
    step = 1 if m["orient"] == 0 else n
    for k in range(m["sp"]):
        assert r1[m["p3"][k]] == node(n, m["g3"][k], co)
        assert r2[m["p4"][k]] == node(n, m["g4"][k], co)
        assert m["g4"][k] - m["g3"][k] == step
    # P1 / P2 in child ring order, each mapped to its parent ring position
    assert m["p1"] == i1 and m["p2"] == i2
    assert [rp.index(r1[p]) for p in m["p1"]] == m["q1"]
    assert [rp.index(r2[p]) for p in m["p2"]] == m["q2"]
    assert sorted(m["q1"] + m["q2"]) == list(range(len(rp)))
    # the two corner couplings across the shared edge
    for e in range(2):
        a1, a2, g1, g2 = m["x12"][4 * e: 4 * e + 4]
        assert r1[m["p1"][a1]] == node(n, g1, co) and r2[m["p2"][a2]] == node(n, g2, co)
        assert g2 - g1 == step
    # workspace row length of the digit planes
    assert m["kpad"] == max(16, -(-2 * m["sp"] // 16) * 16)


@pytest.mark.parametrize("n,leaf", [(5, 4), (12, 4), (23, 4), (37, 5), (64, 8), (100, 16), (129, 16)])
def test_plan_is_the_oracle_tree(shim, n, leaf):
    P = plan(shim, n, leaf)
    assert P["rc"] == 0
    levels, stages = expected_merges(n, leaf)
    L = len(levels) - 1
    assert P["L"] == L == nd_dense.num_levels(n, leaf)
    assert [nd_dense.Box(l["x0"], l["y0"], l["a"], l["b"]) for l in P["leaves"]] == levels[L]
    assert len(P["stages"]) == 2 * L
    for s, (st, want) in enumerate(zip(P["stages"], stages)):
        assert st["orient"] == s % 2
        assert [(m["c1"], m["c2"], m["par"]) for m in st["merges"]] == want
        for m in st["merges"]:
            assert m["orient"] == st["orient"] and m["n"] == n
            check_merge(m, n)


@pytest.mark.parametrize("n,leaf", [(12, 4), (37, 5), (100, 16)])
def test_plan_offsets_chain_and_do_not_overlap(shim, n, leaf):
    P = plan(shim, n, leaf)
    where = {}  # box -> arena offset of its Schur complement
    blocks = []
    for l in P["leaves"]:
        box = nd_dense.Box(l["x0"], l["y0"], l["a"], l["b"])
        r = len(box.ring())
        where[box] = l["off"]
        blocks.append((l["off"], r * r))
    assert sum(b for _, b in blocks) == P["leaf_doubles"]
    for st in P["stages"]:
        ws, dig, ex = [], 0, 0
        for m in st["merges"]:
            assert m["s1"] == where[m["c1"]] and m["s2"] == where[m["c2"]]  # children from the stage before
            assert st["out_base"] <= m["out"] and m["out"] + m["rp"] ** 2 <= st["out_base"] + st["out_doubles"]
            blocks.append((m["out"], m["rp"] ** 2))
            ws.append((m["ws"], 2 * m["sp"] * (2 * m["sp"] + m["rp"])))
            assert m["doff"] == dig and m["doff"] % 2048 == 0 and m["eoff"] == ex
            dig += -(-m["rp"] // 128) * 128 * m["kpad"]
            ex += m["rp"]
        for m in st["merges"]:
            where[m["par"]] = m["out"]
        assert (st["dig_elems"], st["exp_elems"]) == (dig, ex)
        assert sum(b for _, b in ws) == st["ws_doubles"]
        ws.sort()
        assert all(a[0] + a[1] <= b[0] for a, b in zip(ws, ws[1:]))
        assert st["max_m"] == max(2 * m["sp"] for m in st["merges"])
        assert st["max_rp"] == max(m["rp"] for m in st["merges"])
    blocks.sort()
    assert blocks[0][0] == 0 and all(a[0] + a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
    assert blocks[-1][0] + blocks[-1][1] == P["arena"]
    (root,) = P["roots"]
    assert root["r"] == 4 * n - 4 and root["off"] == where[nd_dense.Box(0, 0, n, n)]


def test_plan_without_merges_and_bad_arguments(shim):
    P = plan(shim, 16, 16)  # the whole grid is one leaf
    assert P["rc"] == 0 and P["L"] == 0 and P["stages"] == [] and len(P["leaves"]) == 1
    assert P["roots"][0]["off"] == P["leaves"][0]["off"] == 0
    assert plan(shim, 1, 4)["rc"] == GM_EINVAL
    assert plan(shim, 12, 2)["rc"] == GM_EINVAL
    assert plan(shim, 7, 3)["rc"] == GM_EINVAL  # 7 -> 3, 4 -> 1, 2, 2, 2: a box without a ring
    assert plan(shim, 12, 3)["rc"] == 0 and plan(shim, 12, 3)["L"] == 2


def test_batch_plan_aligns_stages_from_the_root(shim):
    ns, leaves = [40, 12, 100], [5, 4, 16]
    coef = np.array([0, 1600, 1744], dtype=np.int64)
    c_ns = (ctypes.c_int * 3)(*ns)
    c_leaves = (ctypes.c_int * 3)(*leaves)
    B = parse(_call(shim.plan_dump_batch, 3, c_ns, c_leaves, coef.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    assert B["rc"] == 0
    singles = [plan(shim, n, lf) for n, lf in zip(ns, leaves)]
    Lmax = max(p["L"] for p in singles)
    assert B["L"] == Lmax and len(B["stages"]) == 2 * Lmax
    assert B["coef_total"] == max(int(c) + n * n for c, n in zip(coef, ns))
    for pi, (p, n) in enumerate(zip(singles, ns)):
        shift = 2 * (Lmax - p["L"])
        for s, st in enumerate(p["stages"]):
            mine = [m for m in B["stages"][shift + s]["merges"] if m["prob"] == pi]
            assert [(m["c1"], m["c2"], m["par"]) for m in mine] == [(m["c1"], m["c2"], m["par"]) for m in st["merges"]]
            for m in mine:
                check_merge(m, n, int(coef[pi]))
        for s in range(shift):  # a shallower problem has no merges in the finest stages
            assert all(m["prob"] != pi for m in B["stages"][s]["merges"])
        assert B["roots"][pi]["coef"] == coef[pi] and B["roots"][pi]["r"] == 4 * n - 4
    # every Schur complement block of the batch is distinct and inside the arena
    blocks = [(l["off"], (2 * l["a"] + 2 * l["b"] - 4) ** 2) for l in B["leaves"]]
    blocks += [(m["out"], m["rp"] ** 2) for st in B["stages"] for m in st["merges"]]
    blocks.sort()
    assert all(a[0] + a[1] <= b[0] for a, b in zip(blocks, blocks[1:]))
    assert blocks[-1][0] + blocks[-1][1] <= B["arena"]
