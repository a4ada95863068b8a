"""The body-load plan (csrc/loads_plan.cpp, Section 6.3) on the CPU: which leaves hold
body nodes, the load-map columns of every box (a leaf's in the caller's order, a merge's
first child's then second child's, as the oracle's build_loads), the load arena and the
widened interface systems, and the root's column order.

loads_plan.cpp and plan.cpp are compiled with g++ beside tests/load_plan_shim.cpp; the
CUDA headers serve for declarations only.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import nd_dense
from paper_1302_5995_gb300 import inputs

from test_plan_host import expected_merges
from test_server_host import _cuda_include

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GM_EINVAL = -1


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("no CUDA headers")
    out = str(tmp_path_factory.mktemp("loadplan") / "load_plan_shim.so")
    csrc = os.path.join(ROOT, "paper_1302_5995_gb300", "csrc")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", inc, "-o", out,
                           os.path.join(ROOT, "tests", "load_plan_shim.cpp"),
                           os.path.join(csrc, "loads_plan.cpp"), os.path.join(csrc, "plan.cpp")])
    lib = ctypes.CDLL(out)
    lib.load_plan_dump.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.c_int64]
    lib.load_plan_dump.restype = ctypes.c_int64
    return lib


def dump(shim, n, leaf, body):
    body = np.ascontiguousarray(np.asarray(body, dtype=np.int32))
    cap = 1 << 16
    while True:
        buf = np.zeros(cap, dtype=np.int64)
        got = shim.load_plan_dump(n, leaf, body.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), body.size,
                                  buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
        if got >= 0:
            break
        cap = -got
    it = iter(buf[:got].tolist())
    nxt = lambda k: [next(it) for _ in range(k)]
    rc, nbody, arena, root_l, leaf_ws, nleaves, nstages = nxt(7)
    P = dict(rc=rc, nbody=nbody, arena=arena, root_l=root_l, leaf_ws=leaf_ws, leaves=[], leaf_sys=[], stages=[])
    if rc:
        return P
    P["root_order"] = nxt(nbody)
    for _ in range(nleaves):
        d = dict(zip(["x0", "y0", "a", "b", "m", "col0", "ni", "sys", "lout"], nxt(9)))
        d["nodes"] = nxt(d["m"])
        P["leaves"].append(d)
    nsys = sum(1 for d in P["leaves"] if d["ni"] > 0)
    P["leaf_sys"] = [dict(zip(["off", "m", "ncol", "id"], nxt(4))) for _ in range(nsys)]
    for _ in range(nstages):
        nm, ws, maxc = nxt(3)
        merges = []
        for _ in range(nm):
            m = dict(zip(["m1", "m2", "l1", "l2", "lout", "ws", "soff", "sm", "sncol", "sid", "copy_ok"], nxt(11)))
            m["c1"], m["c2"], m["par"] = (nd_dense.Box(*nxt(4)) for _ in range(3))
            merges.append(m)
        P["stages"].append(dict(ws=ws, max_ncol=maxc, merges=merges))
    assert next(it, None) is None
    return P


def expected_columns(n, leaf, body):
    """Box -> caller positions of its load columns, by the oracle's conventions."""
    levels, stages = expected_merges(n, leaf)
    cols = {}
    for box in levels[-1]:
        cols[box] = [i for i, g in enumerate(body) if box.contains((g % n, g // n))]
    for st in stages:
        for (c1, c2, par) in st:
            cols[par] = cols[c1] + cols[c2]
    return cols


@pytest.mark.parametrize("n,leaf,count,seed", [(12, 4, 6, 1), (23, 4, 30, 2), (37, 5, 40, 3), (64, 16, 100, 4),
                                               (16, 16, 5, 5)])
def test_load_plan_columns_and_layout(shim, n, leaf, count, seed):
    body = [int(g) for g in inputs.body_nodes(n, count, seed)]
    # a few loads on the outer ring and on the root's interfaces as well
    for g in (0, n - 1, (n // 2) * n + 3, (n // 2 - 1) * n + n // 2):
        if g not in body:
            body.append(g)
    P = dump(shim, n, leaf, body)
    assert P["rc"] == 0 and P["nbody"] == len(body)
    want = expected_columns(n, leaf, body)
    ring = lambda bx: 2 * bx.a + 2 * bx.b - 4
    blocks = []
    # leaves with loads: their nodes in the caller's order, [A_ii | E_i] when they have an interior
    leaves_with = [bx for bx in nd_dense.quad_tree(n, leaf)[-1] if want[bx]]
    assert [nd_dense.Box(d["x0"], d["y0"], d["a"], d["b"]) for d in P["leaves"]] == leaves_with
    sys_iter = iter(P["leaf_sys"])
    wacc = 0
    for d in P["leaves"]:
        bx = nd_dense.Box(d["x0"], d["y0"], d["a"], d["b"])
        assert d["nodes"] == [body[i] for i in want[bx]] and d["m"] == len(want[bx])
        assert d["ni"] == max(bx.a - 2, 0) * max(bx.b - 2, 0)
        if d["ni"]:
            s = next(sys_iter)
            assert (s["off"], s["m"], s["ncol"]) == (wacc, d["ni"], d["ni"] + d["m"]) and d["sys"] == wacc
            wacc += d["ni"] * (d["ni"] + d["m"])
        else:
            assert d["sys"] == -1
        blocks.append((d["lout"], ring(bx) * d["m"]))
    assert P["leaf_ws"] == wacc
    # merges: widened systems in their own layout, loads of child 1 then child 2
    off = {nd_dense.Box(d["x0"], d["y0"], d["a"], d["b"]): d["lout"] for d in P["leaves"]}
    for st in P["stages"]:
        w = 0
        for k, m in enumerate(st["merges"]):
            assert m["copy_ok"] == 1
            assert (m["m1"], m["m2"]) == (len(want[m["c1"]]), len(want[m["c2"]]))
            assert m["l1"] == off.get(m["c1"], -1) and m["l2"] == off.get(m["c2"], -1)
            sp = len(nd_dense.partition_we(m["c1"], m["c2"], m["par"])[1])
            ncol = 2 * sp + ring(m["par"]) + m["m1"] + m["m2"]
            assert (m["ws"], m["soff"], m["sm"], m["sncol"], m["sid"]) == (w, w, 2 * sp, ncol, k)
            w += 2 * sp * ncol
            if m["m1"] + m["m2"]:
                blocks.append((m["lout"], ring(m["par"]) * (m["m1"] + m["m2"])))
                off[m["par"]] = m["lout"]
            else:
                assert m["lout"] == -1
        assert st["ws"] == w
    blocks.sort()
    assert blocks[0][0] == 0 and all(a[0] + a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
    assert blocks[-1][0] + blocks[-1][1] == P["arena"]
    root = nd_dense.Box(0, 0, n, n)
    assert P["root_order"] == want[root] and sorted(P["root_order"]) == list(range(len(body)))
    assert P["root_l"] == off[root]


def test_load_plan_rejects_bad_lists(shim):
    assert dump(shim, 12, 4, [])["rc"] == GM_EINVAL
    assert dump(shim, 12, 4, [3, 3])["rc"] == GM_EINVAL
    assert dump(shim, 12, 4, [144])["rc"] == GM_EINVAL
    assert dump(shim, 12, 4, [-1])["rc"] == GM_EINVAL
