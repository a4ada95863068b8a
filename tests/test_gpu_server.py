"""Serving runtime: results of batched requests equal the direct solve, LRU admission
within the memory budget, the unbatched baseline mode, and submissions from several
threads."""
import threading

import numpy as np
import pytest

from oracle import nd_dense
from paper_1302_5995_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    return gm


def problems():
    out = []
    for i, (n, leaf) in enumerate(((48, 8), (64, 16), (40, 8))):
        b, c, d = inputs.convection_fields(n, seeds=(20 + i, 30 + i, 40 + i))
        out.append((b, c, d, n, leaf))
    return out


def rel_vec(V, Vo):
    return (np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max()


@pytest.mark.parametrize("batching", [True, False])
def test_requests_match_direct_solves(gm, batching):
    probs = problems()
    Ts = [nd_dense.build(*p).T for p in probs]
    srv = gm.Server(1 << 30, batching=batching)
    ids = [srv.add(gm.build(*p)) for p in probs]
    rng = np.random.default_rng(5)
    reqs = []
    for q in range(60):
        k = int(rng.integers(0, 3))
        n = probs[k][3]
        B = int(rng.integers(1, 9))
        g = np.ascontiguousarray(rng.standard_normal((B, 4 * n)))  # vector j contiguous
        out = np.zeros_like(g)
        reqs.append((srv.submit(ids[k], g, out, B), k, g, out))
    for rid, k, g, out in reqs:
        assert srv.wait(rid) == 0
        assert rel_vec(out.T, Ts[k] @ g.T) < 1e-10
    st = srv.stats()
    assert st["requests"] == 60 and st["vectors"] == sum(r[2].shape[0] for r in reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["vectors_per_s"] > 0
    if batching:
        assert st["solves"] <= 60
    else:
        assert st["solves"] >= 1
    srv.close()


def test_lru_admission_and_eviction(gm):
    probs = problems()
    ops = [gm.build(*p) for p in probs]
    sizes = [op.info()["resident_bytes"] for op in ops]
    srv = gm.Server(sizes[0] + sizes[1] + 1)
    a = srv.add(ops[0])
    b = srv.add(ops[1])
    # touch a, so b is the least recently used one
    g = np.ones((1, 4 * probs[0][3]))
    out = np.zeros_like(g)
    assert srv.wait(srv.submit(a, g, out, 1)) == 0
    c = srv.add(ops[2])
    st = srv.stats()
    assert st["evictions"] == 1 and st["resident_ops"] == 2
    with pytest.raises(gm.GmError):
        srv.submit(b, np.ones((1, 4 * probs[1][3])), np.zeros((1, 4 * probs[1][3])), 1)
    g3 = np.ones((2, 4 * probs[2][3]))
    out3 = np.zeros_like(g3)
    assert srv.wait(srv.submit(c, g3, out3, 2)) == 0
    # an operator larger than the whole budget is refused
    big = gm.build(*probs[1])
    small = gm.Server(1024)
    with pytest.raises(gm.GmError):
        small.add(big)
    small.close()
    srv.close()


def test_submissions_from_threads(gm):
    probs = problems()[:2]
    Ts = [nd_dense.build(*p).T for p in probs]
    srv = gm.Server(1 << 30)
    ids = [srv.add(gm.build(*p)) for p in probs]
    errs = []

    def client(seed):
        rng = np.random.default_rng(seed)
        mine = []
        for _ in range(20):
            k = int(rng.integers(0, 2))
            n = probs[k][3]
            g = np.ascontiguousarray(rng.standard_normal((3, 4 * n)))
            out = np.zeros_like(g)
            mine.append((srv.submit(ids[k], g, out, 3), k, g, out))
        for rid, k, g, out in mine:
            if srv.wait(rid) != 0 or rel_vec(out.T, Ts[k] @ g.T) > 1e-10:
                errs.append((seed, rid))

    th = [threading.Thread(target=client, args=(s,)) for s in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs
    assert srv.stats()["requests"] == 80
    srv.close()


def test_device_buffers(gm):
    import torch
    p = problems()[0]
    T = nd_dense.build(*p).T
    srv = gm.Server(1 << 30)
    oid = srv.add(gm.build(*p))
    n = p[3]
    g = torch.randn(5, 4 * n, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(g)
    torch.cuda.synchronize()
    assert srv.wait(srv.submit(oid, g, out, 5)) == 0
    assert rel_vec(out.cpu().numpy().T, T @ g.cpu().numpy().T) < 1e-10
    srv.close()


def test_solve_many_equals_each_operator_alone(gm):
    """One grouped call over FP64, mixed-precision and HBS operators of different sizes:
    every result equals the operator's own solve bit for bit (the grouped launches run
    the same tiles in the same order)."""
    import torch
    fp = [gm.build(*p) for p in problems()]
    mx = []
    for i, (n, leaf) in enumerate(((128, 16), (96, 12))):
        b, c, d = inputs.convection_fields(n, seeds=(50 + i, 60 + i, 70 + i))
        mx.append(gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED))
    b, c, d = inputs.convection_fields(64, seeds=(80, 81, 82))
    hb = gm.build(b, c, d, 64, 8, tol=1e-9, hbs_leaf=32)
    ops = fp + mx + [hb]
    gen = torch.Generator(device="cuda").manual_seed(3)
    gs = [torch.randn(3 + 5 * i, 4 * op.n, dtype=torch.float64, device="cuda", generator=gen)
          for i, op in enumerate(ops)]
    outs = [torch.zeros_like(g) for g in gs]
    gm.solve_many(ops, gs, outs)
    for op, g, o in zip(ops, gs, outs):
        lone = torch.zeros_like(g)
        op.solve(g, out=lone)
        torch.cuda.synchronize()
        assert torch.equal(o, lone)


def test_solves_complete_while_a_build_is_in_flight(gm):
    """A long build (1024 x 1024 Helmholtz, FP64) runs on the server's build worker while
    solve requests keep arriving: several complete before the build does, and each equals
    the lone solve of its operator within 1e-10."""
    import time
    import torch
    probs = problems()
    lone = [gm.build(*p) for p in probs]
    srv = gm.Server(1 << 36)
    ids = [srv.add(gm.build(*p)) for p in probs]
    cfg = inputs.config3(1024, 16)
    dev = [torch.from_numpy(cfg[k]).cuda() for k in ("b", "c", "d")]
    torch.cuda.synchronize()
    done_at = {}
    srv.set_callback(lambda rid, rc: done_at.setdefault(rid, time.perf_counter()))
    oid, rb = srv.submit_build(*dev, 1024, 16)
    rng = np.random.default_rng(11)
    reqs = []
    t_stop = time.perf_counter() + 20.0
    while not srv.poll(rb)[0] and time.perf_counter() < t_stop:
        k = int(rng.integers(0, 3))
        n = probs[k][3]
        g = np.ascontiguousarray(rng.standard_normal((4, 4 * n)))
        out = np.zeros_like(g)
        reqs.append((srv.submit(ids[k], g, out, 4), k, g, out))
        time.sleep(0.002)
    srv.sync()
    assert srv.wait(rb) == 0
    before = [r for r in reqs if done_at[r[0]] < done_at[rb]]
    assert len(before) >= 3, (len(reqs), len(before))
    for rid, k, g, out in reqs:
        assert srv.wait(rid) == 0
        ref = lone[k].solve(g)
        assert rel_vec(out.T, ref.T) < 1e-10
    srv.set_callback(None)
    srv.close()
