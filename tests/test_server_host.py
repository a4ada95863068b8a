"""The serving runtime's policy (csrc/server.cpp) on the CPU: continuous batching of the
requests pending per operator, the unbatched baseline, admission against the memory
budget with least-recently-used eviction that never takes an operator being served,
requests for an evicted operator, solve errors, statistics, argument errors.

server.cpp is compiled with g++ beside tests/server_fakes.cpp, whose CUDA runtime calls
act on host memory and whose gm_solve / gm_info / gm_free act on fake operators that
record every call (dudn = 1000 * tag + 2 g).  No GPU is involved.
"""
import ctypes
import os
import shutil
import subprocess
import time

import numpy as np
import pytest

import paper_1302_5995_gb300 as gm
from paper_1302_5995_gb300 import GM_EINVAL, GM_ENOMEM, GM_ECUDA, ServerStats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    nvcc = shutil.which("nvcc")
    for d in ([os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")] if nvcc else []) + \
             ["/usr/local/cuda/include"]:
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("no CUDA headers")
    out = str(tmp_path_factory.mktemp("server") / "server_fake.so")
    # -Bsymbolic: the server binds to these fakes even when a real CUDA runtime or the
    # library itself is already loaded into the process
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-pthread", "-Wl,-Bsymbolic", "-I", inc, "-o", out,
                           os.path.join(ROOT, "tests", "server_fakes.cpp"),
                           os.path.join(ROOT, "paper_1302_5995_gb300", "csrc", "server.cpp")])
    L = ctypes.CDLL(out)
    vp, ll = ctypes.c_void_p, ctypes.c_longlong
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "gm_server_create": (ctypes.c_int, [ll, ctypes.c_int, ctypes.POINTER(vp)]),
        "gm_server_add": (ctypes.c_int, [vp, vp, ip]),
        "gm_server_submit": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.POINTER(ll)]),
        "gm_server_wait": (ctypes.c_int, [vp, ll]),
        "gm_server_submit_build": (ctypes.c_int, [vp, vp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                  ip, ctypes.POINTER(ll)]),
        "gm_server_poll": (ctypes.c_int, [vp, ll, ip]),
        "gm_server_set_callback": (ctypes.c_int, [vp, vp, vp]),
        "gm_server_sync": (ctypes.c_int, [vp]),
        "gm_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
        "gm_server_reset_stats": (ctypes.c_int, [vp]),
        "gm_server_destroy": (None, [vp]),
        "fake_op": (vp, [ctypes.c_int, ll, ctypes.c_int, ctypes.c_int]),
        "fake_reset": (None, []),
        "fake_gate": (None, [ctypes.c_int]),
        "fake_wait_blocked": (ctypes.c_int, [ctypes.c_int]),
        "fake_calls": (ctypes.c_int, [ip, ip, ctypes.c_int]),
        "fake_freed": (ctypes.c_int, [ip, ctypes.c_int]),
        "gm_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype, fn.argtypes = res, args
    return L


class Server:
    """A server over the fakes; every test gets a fresh one and the gate opened at exit."""

    def __init__(self, L, budget=1 << 40, batching=1):
        self.L = L
        L.fake_reset()
        h = ctypes.c_void_p()
        assert L.gm_server_create(budget, batching, ctypes.byref(h)) == 0
        self.h = h
        self.keep = []
        self.refused = []

    def add(self, n, nbytes, tag, solve_rc=0):
        op = ctypes.c_int()
        h = self.L.fake_op(n, nbytes, tag, solve_rc)
        rc = self.L.gm_server_add(self.h, h, ctypes.byref(op))
        if rc:
            self.refused.append(h)  # the caller keeps a refused handle
        return rc, op.value

    def submit(self, op, n, batch, seed):
        g = np.random.default_rng(seed).standard_normal((batch, 4 * n))
        out = np.zeros_like(g)
        self.keep.append((g, out))
        rid = ctypes.c_longlong()
        dp = ctypes.POINTER(ctypes.c_double)
        rc = self.L.gm_server_submit(self.h, op, g.ctypes.data_as(dp), out.ctypes.data_as(dp), batch,
                                     ctypes.byref(rid))
        return rc, rid.value, g, out

    def submit_build(self, n):
        coef = np.zeros(n * n)  # read only by a real build
        self.keep.append(coef)
        dp = ctypes.POINTER(ctypes.c_double)
        oid, rid = ctypes.c_int(), ctypes.c_longlong()
        rc = self.L.gm_server_submit_build(self.h, None, coef.ctypes.data_as(dp), coef.ctypes.data_as(dp),
                                           coef.ctypes.data_as(dp), n, 4, 0.0, ctypes.byref(oid), ctypes.byref(rid))
        return rc, oid.value, rid.value

    def poll(self, rid):
        done = ctypes.c_int()
        rc = self.L.gm_server_poll(self.h, rid, ctypes.byref(done))
        return done.value, rc

    def calls(self):
        tags, batches = (ctypes.c_int * 64)(), (ctypes.c_int * 64)()
        k = self.L.fake_calls(tags, batches, 64)
        return list(zip(tags[:k], batches[:k]))

    def freed(self):
        tags = (ctypes.c_int * 64)()
        return list(tags[:self.L.fake_freed(tags, 64)])

    def stats(self):
        st = ServerStats()
        assert self.L.gm_server_stats(self.h, ctypes.byref(st)) == 0
        return st

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.L.fake_gate(0)
        self.L.gm_server_destroy(self.h)
        for h in self.refused:
            self.L.gm_free(h)


def _queue_behind_a_held_solve(s, first_op, n):
    """Hold the worker inside the first operator's solve, so later submissions queue."""
    s.L.fake_gate(1)
    rc, r0, g0, out0 = s.submit(first_op, n, 1, 0)
    assert rc == 0 and s.L.fake_wait_blocked(5000) == 1
    return r0, g0, out0


def test_continuous_batching_groups_pending_requests_per_operator(lib):
    with Server(lib) as s:
        _, A = s.add(3, 10, 1)
        _, B = s.add(4, 10, 2)
        r0, g0, out0 = _queue_behind_a_held_solve(s, A, 3)
        reqs = [s.submit(op, n, k, 10 + i) for i, (op, n, k) in
                enumerate([(A, 3, 2), (B, 4, 1), (A, 3, 3), (B, 4, 2)])]
        s.L.fake_gate(0)
        assert s.L.gm_server_sync(s.h) == 0
        # one grouped solve over every operator's concatenated vectors, operators in
        # order of first arrival
        assert s.calls() == [(1, 1), (1, 5), (2, 3)]
        for (rc, rid, g, out), tag in zip([(0, r0, g0, out0)] + reqs, [1, 1, 2, 1, 2]):
            assert rc == 0 and s.L.gm_server_wait(s.h, rid) == 0
            np.testing.assert_array_equal(out, 1000.0 * tag + 2.0 * g)  # each its own vectors
        st = s.stats()
        assert (st.requests, st.vectors, st.solves, st.evictions) == (5, 9, 2, 0)  # two grouped solves
        assert 0 < st.p50_ms <= st.p99_ms and st.vectors_per_s > 0


def test_unbatched_baseline_solves_each_request(lib):
    with Server(lib, batching=0) as s:
        _, A = s.add(3, 10, 1)
        _, B = s.add(4, 10, 2)
        _queue_behind_a_held_solve(s, A, 3)
        for i, (op, n, k) in enumerate([(A, 3, 2), (B, 4, 1), (A, 3, 3)]):
            assert s.submit(op, n, k, i)[0] == 0
        s.L.fake_gate(0)
        s.L.gm_server_sync(s.h)
        assert s.calls() == [(1, 1), (1, 2), (1, 3), (2, 1)]


def test_budget_admission_evicts_least_recently_used(lib):
    with Server(lib, budget=100) as s:
        _, A = s.add(3, 40, 1)
        _, B = s.add(3, 40, 2)
        rc, rid, _, _ = s.submit(A, 3, 1, 0)  # A is now the more recently used
        assert s.L.gm_server_wait(s.h, rid) == 0
        rc, C = s.add(3, 40, 3)
        assert rc == 0 and s.freed() == [2]  # B was the least recently used
        st = s.stats()
        assert (st.resident_ops, st.resident_bytes, st.evictions) == (2, 80, 1)
        assert s.add(3, 200, 4)[0] == GM_ENOMEM  # larger than the whole budget
        assert s.freed() == [2]  # nothing evicted for it, and it stays the caller's
        assert s.submit(B, 3, 1, 1)[0] == GM_EINVAL  # an evicted operator is unknown


def test_operator_being_served_is_never_evicted(lib):
    with Server(lib, budget=100) as s:
        _, A = s.add(3, 60, 1)
        r0, _, _ = _queue_behind_a_held_solve(s, A, 3)
        assert s.add(3, 60, 2)[0] == GM_ENOMEM  # only A could make room, and it is busy
        s.L.fake_gate(0)
        assert s.L.gm_server_wait(s.h, r0) == 0
        s.L.gm_server_sync(s.h)
        rc, _ = s.add(3, 60, 3)
        assert rc == 0 and 1 in s.freed()


def test_request_for_an_operator_evicted_while_queued_fails(lib):
    with Server(lib, budget=100) as s:
        _, A = s.add(3, 50, 1)
        _, B = s.add(3, 50, 2)
        r0, _, _ = _queue_behind_a_held_solve(s, A, 3)
        rc, r1, _, out1 = s.submit(B, 3, 1, 5)
        assert rc == 0
        assert s.add(3, 50, 3)[0] == 0  # A is busy, so B goes
        s.L.fake_gate(0)
        assert s.L.gm_server_wait(s.h, r0) == 0
        assert s.L.gm_server_wait(s.h, r1) == GM_EINVAL
        assert not out1.any()


def test_solve_error_reaches_the_request(lib):
    with Server(lib) as s:
        _, A = s.add(3, 10, 1, solve_rc=GM_ECUDA)
        rc, rid, _, _ = s.submit(A, 3, 2, 0)
        assert rc == 0 and s.L.gm_server_wait(s.h, rid) == GM_ECUDA
        assert s.stats().requests == 0  # only completed requests count
        assert s.L.gm_server_reset_stats(s.h) == 0 and s.stats().solves == 0


def test_argument_errors_and_destroy(lib):
    h = ctypes.c_void_p()
    assert lib.gm_server_create(0, 1, ctypes.byref(h)) == GM_EINVAL
    with Server(lib) as s:
        _, A = s.add(3, 10, 1)
        assert s.submit(A, 3, 1, 0)[0] == 0
        assert s.L.gm_server_wait(s.h, 0) == GM_EINVAL and s.L.gm_server_wait(s.h, 99) == GM_EINVAL
        dp = ctypes.POINTER(ctypes.c_double)
        rid = ctypes.c_longlong()
        x = np.zeros(12)
        assert lib.gm_server_submit(s.h, A, x.ctypes.data_as(dp), x.ctypes.data_as(dp), 0,
                                    ctypes.byref(rid)) == GM_EINVAL
        assert lib.gm_server_sync(None) == GM_EINVAL
        s.add(3, 10, 2)
    assert sorted(s.freed()) == [1, 2]  # destroy frees every resident operator
    lib.gm_server_destroy(None)


def test_build_request_runs_beside_solves_and_before_the_solves_queued_for_it(lib):
    with Server(lib) as s:
        _, A = s.add(3, 10, 1)
        _queue_behind_a_held_solve(s, A, 3)
        rc, X, rb = s.submit_build(5)
        assert rc == 0
        rc, rs, g, out = s.submit(X, 5, 2, 7)  # the operator may not exist yet: it is being built
        assert rc == 0
        # the build worker does not wait for the solve worker, which is still held
        assert s.L.gm_server_wait(s.h, rb) == 0
        assert s.poll(rs) == (0, 0)
        s.L.fake_gate(0)
        assert s.L.gm_server_wait(s.h, rs) == 0 and s.L.gm_server_wait(s.h, rb) == 0
        assert s.poll(rb) == (1, 0)
        assert s.calls() == [(1, 1), (5, -1), (5, 2)]  # the build, then its solve
        np.testing.assert_array_equal(out, 1000.0 * 5 + 2.0 * g)
        st = s.stats()
        assert st.resident_ops == 2 and st.resident_bytes == 10 + 50


def test_failed_build_fails_its_queued_solves(lib):
    with Server(lib) as s:
        _, A = s.add(3, 10, 1)
        _queue_behind_a_held_solve(s, A, 3)
        rc, X, rb = s.submit_build(13)  # the fake reports a singular problem for n = 13
        rc, rs, _, out = s.submit(X, 13, 1, 8)
        s.L.fake_gate(0)
        assert s.L.gm_server_wait(s.h, rb) == gm.GM_ESINGULAR
        assert s.L.gm_server_wait(s.h, rs) == GM_EINVAL and not out.any()
        assert s.submit(X, 13, 1, 9)[0] == GM_EINVAL  # the id never became an operator


def test_build_requests_are_admitted_under_the_budget(lib):
    with Server(lib, budget=100) as s:
        _, A = s.add(3, 60, 1)
        rc, X, rb = s.submit_build(20)  # 200 bytes: more than the whole budget
        assert rc == 0 and s.L.gm_server_wait(s.h, rb) == GM_ENOMEM
        rc, Y, rb = s.submit_build(5)  # 50 bytes: the least recently used operator makes room
        assert s.L.gm_server_wait(s.h, rb) == 0
        assert s.freed() == [20, 1]  # the refused build's operator, then the evicted one
        st = s.stats()
        assert st.resident_ops == 1 and st.resident_bytes == 50 and st.evictions == 1


def test_poll_and_build_argument_errors(lib):
    with Server(lib) as s:
        done = ctypes.c_int()
        assert lib.gm_server_poll(s.h, 42, ctypes.byref(done)) == GM_EINVAL
        assert lib.gm_server_poll(None, 1, ctypes.byref(done)) == GM_EINVAL
        oid, rid = ctypes.c_int(), ctypes.c_longlong()
        assert lib.gm_server_submit_build(s.h, None, None, None, None, 8, 4, 0.0, ctypes.byref(oid),
                                          ctypes.byref(rid)) == GM_EINVAL


CALLBACK = ctypes.CFUNCTYPE(None, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p)


def test_completion_callback_sees_every_request(lib):
    with Server(lib) as s:
        seen = []
        polled = []

        def on_done(rid, rc, user):
            seen.append((rid, rc))
            polled.append(s.poll(rid))  # calling back into the server from the callback

        cb = CALLBACK(on_done)
        assert lib.gm_server_set_callback(s.h, ctypes.cast(cb, ctypes.c_void_p), None) == 0
        _, A = s.add(3, 10, 1)
        _, B = s.add(3, 10, 2, solve_rc=GM_ECUDA)
        rids = [s.submit(A, 3, 1, 1)[1], s.submit(B, 3, 2, 2)[1], s.submit(A, 3, 3, 3)[1]]
        _, _, rb = s.submit_build(5)
        for r in rids + [rb]:
            s.L.gm_server_wait(s.h, r)
        s.L.gm_server_sync(s.h)
        for _ in range(200):  # callbacks run just after the results become visible
            if len(seen) == 4:
                break
            time.sleep(0.01)
        assert sorted(seen) == sorted([(rids[0], 0), (rids[1], GM_ECUDA), (rids[2], 0), (rb, 0)])
        assert all(done == 1 for done, _ in polled)
        assert lib.gm_server_set_callback(s.h, None, None) == 0
        assert lib.gm_server_set_callback(None, None, None) == GM_EINVAL
