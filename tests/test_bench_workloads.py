"""bench.py's non-headline workloads (problemset, bodyloads) run end to end on the CPU
with the library replaced by stand-in operators and the CUDA calls by no-ops, so that
their bookkeeping (timing, error measures, JSON line) is exercised before a GPU runs
them.  The numbers here are meaningless; the structure is what is checked."""
import json
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
import paper_1302_5995_gb300 as gm
from paper_1302_5995_gb300 import build_ext


class FakeOp:
    def __init__(self, n, scale=2.0, nbody=0, hbs=False):
        self.n, self.scale, self.nbody, self.hbs = n, scale, nbody, hbs

    def solve(self, G, out=None, stream=None):
        return G * self.scale

    def solve_loads(self, g, f, out=None, stream=None):
        return g * self.scale

    def load_operator(self):
        h = 1.0 / (self.n + 1)
        return np.full((4 * self.n, self.nbody), -h / (4 * self.n))  # columns sum to -h

    def info(self):
        return {"pivot_fallback": 0, "hbs_operator_bytes": 1000 * self.n if self.hbs else 0,
                "hbs_max_rank": 20 if self.hbs else 0}

    def free(self):
        pass


@pytest.fixture
def fake_gpu(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(build_ext, "build", lambda *a, **k: None)

    def build(b, c, d, n, leaf, tol=0.0, precision=gm.PREC_FP64, **k):
        return FakeOp(n, 2.0 * (1 + 1e-12) if precision == gm.PREC_MIXED else 2.0, hbs=tol > 0)

    def build_network(sx, sy, n, leaf, body=None, tol=0.0, **k):
        return FakeOp(n, nbody=0 if body is None else len(body), hbs=tol > 0)

    monkeypatch.setattr(gm, "build", build)
    monkeypatch.setattr(gm, "build_network", build_network)


def _line(capsys):
    out = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(out) == 1
    return json.loads(out[0])


def test_problemset_workload_line(fake_gpu, capsys):
    bench.run_problemset(types.SimpleNamespace(steps=1))
    line = _line(capsys)
    assert line["workload"] == "problemset" and line["n"] == 512
    res = line["results"]
    assert set(res) == set(bench_problems())
    for name, row in res.items():
        assert row["fp64_build_ms"] >= 0 and "hbs_M_over_n" in row
        if not name.startswith("random"):
            assert row["mixed_e1_vs_fp64"] == pytest.approx(1e-12, rel=1e-3)
            assert row["mixed_fell_back_to_fp64"] is False


def bench_problems():
    from paper_1302_5995_gb300 import inputs
    return list(inputs.PAPER_PROBLEMS) + ["random1", "random2"]


def test_bodyloads_workload_line(fake_gpu, capsys):
    bench.run_bodyloads(types.SimpleNamespace(steps=1))
    line = _line(capsys)
    assert line["workload"] == "bodyloads" and line["precision"] == "fp64"
    assert set(line["results"]) == {"10", "100", "1000"}
    for row in line["results"].values():
        assert row["build_ms"] >= 0 and row["solve_ms"] >= 0
        assert row["conservation_err"] < 1e-12
