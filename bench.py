"""Benchmark: build the DtN operator and solve a batch of Dirichlet vectors.

Workload (one step): the 512 x 512 convection-diffusion-reaction problem (b, c, d smooth
random Fourier fields, seeds 1-3), leaf boxes 16 x 16, then the solve of 256 Gaussian
boundary vectors (seed 4).  Metric: build gridpoints/s (n^2 / step time), with solve
vectors/s, error against the FP64 oracle and p50/p99 step latency alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gm|reference]
                    [--precision fp64|mixed] [--workload build|serving|problemset|bodyloads]

N > 1 runs under torchrun as independent replicas (one problem per GPU, no collective).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build gridpoints/s and DtN solve vectors/s (p50/p99 latency) at stated rel. err vs FP64"
UNIT = "gridpoints/s"
N_GRID, LEAF, NVEC = 512, 16, 256
WORKLOAD = ("convection-diffusion-reaction, b,c,d = 8-mode Fourier fields (seeds 1-3), 512x512 grid "
            "(N=262144), leaf 16x16, build + solve of 256 Gaussian boundary vectors (seed 4)")
# Peaks.  FP64 and FP32 pipes from unit counts and the maximum SM clock:
#   FP64: 152 SMs x 4 flop/clk/SM (2 DFMA) x 2070 MHz = 1.259 TFLOP/s
#   FP32: 152 SMs x 256 flop/clk/SM (128 FFMA) x 2070 MHz = 80.5 TFLOP/s
# Split products: the measured bf16 dense peak divided by the digit-pair products one
# algorithmic multiply-add costs (S(S+1)/2 for S digits per operand).
SMS, SM_MAX_MHZ = 152, 2070.0
FP64_PEAK_TFLOPS = SMS * 4 * SM_MAX_MHZ * 1e6 / 1e12
FP32_PEAK_TFLOPS = SMS * 256 * SM_MAX_MHZ * 1e6 / 1e12
DF32_OPS = 18
SPLIT_DIGITS = 6


def bf16_peak_tflops():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


_LIVE_PEAKS = {}


def live_peaks():
    """FP64 and FP32 (no TF32) dense GEMM rates of this GPU, measured now with cuBLAS
    through torch.matmul (4096^3, best of 5, CUDA events): the denominators of the FP64 /
    FP32 families' roofline fractions ("measured"), beside the unit-count peaks."""
    if _LIVE_PEAKS:
        return _LIVE_PEAKS
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        n = 4096
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        best = float("inf")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(6):
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = prev
    _LIVE_PEAKS.update(out)
    return out


def family_roofline(precision, fam):
    """(bound, peak TFLOP/s, source) of a kernel family of the timed operator build."""
    if precision == "fp64":
        pk = live_peaks()["fp64"]
        return "alu", pk, (f"FP64 DGEMM measured in this run (cuBLAS, 4096^3): {pk:.3f} TFLOP/s; unit-count "
                           f"peak {FP64_PEAK_TFLOPS:.3f} (152 SMs x 4 flop/clk x 2070 MHz)")
    if fam == "leaf":  # double-float arithmetic: 18 FP32 operations per multiply-add
        pk = live_peaks()["fp32"]
        return "alu", pk / DF32_OPS, (f"FP32 SGEMM measured in this run ({pk:.1f} TFLOP/s, no TF32) / {DF32_OPS} FP32 "
                                      "operations per double-float multiply-add (product 7, sum 11)")
    if fam == "panel":
        pk = live_peaks()["fp32"]
        return "alu", pk, f"FP32 SGEMM measured in this run ({pk:.1f} TFLOP/s, no TF32)"
    bf, src = bf16_peak_tflops()
    pairs = SPLIT_DIGITS * (SPLIT_DIGITS + 1) // 2
    return "tensor", bf / pairs, (f"bf16 dense peak ({src} {bf:.1f} TFLOP/s) / {pairs} digit-pair products "
                                  f"per algorithmic multiply-add ({SPLIT_DIGITS} digits)")
# DRAM traffic of the dominant kernel from an ncu capture (profiles/), per launch, with the
# source digest it was taken at; reported as null once the kernel source changes.
# gj_update: k_blk_update_tp + k_blk_update, one timed step's 158 launches
# (profiles/launches_convdiff512_mixed.md).
TRAFFIC = {"gj_update": (19947829.5, "fcbb31c29808")}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t, world, device=None):
    """The step time the job reports: the slowest rank's (all-reduce MAX); ranks are
    independent replicas, so this is the only collective of the benchmark."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(units_per_rank, t_ms, world):
    """Units all ranks processed (weak scaling: the same workload per rank) per second."""
    return world * units_per_rank / (t_ms * 1e-3)


# The sources a kernel family's code comes from (its translation unit and the headers it
# includes); a traffic figure stays valid while these are unchanged.
FAMILY_SOURCES = {"gj_update": ("blocked.cu", "blocked.h", "mixed_dev.cuh", "gm_internal.h", "kernels.h")}


def source_digest(family=None):
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1302_5995_gb300", "csrc")
    files = FAMILY_SOURCES.get(family) or sorted(os.listdir(csrc))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", self.gpu], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        loaded = [x for x in sm if smax and x > 0.3 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def make_inputs():
    import numpy as np
    from paper_1302_5995_gb300 import inputs
    cfg = inputs.config2(N_GRID, NVEC)
    Gv = np.ascontiguousarray(cfg["G"].T)  # 256 vectors, each contiguous
    return cfg, Gv


def cpu_oracle_step(cfg):
    """One step of the oracle: the paper's dense nested dissection in FP64 + the solve."""
    from oracle import nd_dense
    t0 = time.perf_counter()
    T = nd_dense.build(cfg["b"], cfg["c"], cfg["d"], N_GRID, LEAF).T
    V = nd_dense.solve(T, cfg["G"])
    return time.perf_counter() - t0, T, V


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg, _ = make_inputs()
    cores = os.cpu_count()
    for _ in range(args.warmup):
        cpu_oracle_step(cfg)
    ts = [cpu_oracle_step(cfg)[0] for _ in range(args.steps)]
    t = statistics.mean(ts)
    value = N_GRID * N_GRID / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_GRID, "leaf": LEAF, "nvec": NVEC, "precision": "fp64"},
        "solve_vectors_per_s": None,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "full workload per step: numpy/LAPACK dense nested dissection "
                                   "(oracle O2) + T @ G, default BLAS threading on all host cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gm(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1302_5995_gb300 import build_ext
    build_ext.build()
    import paper_1302_5995_gb300 as gm

    prec = gm.PREC_MIXED if args.precision == "mixed" else gm.PREC_FP64
    extra = dict(split_digits=SPLIT_DIGITS) if args.precision == "mixed" else {}
    cfg, Gv = make_inputs()
    n = N_GRID
    dev = torch.device("cuda", local)
    b, c, d = (torch.from_numpy(cfg[k]).to(dev) for k in "bcd")
    G = torch.from_numpy(Gv).to(dev)
    V = torch.empty_like(G)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > L2

    if args.graph:
        extra["graph"] = True
    if args.autotune:
        extra["autotune"] = True

    def step(timing):
        kw = dict(extra)
        if timing:  # an instrumented build is neither recorded nor replayed
            kw.pop("graph", None)
        op = gm.build(b, c, d, n, LEAF, precision=prec, stream=stream, timing=timing, **kw)
        op.solve(G, out=V, stream=stream)
        return op

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False).free()
    barrier()
    # one instrumented step (every launch bracketed by events): the per-family breakdown,
    # and which family dominates
    flush.fill_(1.0)
    barrier()
    op = step(True)
    torch.cuda.synchronize()
    inf = op.info()
    brk_ms = dict(inf["kernel_ms"])
    brk_fl = dict(inf["kernel_flops"])
    op.free()
    dom = max(brk_ms, key=lambda f: brk_ms[f])
    # timed region: events around every step; only the dominant family's launches carry
    # their own event pairs (instrumenting all ~1700 launches would slow the step)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    step_ms, build_ms, solve_ms, launches = [], [], [], 0
    dom_ms, dom_fl, dom_n = 0.0, 0.0, 0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        ev[0].record(stream)
        op = gm.build(b, c, d, n, LEAF, precision=prec, stream=stream, timing=False if args.graph else [dom],
                      **extra)
        ev[1].record(stream)
        op.solve(G, out=V, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev[0].elapsed_time(ev[2]))
        build_ms.append(ev[0].elapsed_time(ev[1]))
        solve_ms.append(ev[1].elapsed_time(ev[2]))
        inf = op.info()
        launches += inf["launches"] + 1
        if not args.graph:
            dom_ms += inf["kernel_ms"][dom]
            dom_fl += inf["kernel_flops"][dom]
            dom_n += inf["kernel_launches"][dom]
        op.free()
    if args.graph:  # a replayed build has no per-family events: the instrumented step's figures
        dom_ms, dom_fl, dom_n = brk_ms[dom] * args.steps, brk_fl[dom] * args.steps, inf["kernel_launches"][dom] * args.steps
    barrier()
    clk = clocks.stop()
    t_step = max_over_ranks(statistics.mean(step_ms), world, dev)
    # accuracy of this run's result against the FP64 oracle (rank 0 only, after timing)
    result = {}
    if rank == 0:
        result["V"] = V.cpu().numpy()
        op = gm.build(b, c, d, n, LEAF, precision=prec, stream=stream, **extra)  # after timing: T itself
        result["T"] = op.dtn()
        op.free()
    # end-to-end through the C ABI with pinned host buffers (copies inside the timing)
    hb = [torch.from_numpy(cfg[k]).pin_memory() for k in "bcd"]
    hG = torch.from_numpy(Gv).pin_memory()
    hV = torch.empty_like(hG).pin_memory()
    h2d = 3 * n * n * 8 + Gv.size * 8
    d2h = Gv.size * 8
    e2e_t = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = gm.build(hb[0].numpy(), hb[1].numpy(), hb[2].numpy(), n, LEAF, precision=prec, stream=stream,
                      **extra)
        op.solve(hG.numpy(), out=hV.numpy(), stream=stream)
        t1 = time.perf_counter()
        op.free()
        if it >= args.warmup:
            e2e_t.append(t1 - t0)
    e2e_step = statistics.mean(e2e_t)
    # the plain FP64 GPU path on the same workload, for the equal-accuracy comparison
    fp64 = None
    if args.precision == "mixed":
        fb, fs = [], []
        for it in range(2 + 3):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ev[0].record(stream)
            op = gm.build(b, c, d, n, LEAF, precision=gm.PREC_FP64, stream=stream)
            ev[1].record(stream)
            op.solve(G, out=V, stream=stream)
            ev[2].record(stream)
            torch.cuda.synchronize()
            if it >= 2:
                fb.append(ev[0].elapsed_time(ev[1]))
                fs.append(ev[1].elapsed_time(ev[2]))
            op.free()
        fp64 = {"build_ms": statistics.mean(fb), "solve_ms": statistics.mean(fs),
                "value": n * n / ((statistics.mean(fb) + statistics.mean(fs)) * 1e-3) * world,
                "solve_vectors_per_s": NVEC / (statistics.mean(fs) * 1e-3) * world, "steps": 3}
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    # error vs the FP64 oracle, and the oracle's own time as the CPU baseline
    t_cpu, To, Vo = cpu_oracle_step(cfg)
    Vg = result["V"].reshape(NVEC, 4 * n).T
    rel_err = float((np.linalg.norm(Vg - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max())
    rel_err_T = float(np.linalg.norm(result["T"] - To) / np.linalg.norm(To))
    achieved = dom_fl / (dom_ms * 1e-3) / 1e12
    bound, peak, peak_src = family_roofline(args.precision, dom)
    tr = TRAFFIC.get(dom)
    traffic = tr[0] if (tr and tr[1] == source_digest(dom)) else None
    sorted_ms = sorted(step_ms)
    line = {
        "metric": METRIC, "value": whole_job_value(n * n, t_step, world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "split-f64 (6 bf16 digits, df32 storage)" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "leaf": LEAF, "nvec": NVEC, "precision": args.precision,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "graph": bool(args.graph), "autotune": bool(args.autotune),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "build_ms": statistics.mean(build_ms), "solve_ms": statistics.mean(solve_ms),
        "build_gridpoints_per_s": n * n / (statistics.mean(build_ms) * 1e-3) * world,
        "solve_vectors_per_s": NVEC / (statistics.mean(solve_ms) * 1e-3) * world,
        "latency_ms": {"p50": sorted_ms[len(sorted_ms) // 2],
                       "p99": sorted_ms[min(len(sorted_ms) - 1, int(0.99 * len(sorted_ms)))]},
        "rel_err_vs_fp64_oracle": rel_err,
        "rel_err_T_frobenius_vs_fp64_oracle": rel_err_T,
        "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "launches_per_step": dom_n // args.steps,
                     "ms_per_step": dom_ms / args.steps},
        "kernel_ms_per_step": brk_ms,
        "kernel_breakdown_note": "one extra step with every launch timed (event pairs add overhead); "
                                 "the timed steps instrument only the roofline family",
        "kernel_roofline": {f: {"bound": family_roofline(args.precision, f)[0],
                                "achieved_tflops": brk_fl[f] / max(brk_ms[f], 1e-9) / 1e9,
                                "frac": brk_fl[f] / max(brk_ms[f], 1e-9) / 1e9 / family_roofline(args.precision, f)[1]}
                            for f in brk_ms if brk_fl[f] > 0},
        "fp64_path": fp64,
        "cpu_baseline": {"value": n * n / t_cpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "one full step: numpy/LAPACK dense nested dissection (oracle O2) + T @ G "
                                   "of the 256 vectors, default BLAS threading"},
        "rel_err_bound": 1e-8 if args.precision == "mixed" else 1e-10,
        "e2e": {"value": world * n * n / e2e_step, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step * 1e3},
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Serving workload (the solve stage under load): 32 resident operators, n uniform on
    {256, 384, 512, 768, 1024, 1536} (seed 7) plus one at n = 2048 (an 8192 x 8192 T),
    convection and variable-wavespeed Helmholtz fields alternating, mixed precision with
    the automatic FP64 fallback.  Solve requests arrive as a Poisson process with B ~
    U{1..64} Gaussian vectors for a uniformly chosen operator, at 0.25x, 0.5x and 0.9x the
    saturated batched rate; every `quota` requests a new operator is submitted to the
    server's build worker (it overlaps the solves and evicts the least recently used
    operator when admitted).  Baseline: the unbatched FP64 apply -- a server with one
    solve per request over FP64 builds of the same operators.  One JSON line (not the
    headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm

    rng = np.random.default_rng(7)
    sizes = [256, 384, 512, 768, 1024, 1536]
    ns = [int(x) for x in rng.choice(sizes, 31)] + [2048]
    ks = {}

    def fields(n, j):
        if j % 2 == 0:
            return inputs.convection_fields(n, seeds=(200 + 3 * j, 201 + 3 * j, 202 + 3 * j))
        if n not in ks:
            ks[n] = inputs.nudged_wavenumber(n, 16)
        return inputs.helmholtz_fields(n, ks[n])

    dev_fields = {}

    def get_fields(j, n):
        if (j, n) not in dev_fields:
            dev_fields[(j, n)] = [torch.from_numpy(x).cuda() for x in fields(n, j)]
        return dev_fields[(j, n)]

    quota, per_rate = 200, args.serve_requests
    vec_pool = {n: torch.from_numpy(inputs.gaussian_vectors(n, 64, 9 + n).T.copy()).pin_memory()
                for n in sizes + [2048]}
    outs = {n: torch.empty((64, 4 * n), dtype=torch.float64).pin_memory() for n in sizes + [2048]}

    def make_server(batching, precision):
        t0 = time.perf_counter()
        ops = [gm.build(*get_fields(j, n), n, 16, precision=precision) for j, n in enumerate(ns)]
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        budget = sum(op.info()["resident_bytes"] for op in ops) + 1
        srv = gm.Server(budget, batching=batching)
        live = [(srv.add(op), n) for op, n in zip(ops, ns)]
        return srv, live, t_build

    def run(srv, live, rate_req_s, precision, j0):
        srv.reset_stats()
        ids, builds = [], []
        t0 = time.perf_counter()
        t_next = 0.0
        j = j0
        for q in range(per_rate):
            if rate_req_s:
                t_next += rng.exponential(1.0 / rate_req_s)
                while time.perf_counter() - t0 < t_next:
                    pass
            k = int(rng.integers(0, len(live)))
            oid, n = live[k]
            B = int(rng.integers(1, 65))
            try:
                ids.append(srv.submit(oid, vec_pool[n], outs[n], B))
            except gm.GmError:  # evicted meanwhile
                pass
            if (q + 1) % quota == 0:  # a new operator, built on the server's build worker
                n2 = int(rng.choice(sizes))
                oid2, rid = srv.submit_build(*get_fields(j, n2), n2, 16, precision=precision)
                builds.append(rid)
                live.append((oid2, n2))
                j += 1
        for rid in ids + builds:
            srv.wait(rid)
        srv.sync()
        st = srv.stats()
        # the operators still resident (the evicted ones are gone from the server)
        live[:] = live[-st["resident_ops"]:] if st["resident_ops"] else live
        return st, j

    keys = ("p50_ms", "p99_ms", "vectors_per_s", "solves", "requests", "evictions")
    res = {}
    srv_b, live_b, tb_b = make_server(True, gm.PREC_MIXED)
    sat, j = run(srv_b, live_b, 0.0, gm.PREC_MIXED, 100)
    res["saturated"] = {k: sat[k] for k in keys}
    sat_req = sat["vectors_per_s"] / 32.5
    rates = {f: f * sat_req for f in (0.25, 0.5, 0.9)}
    for f, r in rates.items():
        st, j = run(srv_b, live_b, r, gm.PREC_MIXED, j)
        res[f"{f}x"] = {"offered_req_s": r, "batched": {k: st[k] for k in keys}}
    srv_b.close()
    srv_u, live_u, tb_u = make_server(False, gm.PREC_FP64)
    for f, r in rates.items():
        st, j = run(srv_u, live_u, r, gm.PREC_FP64, j)
        res[f"{f}x"]["unbatched_fp64"] = {k: st[k] for k in keys}
    srv_u.close()
    print(json.dumps({"workload": "serving", "operators": f"32 resident: n = {ns}, convection / Helmholtz "
                      "alternating; batched: mixed precision (automatic FP64 fallback), one grouped apply per "
                      "batch; baseline: FP64 operators, one apply per request",
                      "requests_per_rate": per_rate, "vectors_per_request": "U{1..64}", "arrivals": "Poisson",
                      "build_every": quota, "initial_build_s": {"batched_set": tb_b, "fp64_set": tb_u},
                      "results": res}), flush=True)


def _timed(fn, reps):
    """Median host time (ms) of fn() over reps calls, each bracketed by device syncs."""
    import torch
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
        del out
    return statistics.median(ts)


def run_problemset(args):
    """The paper's problem set (Section 6.1: Laplace, Diffusion-Convection I-IV, Helmholtz
    I-IV, Random Laplacian I-II) at n = 512, leaf 16: FP64 and mixed build times, the
    mixed build's e1 / e2 (random unit and smooth boundary vectors) against the FP64
    build, whether the automatic mode fell back to FP64, and the root operator's size in
    HBS form at tol 1e-7 (the paper's M(n) and M(n)/n).  One JSON line (not the headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm

    n, leaf, reps = 512, 16, max(1, args.steps)
    R = torch.from_numpy(np.ascontiguousarray(inputs.error_vectors(n, 17).T)).cuda()
    res = {}
    for name in list(inputs.PAPER_PROBLEMS) + ["random1", "random2"]:
        row = {}
        if name.startswith("random"):
            sx, sy = (inputs.random_laplacian_1 if name == "random1" else inputs.random_laplacian_2)(n)
            sx, sy = torch.from_numpy(sx).cuda(), torch.from_numpy(sy).cuda()
            ref = gm.build_network(sx, sy, n, leaf)
            row["fp64_build_ms"] = _timed(lambda: gm.build_network(sx, sy, n, leaf), reps)
            try:
                inf = gm.build_network(sx, sy, n, leaf, tol=1e-7, hbs_leaf=64).info()
                row["hbs_M_MB"] = inf["hbs_operator_bytes"] / 2**20
                row["hbs_M_over_n"] = inf["hbs_operator_bytes"] / 2**20 / n
                row["hbs_max_rank"] = inf["hbs_max_rank"]
            except gm.GmError as err:
                row["hbs"] = str(err)
        else:
            b, c, d = (torch.from_numpy(x).cuda() for x in inputs.paper_problem(name, n))
            ref = gm.build(b, c, d, n, leaf)
            row["fp64_build_ms"] = _timed(lambda: gm.build(b, c, d, n, leaf), reps)
            mixed = gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED)
            row["mixed_build_ms"] = _timed(lambda: gm.build(b, c, d, n, leaf, precision=gm.PREC_MIXED), reps)
            row["mixed_fell_back_to_fp64"] = bool(mixed.info()["pivot_fallback"])
            V, Vr = mixed.solve(R), ref.solve(R)
            e = (torch.linalg.norm(V - Vr, dim=1) / torch.linalg.norm(Vr, dim=1)).cpu().tolist()
            row["mixed_e1_vs_fp64"], row["mixed_e2_vs_fp64"] = e
            try:
                inf = gm.build(b, c, d, n, leaf, tol=1e-7, hbs_leaf=64).info()
                row["hbs_M_MB"] = inf["hbs_operator_bytes"] / 2**20
                row["hbs_M_over_n"] = inf["hbs_operator_bytes"] / 2**20 / n
                row["hbs_max_rank"] = inf["hbs_max_rank"]
            except gm.GmError as err:
                row["hbs"] = str(err)
        res[name] = row
    print(json.dumps({"workload": "problemset", "n": n, "leaf": leaf, "reps": reps, "timing": "host, synced",
                      "data": "synthetic (the paper's analytic fields; seeded networks)", "results": res}),
          flush=True)


# Table error of the paper (e1, e2 of its HBS solution operator at local tolerance 1e-7,
# n = 1024, against GMRES): context for the line below, not a target.
PAPER_TABLE_ERROR = {"laplace": (6.3e-7, 3.6e-7), "diffconv1": (1.5e-6, 1.3e-6), "diffconv2": (8.7e-6, 8.2e-6),
                     "diffconv3": (5.6e-7, 3.4e-7), "diffconv4": (4.1e-8, 4.1e-8), "helmholtz1": (1.4e-4, 4.8e-7),
                     "helmholtz2": (1.1e-6, 5.1e-6), "helmholtz3": (1.2e-5, 5.7e-4), "helmholtz4": (8.2e-4, 1.2e-3),
                     "random1": (1.8e-7, 1.2e-7), "random2": (1.4e-5, 8.1e-6)}


def run_errors(args):
    """The paper's error experiment (Section 6.1, Table error) at its size: the eleven
    problems at n = 1024, leaf 16, built on the GPU with the HBS path at tol 1e-7 (the
    paper's local tolerance; accelerated merges for shared edges >= 128 and the HBS root;
    the networks with an HBS root), and e1 / e2 -- the relative l2 errors of T r for a
    random unit r and for a smooth r -- against the oracle O2 (the paper used GMRES);
    the dense FP64 GPU build's e1 / e2 beside them, M(n) of the HBS operator, and the
    paper's own e1 / e2 as context.  One JSON line (not the headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    from oracle import nd_dense

    n, leaf, tol = args.n, 16, 1e-7
    R = inputs.error_vectors(n, 17)
    Rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda()
    res = {}
    for name in list(inputs.PAPER_PROBLEMS) + ["random1", "random2"]:
        row = {"paper_e1_e2": PAPER_TABLE_ERROR[name]}
        t0 = time.perf_counter()
        if name.startswith("random"):
            sx, sy = (inputs.random_laplacian_1 if name == "random1" else inputs.random_laplacian_2)(n)
            # the oracle's network build (one load at a corner node rides along; T is unchanged)
            To = nd_dense.build_loads(nd_dense.Problem.network(sx, sy, n), leaf, [0])[0]
            dx, dy = torch.from_numpy(sx).cuda(), torch.from_numpy(sy).cuda()
            hb = gm.build_network(dx, dy, n, leaf, tol=tol, hbs_leaf=64)
            dn = gm.build_network(dx, dy, n, leaf)
        else:
            f = inputs.paper_problem(name, n)
            To = nd_dense.build(*f, n, leaf).T
            b, c, d = (torch.from_numpy(x).cuda() for x in f)
            hb = gm.build(b, c, d, n, leaf, tol=tol, hbs_leaf=64, hbs_min_edge=128)
            dn = gm.build(b, c, d, n, leaf)
        row["oracle_s"] = time.perf_counter() - t0
        if To is not None:
            Vo = To @ R
            for tag, op in (("hbs", hb), ("dense_fp64", dn)):
                V = op.solve(Rd).cpu().numpy().T
                e = np.linalg.norm(V - Vo, axis=0) / np.linalg.norm(Vo, axis=0)
                row[f"{tag}_e1"], row[f"{tag}_e2"] = float(e[0]), float(e[1])
        inf = hb.info()
        row["hbs_M_MB"] = inf["hbs_operator_bytes"] / 2**20
        row["hbs_M_over_n"] = inf["hbs_operator_bytes"] / 2**20 / n
        row["hbs_max_rank"] = inf["hbs_max_rank"]
        row["hbs_fallbacks"] = inf["hbs_fallbacks"]
        res[name] = row
    print(json.dumps({"workload": "errors", "n": n, "leaf": leaf, "tol": tol,
                      "reference": "oracle O2 (dense FP64 nested dissection); the paper's reference was GMRES",
                      "data": "synthetic (the paper's analytic fields; seeded networks)", "results": res}), flush=True)


def run_bodyloads(args):
    """Body loads (Section 6.3) on the paper's body-load problem, Random Laplacian I at
    512 x 512, leaf 16, with N_body = 10, 100, 1000 loads in a localized window: FP64 build
    time of T and F, time of one solve T g + F f, and the conservation error of F (every
    column sums to -h).  One JSON line (not the headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm

    n, leaf, reps = 512, 16, max(1, args.steps)
    h = 1.0 / (n + 1)
    sx, sy = (torch.from_numpy(x).cuda() for x in inputs.random_laplacian_1(n))
    res = {}
    for nb in (10, 100, 1000):
        body = inputs.body_nodes(n, nb, 40 + nb).astype(np.int32)
        op = gm.build_network(sx, sy, n, leaf, body)
        build_ms = _timed(lambda: gm.build_network(sx, sy, n, leaf, body), reps)
        g = torch.from_numpy(inputs.gaussian_vectors(n, 1, 41).T.copy()).cuda()
        f = torch.from_numpy(inputs.body_load_vectors(nb, 1, 42).T.copy()).cuda()
        solve_ms = _timed(lambda: op.solve_loads(g, f), max(reps, 10))
        F = op.load_operator()
        res[str(nb)] = {"build_ms": build_ms, "solve_ms": solve_ms,
                        "conservation_err": float(np.abs(F.sum(axis=0) + h).max() / h)}
    print(json.dumps({"workload": "bodyloads", "problem": "Random Laplacian I (conductivities U(1,2))", "n": n,
                      "leaf": leaf, "precision": "fp64", "reps": reps, "timing": "host, synced",
                      "results": res}), flush=True)


# The paper's Table nested_times (Matlab, 2.4 GHz laptop; its n counts the boundary):
# (problem, n) -> (T_build s, T_solve s) of the accelerated build at local tolerance 1e-7.
PAPER_TIMES = {("laplace", 512): (13.44, 0.013), ("laplace", 1024): (45.25, 0.027),
               ("laplace", 2048): (135.01, 0.058), ("laplace", 4096): (450.73, 0.107),
               ("helmholtz4", 512): (50.78, 0.013), ("helmholtz4", 1024): (193.58, 0.027),
               ("helmholtz4", 2048): (765.35, 0.056), ("helmholtz4", 4096): (3167.56, 0.115)}


def run_paper_times(args):
    """The paper's timing table (Table nested_times): Laplace and Helmholtz IV (40 points
    per wavelength) at n = 512 ... 4096, leaf 16.  For each: the accelerated build at
    local tolerance 1e-7 (HBS for merges with shared edge >= 128 and the root, FP64
    merges) and the solve of one boundary vector, then the dense build (mixed precision
    with the automatic FP64 fallback) and its one-vector solve; the accelerated operator's
    relative error against the dense one on four Gaussian vectors.  The paper's own times
    ride along as context.  One JSON line (not the headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm

    ns = [int(x) for x in args.sizes.split(",")]
    res = {}
    for name in ("laplace", "helmholtz4"):
        for n in ns:
            b, c, d = (torch.from_numpy(x).cuda() for x in inputs.paper_problem(name, n))
            reps = 3 if n <= 1024 else 1
            G = torch.from_numpy(np.ascontiguousarray(inputs.gaussian_vectors(n, 4, 51).T)).cuda()
            g1 = G[:1].contiguous()
            hbs = lambda: gm.build(b, c, d, n, 16, tol=1e-7, hbs_leaf=64, hbs_min_edge=128)
            row = {"paper_build_s": PAPER_TIMES[(name, n)][0], "paper_solve_s": PAPER_TIMES[(name, n)][1]}
            try:
                op = hbs()
            except gm.GmError as e:
                row["hbs_error"] = str(e)
                res[f"{name}_{n}"] = row
                continue
            row["hbs_build_ms"] = _timed(hbs, reps)
            row["hbs_solve_one_ms"] = _timed(lambda: op.solve(g1), 10)
            inf = op.info()
            row["hbs_fallbacks"] = inf["hbs_fallbacks"]
            row["hbs_max_rank"] = inf["hbs_max_rank"]
            row["hbs_M_MB"] = inf["hbs_operator_bytes"] / 2**20
            Vh = op.solve(G).cpu().numpy()
            op.free()
            dense = lambda: gm.build(b, c, d, n, 16, precision=gm.PREC_MIXED)
            od = dense()
            row["dense_build_ms"] = _timed(dense, reps)
            row["dense_solve_one_ms"] = _timed(lambda: od.solve(g1), 10)
            row["dense_in_fp64"] = bool(od.info()["pivot_fallback"])
            Vd = od.solve(G).cpu().numpy()
            od.free()
            row["hbs_rel_err_vs_dense"] = float((np.linalg.norm(Vh - Vd, axis=1) / np.linalg.norm(Vd, axis=1)).max())
            res[f"{name}_{n}"] = row
    print(json.dumps({"workload": "paper_times", "leaf": 16, "tol": 1e-7, "timing": "host, synced, median",
                      "data": "synthetic (the paper's analytic fields)",
                      "note": "the paper's n counts the boundary (h = 1/(n-1)); here n unknowns per side",
                      "results": res}), flush=True)


def _fields_dev(cfg, dev=None):
    import torch
    return [torch.from_numpy(cfg[k]).to(dev or "cuda") for k in ("b", "c", "d")]


def run_cfg3(args):
    """Variable-wavespeed Helmholtz at 10 points per wavelength, 1024 x 1024 unknowns,
    leaf 16, plane-wave data (64 vectors): the HBS build (accelerated merges for shared
    edges >= 128, HBS root, tol 1e-9, FP64) and its solve.  Value: build gridpoints/s of
    the HBS build; the dense FP64 build alongside; error against O2 on 8 of the vectors.
    One JSON line with roofline, cpu_baseline and e2e (not the headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    from oracle import nd_dense

    n, leaf, tol, m = 1024, 16, 1e-9, 64
    cfg = inputs.config3(n, leaf)
    b, c, d = _fields_dev(cfg)
    Gv = np.ascontiguousarray(cfg["G"].T)
    G = torch.from_numpy(Gv).cuda()
    V = torch.empty_like(G)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    kw = dict(tol=tol, hbs_leaf=m, hbs_min_edge=128, stream=stream)
    for _ in range(args.warmup):
        gm.build(b, c, d, n, leaf, **kw).free()
    torch.cuda.synchronize()
    op = gm.build(b, c, d, n, leaf, timing=True, **kw)
    inf = op.info()
    brk_ms, brk_fl = dict(inf["kernel_ms"]), dict(inf["kernel_flops"])
    op.free()
    dom = max(brk_ms, key=lambda f: brk_ms[f])
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    bms, sms, launches = [], [], 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ev[0].record(stream)
        op = gm.build(b, c, d, n, leaf, **kw)
        ev[1].record(stream)
        op.solve(G, out=V, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        bms.append(ev[0].elapsed_time(ev[1]))
        sms.append(ev[1].elapsed_time(ev[2]))
        info = op.info()
        launches += info["launches"]
        op.free()
    clk = clocks.stop()
    # e2e: host (pinned) fields and vectors, copies inside the timing
    hb = [torch.from_numpy(cfg[k]).pin_memory() for k in ("b", "c", "d")]
    hG = torch.from_numpy(Gv).pin_memory()
    hV = torch.empty_like(hG).pin_memory()
    e2e = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = gm.build(hb[0].numpy(), hb[1].numpy(), hb[2].numpy(), n, leaf, **kw)
        op.solve(hG.numpy(), out=hV.numpy(), stream=stream)
        e2e.append(time.perf_counter() - t0)
        op.free()
    # the dense FP64 build of the same problem
    dn = []
    for it in range(3):
        torch.cuda.synchronize()
        ev[0].record(stream)
        op = gm.build(b, c, d, n, leaf, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if it:
            dn.append(ev[0].elapsed_time(ev[1]))
        Vd = op.solve(G[:8].contiguous()).cpu().numpy()
        op.free()
    # the oracle (O2, FP64 dense nested dissection), timed: the CPU baseline
    t0 = time.perf_counter()
    res = nd_dense.build(cfg["b"], cfg["c"], cfg["d"], n, leaf)
    t_cpu = time.perf_counter() - t0
    Vo = res.T @ cfg["G"][:, :8]
    rel = lambda A: float((np.linalg.norm(A - Vo, axis=0) / np.linalg.norm(Vo, axis=0)).max())
    bound = max(1e-10, np.finfo(float).eps * np.linalg.cond(res.S_root, 1))
    t_b, t_s = statistics.mean(bms), statistics.mean(sms)
    bound_kind, peak, src = family_roofline("fp64", dom)
    line = {
        "workload": "cfg3", "metric": METRIC, "value": n * n / (t_b * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_b + t_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "variable-wavespeed Helmholtz, 10 points per wavelength, 1024x1024, leaf 16, "
                               "HBS (tol 1e-9, node size 64) for merges with shared edge >= 128 and the root; "
                               "64 plane-wave vectors (32 angles, seed 5)",
                   "n": n, "leaf": leaf, "tol": tol, "k": cfg["k"],
                   "l2": "flushed before every timed step (256 MiB write)"},
        "build_ms": t_b, "solve_ms": t_s, "solve_vectors_per_s": 64 / (t_s * 1e-3),
        "hbs": {k: info[k] for k in ("hbs_levels", "hbs_max_rank", "hbs_merges", "hbs_update_rank",
                                      "hbs_operator_bytes", "resident_bytes")},
        "rel_err_vs_fp64_oracle": rel(V[:8].cpu().numpy().T), "rel_err_bound": 1e-4,
        "dense_fp64": {"build_ms": statistics.mean(dn), "rel_err_vs_fp64_oracle": rel(Vd.T),
                       "rel_err_bound": bound},
        "roofline": {"kernel": dom, "bound": bound_kind, "achieved": brk_fl[dom] / brk_ms[dom] / 1e9,
                     "peak": peak, "unit": "TFLOP/s", "frac": brk_fl[dom] / brk_ms[dom] / 1e9 / peak,
                     "traffic": None, "peak_source": src},
        "kernel_ms_per_step": brk_ms, "kernel_flops_per_step": brk_fl,
        "cpu_baseline": {"value": n * n / t_cpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "one dense FP64 build of the same problem by the oracle O2 (numpy/LAPACK)"},
        "e2e": {"value": n * n / statistics.mean(e2e), "unit": UNIT, "h2d_bytes_per_step": 3 * n * n * 8 + Gv.size * 8,
                "d2h_bytes_per_step": Gv.size * 8, "ms_per_step": statistics.mean(e2e) * 1e3},
        "clocks": clk, "gpu_launches": launches // max(args.steps, 1),
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The batched build: 64 independent problems, n uniform on {128, 192, 256, 384, 512}
    (seed 6), convection and variable-wavespeed Helmholtz alternating, leaf 16, mixed
    precision with the automatic FP64 fallback, in one gm_build_batch call.  Value: total
    gridpoints / batch build time (device, CUDA events); the same problems built one by
    one alongside; error of one problem per size against O2.  One JSON line (not the
    headline)."""
    import numpy as np
    import torch
    from paper_1302_5995_gb300 import build_ext, inputs
    build_ext.build()
    import paper_1302_5995_gb300 as gm
    from oracle import nd_dense

    probs = inputs.config4()
    dev = [tuple(torch.from_numpy(p[k]).cuda() for k in ("b", "c", "d")) + (p["n"], p["leaf"]) for p in probs]
    total = sum(p["n"] ** 2 for p in probs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ev[0].record(stream)
        out = fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), out

    batch = lambda: gm.build_batch(dev, precision=gm.PREC_MIXED, stream=stream, graph=args.graph,
                                   autotune=args.autotune)
    for _ in range(args.warmup):
        for op in batch():
            op.free()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clocks.start()
    tb = []
    for _ in range(args.steps):
        t, ops = timed(batch)
        tb.append(t)
        last = ops
    clk = clocks.stop()
    fell = sum(op.info()["pivot_fallback"] for op in last)
    ts = []
    for _ in range(2):
        t, ops = timed(lambda: [gm.build(*p, precision=gm.PREC_MIXED, stream=stream) for p in dev])
        ts.append(t)
        for op in ops:
            op.free()
    # one problem per size against O2
    errs = {}
    t_cpu, pts = 0.0, 0
    for i, p in enumerate(probs):
        if p["n"] in errs:
            continue
        G = inputs.gaussian_vectors(p["n"], 8, 70 + i)
        t0 = time.perf_counter()
        To = nd_dense.build(p["b"], p["c"], p["d"], p["n"], p["leaf"]).T
        if p["n"] <= 256:
            t_cpu += time.perf_counter() - t0
            pts += p["n"] ** 2
        V = last[i].solve(np.ascontiguousarray(G.T)).reshape(8, 4 * p["n"]).T
        errs[p["n"]] = float((np.linalg.norm(V - To @ G, axis=0) / np.linalg.norm(To @ G, axis=0)).max())
    # e2e: host coefficient arrays
    hp = [(p["b"], p["c"], p["d"], p["n"], p["leaf"]) for p in probs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ops = gm.build_batch(hp, precision=gm.PREC_MIXED, stream=stream)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    for op in ops:
        op.free()
    t = statistics.mean(tb)
    line = {
        "workload": "batch", "metric": METRIC, "value": total / (t * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "split-f64 (6 bf16 digits, df32 storage); FP64 for the fallback problems",
        "data": "synthetic",
        "config": {"workload": "64 problems, n uniform on {128,192,256,384,512} (seed 6), convection / Helmholtz "
                               "(10 ppw) alternating, leaf 16, one gm_build_batch", "gridpoints": total,
                   "graph": bool(args.graph), "autotune": bool(args.autotune),
                   "l2": "flushed before every timed step (256 MiB write)"},
        "single_builds_ms": statistics.mean(ts), "speedup_vs_single_builds": statistics.mean(ts) / t,
        "problems_in_fp64_fallback": fell,
        "rel_err_vs_fp64_oracle_by_n": errs, "rel_err_bound": 1e-8,
        "cpu_baseline": {"value": pts / t_cpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "oracle O2 builds of the batch's first problem of each size <= 256"},
        "e2e": {"value": total / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * 8 * total, "d2h_bytes_per_step": 0,
                "ms_per_step": t_e2e * 1e3},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gm", "reference"], default="gm")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--workload", choices=["build", "cfg3", "batch", "serving", "problemset", "errors", "bodyloads",
                                           "paper_times"],
                    default="build",
                    help="build: the headline build+solve step; cfg3, batch, serving, problemset, bodyloads: "
                         "other workloads (not the headline)")
    ap.add_argument("--serve-requests", type=int, default=600)
    ap.add_argument("--n", type=int, default=1024, help="grid of the errors workload")
    ap.add_argument("--sizes", default="512,1024,2048,4096", help="grids of the paper_times workload")
    ap.add_argument("--graph", type=int, default=0, help="record each plan's build into a CUDA graph and replay it")
    ap.add_argument("--autotune", type=int, default=0, help="time a few launch shapes on the first build of a plan")
    args = ap.parse_args()
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "cfg3":
        run_cfg3(args)
        return
    if args.workload == "errors":
        run_errors(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "problemset":
        run_problemset(args)
        return
    if args.workload == "paper_times":
        return run_paper_times(args)
    if args.workload == "bodyloads":
        run_bodyloads(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gm(args)


if __name__ == "__main__":
    main()
