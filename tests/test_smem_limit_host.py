"""The dynamic shared-memory limit of a kernel is one value per function, shared by the
host threads that launch it (the side-by-side merges of a stage run on several).
csrc/smem_limit.h raises it under a lock and never lowers it; checked here with g++
against a fake cudaFuncSetAttribute (tests/smem_limit_shim.cpp) whose fake launches
fail above the limit in force, as real ones do.  No GPU is involved.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    nvcc = shutil.which("nvcc")
    for d in ([os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")] if nvcc else []) + \
             ["/usr/local/cuda/include"]:
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


@pytest.fixture()
def shim(tmp_path):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("no CUDA headers")
    out = str(tmp_path / "smem_limit_shim.so")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-pthread", "-Wl,-Bsymbolic", "-I", inc,
                           "-o", out, os.path.join(ROOT, "tests", "smem_limit_shim.cpp")])
    L = ctypes.CDLL(out)
    for name, args in {"shim_interleaved": [ctypes.c_int] * 3, "shim_stress": [ctypes.c_int, ctypes.c_int, ctypes.c_uint],
                       "shim_too_large": [], "shim_limit": [ctypes.c_int], "shim_sets": []}.items():
        getattr(L, name).restype = ctypes.c_int
        getattr(L, name).argtypes = args
    return L


def test_per_launch_setting_loses_to_an_interleaved_thread(shim):
    """The interleaving that made a merge's QR launch fail: the limit set for a large
    request is lowered by another thread's small one before the large launch."""
    assert shim.shim_interleaved(0, 150 * 1024, 40 * 1024) == 1


def test_raised_limit_serves_both(shim):
    assert shim.shim_interleaved(1, 150 * 1024, 40 * 1024) == 0
    assert shim.shim_limit(0) == 150 * 1024
    sets = shim.shim_sets()
    assert shim.shim_interleaved(1, 100 * 1024, 10 * 1024) == 0  # below the limit: no call at all
    assert shim.shim_sets() == sets


def test_many_threads_never_fail_and_the_limit_is_the_largest_request(shim):
    assert shim.shim_stress(16, 2000, 7) == 0
    assert 190 * 1024 <= shim.shim_limit(0) <= 200 * 1024
    assert 190 * 1024 <= shim.shim_limit(1) <= 200 * 1024


def test_refused_request_keeps_the_limit(shim):
    assert shim.shim_too_large() == 0
    assert shim.shim_limit(1) == 64 * 1024
