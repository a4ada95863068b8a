"""The Python binding's ctypes structures have the C header's layout: for gm_opts,
gm_info_t, gm_problem and gm_server_stats_t, gcc compiles include/gm.h and prints each
struct's size and every field's offset, which must equal ctypes.sizeof and the ctypes
field offsets (a mismatch would silently corrupt every call that passes the struct)."""
import ctypes
import os
import subprocess

import pytest

import paper_1302_5995_gb300 as gm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"gm_opts": gm.Opts, "gm_info_t": gm.Info, "gm_problem": gm.Problem, "gm_server_stats_t": gm.ServerStats}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gm.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, key, val = line.split()
        out[(cname, key)] = int(val)
    return out


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_binding_structs_match_the_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == c_layout[(cname, "size")]
    for fname, _ in cls._fields_:
        assert getattr(cls, fname).offset == c_layout[(cname, fname)], fname
