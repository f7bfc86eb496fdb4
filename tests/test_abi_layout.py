"""The binding's views of the C ABI's structs (ctypes structures and numpy record
types) have the header's layout: a small C program compiled against
include/aln_gb300.h prints sizeof and offsetof of every field, and each must
equal the binding's (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1505_07855_gb300 as aln
from paper_1505_07855_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CTYPES = ["fm_build_opts", "fm_index_info_t", "aln_batch", "aln_params", "aln_result", "aln_server_config",
          "aln_server_stats_t"]
NUMPY = {"aln_hit": aln.HIT_DTYPE, "aln_read_result": aln.RES_DTYPE, "aln_pair_result": aln.PAIR_DTYPE}


def _c_layout(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aln_gb300.h"', "int main(void) {"]
    for name in CTYPES:
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in getattr(_lib, name)._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    for name, dt in NUMPY.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in dt.names:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append('printf("aln_pair_stats size %zu\\n", sizeof(aln_pair_stats));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for ln in out.splitlines():
        struct, field, value = ln.split()
        layout[(struct, field)] = int(value)
    return layout


def test_binding_structs_have_the_header_layout(tmp_path):
    c = _c_layout(tmp_path)
    for name in CTYPES:
        cls = getattr(_lib, name)
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[(name, f)], f"{name}.{f}"
    for name, dt in NUMPY.items():
        assert dt.itemsize == c[(name, "size")], name
        for f in dt.names:
            assert dt.fields[f][1] == c[(name, f)], f"{name}.{f}"
    # aln_pair_stats is read as 8 uint32 words, the first six named
    assert c[("aln_pair_stats", "size")] == 32 and len(aln.PAIR_STATS_FIELDS) == 6
