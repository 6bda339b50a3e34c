"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/bfs.h (CPU only: no compute call is made)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(bfs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2503_00430_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bfs_graph_upload", "bfs_graph_free", "bfs_single", "bfs_single_ex", "bfs_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches_header(lib_path):
    import paper_2503_00430_gb300 as B
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
    assert sorted(B.exported_names()) == declared_functions()
    B.load(lib_path)
    assert B.bfs_strerror(B.BFS_ETIMEOUT) == "device-side wait timed out"
    p = B.bfs_params_default()
    assert (p.alpha, p.beta, p.tau_inv, p.large_diameter_degree) == (14, 24, 20, 7)


def test_host_only_calls_fail_cleanly_without_gpu(lib_path):
    import paper_2503_00430_gb300 as B
    B.load(lib_path)
    import numpy as np
    with pytest.raises(B.BfsError) as e:
        B.bfs_graph_upload(np.array([0, 0], dtype=np.int64), np.zeros(0, dtype=np.int32), n=0)
    assert e.value.code == B.BFS_EINVAL



def test_graph_class_keys():
    import paper_2503_00430_gb300 as B
    assert B.graph_class(4096 * 4096, 67092480).startswith("large_diameter")
    assert B.graph_class(1 << 25, 1047207640) == "dense_n2e25"
    assert B.graph_class(1 << 24, 268435294) == "sparse_n2e24"


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C sizes and field offsets (a tiny C
    program compiled against include/bfs.h prints them)."""
    import paper_2503_00430_gb300 as B
    structs = {"bfs_params": B.bfs_params, "bfs_stats": B.bfs_stats, "bfs_level_stat": B.bfs_level_stat,
               "bfs_multi_stats": B.bfs_multi_stats, "bfs_dup_level": B.bfs_dup_level,
               "bfs_dup_stats": B.bfs_dup_stats, "bfs_graphset_stats": B.bfs_graphset_stats,
               "bfs_query_stats": B.bfs_query_stats, "bfs_tune_report": B.bfs_tune_report}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bfs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)
