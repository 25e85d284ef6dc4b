"""The C-ABI library builds, loads and exports every symbol of include/vor.h.

CPU only: nothing here launches device work.
"""

import ctypes
import os
import re

import pytest

import paper_1212_1095_gb300 as vg

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared(header):
    text = open(os.path.join(HEADER, header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vor_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    vg.build_library()
    return vg.library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("vor.h")
    assert "vor_build_async" in names and "vor_status" in names
    for name in names:
        assert hasattr(lib, name), name


def test_host_only_entry_points(lib):
    o = vg.vor_opts_default()
    assert (o.bucket_side, o.lanes_per_cell, o.target, o.exact_only, o.check_duplicates,
            o.collect_stats) == (0, 0, 0, 0, 1, 0)
    assert vg.vor_edge_capacity(1000) >= 10 * 1000
    assert vg.vor_delaunay_capacity(1000) >= 3 * 1000 - 6
    ws = vg.vor_workspace_bytes(1 << 20, 1 << 20, o)
    assert ws > (1 << 20) * 16
    assert vg.vor_workspace_bytes(0, 1 << 20, o) == -1
    assert vg.vor_workspace_bytes(10, (1 << 20) + 1, o) == -1
    assert vg.vor_workspace_bytes(10, 1 << 20, vg.vor_opts_default(lanes_per_cell=3)) == -1
    assert vg.vor_host_scratch_bytes(100) > 100 * 8
    assert vg.vor_strerror(-3) == "two sites are equal"
    assert vg.vor_strerror(0) == "ok"


def test_argument_errors_need_no_gpu(lib):
    # null pointers are rejected before any CUDA call
    o = vg.vor_opts_default()
    out = vg.VorOut()
    rc = vg.vor_build_async(0, 10, 1000, o, 0, 0, out, 0)
    assert rc == -1


def test_no_cpu_fallback_in_the_package():
    # the product path never imports the oracle
    pkg = os.path.dirname(vg.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(root, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "vor_oracle" not in src, f
