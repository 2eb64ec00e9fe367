"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/ivm.h declares (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import numpy as np

import oracle
from paper_2501_02747_gb300 import build, ivm
from paper_2501_02747_gb300 import scenegen as sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(ivm_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    declared = declared_functions()
    assert {"ivm_create", "ivm_destroy", "ivm_build_matrix", "ivm_build_table",
            "ivm_expand_image_tree", "ivm_strerror"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    assert declared <= exported, declared - exported
    # the binding describes exactly the declared functions
    assert set(ivm.SIGNATURES) == declared
    L = ivm.lib()
    for name in declared:
        assert getattr(L, name) is not None


def test_strerror_is_host_only():
    L = ivm.lib()
    assert L.ivm_strerror(0) == b"ok"
    assert b"range" in L.ivm_strerror(2)
    assert L.ivm_strerror(999) == b"unknown error"


def test_struct_layouts_match_header():
    assert ctypes.sizeof(ivm.ivm_facet) == 40
    assert ctypes.sizeof(ivm.ivm_params) == 32
    assert ctypes.sizeof(ivm.ivm_tree_summary) == 24
    assert ctypes.sizeof(ivm.ivm_stats) == 10 * 8 + 6 * 4 + 8
    assert ctypes.sizeof(ivm.ivm_range) == 32 == ivm.RANGE_DTYPE.itemsize
    assert ctypes.sizeof(ivm.ivm_range_summary) == 32


def test_oracle_entries_agree_with_rows():
    sc = sg.tiny()
    n = sc.n_facets
    M = np.unpackbits(oracle.matrix(sc.facets, 3).view(np.uint8), bitorder="little") \
        .reshape(n, -1)[:, :n]
    rng = np.random.default_rng(5)
    pairs = rng.integers(0, n, (60, 2))
    assert (oracle.pair_entries(sc.facets, 3, pairs) == M[pairs[:, 0], pairs[:, 1]]).all()
    tab, los = oracle.table(sc.facets, 3, sc.tx, sc.rx)
    T = np.unpackbits(tab.view(np.uint8), bitorder="little").reshape(tab.shape[0], 2, -1)[:, :, :n]
    ts = rng.integers(0, sc.n_snap, 40)
    js = rng.integers(0, n, 40)
    assert (oracle.table_entries(sc.facets, 3, sc.rx[ts], js) == T[ts, 1, js]).all()
    assert (oracle.table_entries(sc.facets, 3, sc.tx[ts], js) == T[ts, 0, js]).all()
    assert (oracle.los_entries(sc.facets, 3, sc.tx[ts], sc.rx[ts]) == los[ts]).all()
