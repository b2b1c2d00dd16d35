"""The C-ABI library loads and exports every entry point that include/fs.h
declares, and the Python binding declares a prototype for each (no compute
calls: these tests run without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_2604_22092_gb300 as fs
from paper_2604_22092_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:fs_status|const char\*)\s+(fs_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ["fs_graph_create", "fs_sim_init", "fs_sim_step", "fs_sim_run", "fs_graph_destroy",
                     "fs_sim_destroy", "fs_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    L = fs.load()
    raw = ctypes.CDLL(_abi.lib_path())
    for name in declared_entry_points():
        assert hasattr(raw, name), name
        assert name in _abi.PROTOTYPES, f"binding lacks {name}"
    assert fs.fs_version().startswith("flashstep")
    assert L.fs_last_error() is not None


def test_binding_names_match_c_entry_points():
    for name in declared_entry_points():
        assert callable(getattr(fs, name)), name


def test_oracle_is_not_imported_by_the_product_package():
    pkg = os.path.join(ROOT, "paper_2604_22092_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text
                assert "fs_oracle" not in text, f
