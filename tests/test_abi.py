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


# typedef name in include/fs.h -> ctypes mirror in the binding
_STRUCTS = {"fs_law": "fs_law", "fs_sim_params": "fs_sim_params", "fs_graph_opts": "fs_graph_opts",
            "fs_graph_info_t": "fs_graph_info", "fs_server_cfg": "fs_server_cfg", "fs_server_stats": "fs_server_stats"}


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler gives
    the header's struct (checked by compiling a probe against include/fs.h)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fs.h"', "int main(void) {"]
    for cname, pname in _STRUCTS.items():
        cls = getattr(_abi, pname)
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, pname in _STRUCTS.items():
        cls = getattr(_abi, pname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_bounds_checked_library_exports_the_same_boundary():
    from paper_2604_22092_gb300 import _build_lib
    _build_lib.build()
    raw = ctypes.CDLL(_build_lib.LIB_BOUNDS)
    for name in declared_entry_points():
        assert hasattr(raw, name), name
    e = ctypes.c_int32()
    assert raw.fs_debug_bounds_build(ctypes.byref(e)) == 0 and e.value == 1


def test_test_hooks_validate_their_arguments():
    """The failure-detection settings: host-side checks only (no GPU work)."""
    assert not fs.fs_debug_bounds_build()
    with pytest.raises(fs.FsError) as e:
        fs.fs_test_inject(fs.FS_TEST_BOUNDS_SHRINK, 3)     # normal build: no bounds checks
    assert e.value.status == 7
    with pytest.raises(fs.FsError) as e:
        fs.fs_test_inject(fs.FS_TEST_WAIT_TIMEOUT, -1)
    assert e.value.status == 1
    with pytest.raises(fs.FsError) as e:
        fs.fs_test_inject(99, 0)
    assert e.value.status == 1
    fs.fs_test_inject(fs.FS_TEST_WAIT_TIMEOUT, 64)
    fs.fs_test_inject(fs.FS_TEST_WAIT_TIMEOUT, 0)


def test_allocator_entry_points_validate_their_arguments():
    """fs_set_allocator with one function but not the other is refused; the
    cache query works without a GPU (nothing cached)."""
    L = fs.load()
    fa = _abi.ALLOC_FN(lambda n, ctx: 0)
    assert L.fs_set_allocator(fa, _abi.FREE_FN(), None) == 1
    assert L.fs_set_allocator(_abi.ALLOC_FN(), _abi.FREE_FN(), None) == 0
