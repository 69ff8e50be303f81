"""CPU checks of the C ABI boundary: the library builds, loads, and exports every entry point
that include/*.h declares; host-side validation rejects bad arguments without touching a GPU;
and the product package never reaches the oracle."""

import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(stmf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_1911_03813_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("stmf_create", "stmf_destroy", "stmf_fg", "stmf_norm_x", "stmf_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(stmf_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        getattr(lib, name)


def test_validation_needs_no_gpu(libpath):
    from paper_1911_03813_gb300 import stmf
    L = stmf.lib()
    # NULL context and NULL arguments are rejected before any CUDA call
    assert L.stmf_fg(None, None, None, 3, 2, None, None, None, None, None, None, None) == 1
    assert L.stmf_norm_x(None, None, None, 3, None, None) == 1
    assert L.stmf_create(0, None) == 1
    assert stmf.status_string(0) == "STMF_OK"
    assert L.stmf_version() >= 100


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1911_03813_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if not path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            continue
        src = open(path).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), path
        assert "oracle/" not in src, path
    # and the oracle imports nothing from the product package
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_1911_03813_gb300" not in open(path).read(), path
