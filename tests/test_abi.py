"""The C ABI library builds, loads and exports every entry point of include/*.h (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1707_04228_gb300 import lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(gl_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("gl_create", "gl_setup", "gl_solve", "gl_stress", "gl_apply_K", "gl_apply_prec"):
        assert must in names


def test_library_exports_every_declared_symbol(gl_lib):
    for name in declared_functions():
        assert hasattr(gl_lib, name), name
    assert set(declared_functions()) == set(lib.SIGNATURES)


def test_error_strings_without_gpu(gl_lib):
    assert gl_lib.gl_strerror(0) == b"ok"
    assert gl_lib.gl_strerror(-4) == b"matrix not positive definite"
    assert gl_lib.gl_strerror(12345) == b"unknown error"


def test_binding_refuses_missing_library(tmp_path):
    with pytest.raises(ImportError):
        lib.load(str(tmp_path / "nope.so"))
