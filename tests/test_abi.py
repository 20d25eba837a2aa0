"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/mb.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mb.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mb_status|void|int|size_t|const char \*)\s*(mb_\w+)\s*\(", src, re.M)))


def test_header_declares_the_sweep_calls():
    names = declared()
    for n in ("mb_create", "mb_step", "mb_sweep", "mb_read_state", "mb_write_state", "mb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1711_11361_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_1711_11361_gb300 import mb
    assert sorted(mb.EXPORTS) == declared()
