"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ph_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def _lib_path():
    from paper_1802_09824_gb300 import build
    if not os.path.exists(build.OUT):
        build.build()
    return build.OUT


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["ph_build_leaves", "ph_leaf_pairs", "ph_pp_accel", "ph_free", "ph_last_error",
                 "ph_build_leaves_batched", "ph_status"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_last_error_callable_without_gpu():
    lib = ctypes.CDLL(_lib_path())
    lib.ph_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.ph_last_error(), bytes)   # empty in a fresh process


def test_binding_names_match_header():
    from paper_1802_09824_gb300 import binding
    for n in _declared():
        assert hasattr(binding, n), n
