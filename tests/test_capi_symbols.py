"""The C-ABI library loads without a GPU and exports every function that
include/cvd.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(cvd_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["cvd_guest_create", "cvd_guest_destroy", "cvd_translate", "cvd_copy_from_guest", "cvd_copy_to_guest",
              "cvd_mmap_install", "cvd_copy_batch", "cvd_tune"]:
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_1304_3771_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1304_3771_b300 import cvd
    assert sorted(cvd.SIGNATURES) == declared_functions()
