"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/srmc.h declares (no compute calls here)."""
import os
import re

from paper_2407_21085_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "srmc.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srmc_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("srmc_create", "srmc_solve", "srmc_solve_step", "srmc_eval", "srmc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    B.build()
    import ctypes
    lib = ctypes.CDLL(B.LIB)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing
    lib.srmc_version.restype = ctypes.c_int
    assert lib.srmc_version() == 1


def test_product_path_does_not_import_the_oracle():
    # the package never imports, links or loads anything under oracle/
    pkg = os.path.dirname(B.__file__)
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|libsrmc_oracle|srmc_oracle\.h", re.M)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                assert not pat.search(open(os.path.join(root, f)).read()), f
