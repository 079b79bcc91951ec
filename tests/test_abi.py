"""The C-ABI library loads and exports every entry point include/rmc.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rmc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("rmc_build_leaf", "rmc_couple", "rmc_lowest", "rmc_kron_matvec", "rmc_rotate_op", "rmc_syev"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2609_02394_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_2609_02394_b300 as P
    assert sorted(P.EXPORTED) == declared_functions()


def test_no_cpu_fallback_without_library(tmp_path):
    import paper_2609_02394_b300 as P
    with pytest.raises(RuntimeError):
        P._lib = None
        try:
            P.load_library(str(tmp_path / "missing.so"))
        finally:
            P._lib = None
