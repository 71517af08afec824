"""The C-ABI library loads and exports every function include/hfsem.h
declares (no GPU needed: nothing is called)."""
import os
import re

from tests._common import ensure_built
from paper_1808_02937_gb300 import hfsem as H

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hfsem.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hfsem_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert declared() == sorted(H.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = ensure_built()
    for name in declared():
        assert hasattr(lib, name), name


def test_status_strings():
    lib = ensure_built()
    assert lib.hfsem_status_str(0) == b"ok"
    assert lib.hfsem_status_str(1) == b"invalid argument"
