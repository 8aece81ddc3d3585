"""The C ABI library loads on any host and exports every declared symbol.

No compute call is made here (no GPU needed): the header's prototypes are
parsed and each name is looked up in libcdmd.so.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdmd.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdmd_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1512_04205_gb300 import build, cdmd
    build.build()
    return cdmd.load_library()


def test_header_declares_the_four_passes():
    names = _declared()
    for required in ("cdmd_sketch", "cdmd_decompose", "cdmd_lift", "cdmd_subtract"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1512_04205_gb300 import cdmd
    assert sorted(cdmd.EXPORTED) == _declared()


def test_status_strings_without_gpu(lib):
    lib.cdmd_status_string.restype = __import__("ctypes").c_char_p
    assert lib.cdmd_status_string(0) == b"CDMD_OK"
    assert lib.cdmd_status_string(5) == b"CDMD_ERR_RANK_DEFICIENT"
