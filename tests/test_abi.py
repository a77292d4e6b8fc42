"""The C ABI library builds, loads and exports every symbol include/fwi.h declares (CPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fwi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1504_08340_gb300 import build as b
    from paper_1504_08340_gb300.fwi import EXPORTS

    path = b.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations found"
    assert set(declared) == set(EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_fails_loudly_without_library(tmp_path):
    import pytest

    from paper_1504_08340_gb300 import fwi

    with pytest.raises(ImportError):
        saved = fwi._lib
        fwi._lib = None
        try:
            fwi.load_library(str(tmp_path / "missing.so"))
        finally:
            fwi._lib = saved


def test_status_strings():
    from paper_1504_08340_gb300 import build as b

    lib = ctypes.CDLL(b.build())
    lib.fwi_status_string.restype = ctypes.c_char_p
    for code in range(8):
        assert lib.fwi_status_string(code)
