"""The C-ABI library loads and exports every function that include/spdhss.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "spdhss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:spdhss_status|const char\*|int64_t|void)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_declared_symbols():
    from paper_2011_07632_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    lib.spdhss_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.spdhss_version()


def test_binding_signatures_cover_header():
    from paper_2011_07632_gb300 import native
    assert set(_declared()) <= set(native.exported_symbols())
