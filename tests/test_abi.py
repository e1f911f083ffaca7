"""The C ABI library loads and exports every entry point include/mf.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_builds_and_exports_all_symbols():
    from paper_2209_09848_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_calls_without_gpu():
    import paper_2209_09848_gb300 as mf
    assert "sm_103a" in mf.version()
    assert isinstance(mf.last_error(), str)


def test_invalid_table_arguments_rejected_on_host():
    import paper_2209_09848_gb300 as mf
    import pytest
    with pytest.raises(mf.MFError) as e:
        mf.prf_table_create([0.1, 0.2], [0.0, 0.0], 0)
    assert e.value.status == 1
    with pytest.raises(mf.MFError):
        mf.prf_table_create([float("inf")], [0.0], 5)
