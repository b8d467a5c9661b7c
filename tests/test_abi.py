"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/gadi.h (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gadi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gadi_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2501_04229_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "gadi_create" in names and "gadi_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2501_04229_gb300 import gadi
    assert sorted(gadi.EXPORTS) == _declared()


def test_status_strings_without_gpu(lib_path):
    from paper_2501_04229_gb300 import gadi
    gadi.load(lib_path)
    assert gadi.status_str(0) == "GADI_OK"
    assert gadi.status_str(7) == "GADI_ERR_TIMEOUT"


def test_missing_library_fails_loudly(tmp_path):
    from paper_2501_04229_gb300 import gadi
    saved = gadi._lib
    gadi._lib = None
    try:
        with pytest.raises(RuntimeError):
            gadi.load(str(tmp_path / "libgadi.so"))
    finally:
        gadi._lib = saved
