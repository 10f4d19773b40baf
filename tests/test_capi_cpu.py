"""C-ABI checks that need no GPU: the library builds for sm_103a and loads, exports every entry
point that include/qew.h declares, the binding knows exactly those, and argument errors that
are caught before any device work come back as statuses with a message."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "qew.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qew_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1211_7275_gb300 import _capi
    return _capi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_matches_header():
    from paper_1211_7275_gb300 import _capi
    assert sorted(_capi.SIGNATURES) == _declared()


def test_library_is_sm_103a():
    from paper_1211_7275_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


def test_argument_errors_without_device(lib):
    h = ctypes.c_void_p()
    assert lib.qew_create(ctypes.byref(h), 0, 1, 1.0, 0.1, 0, 1) == -1
    assert h.value is None
    assert b"chain length" in lib.qew_last_error(None)
    assert lib.qew_create(ctypes.byref(h), 16, 0, 1.0, 0.1, 0, 1) == -1
    assert lib.qew_create(ctypes.byref(h), 16, 1, 1.0, 0.7, 0, 1) == -1
    assert b"dt" in lib.qew_last_error(None)
    assert lib.qew_create(ctypes.byref(h), 16, 1, float("nan"), 0.1, 0, 1) == -1
    assert lib.qew_create(ctypes.byref(h), 16, 1, 4096.0, 0.1, 0, 1) == -1
    assert b"|f| < 2^12" in lib.qew_last_error(None)
    assert lib.qew_create(ctypes.byref(h), 16, 1, 1.0, 0.1, 7, 1) == -1
    assert lib.qew_create(ctypes.byref(h), 1 << 31, 1, 1.0, 0.1, 0, 1) == -1
    assert lib.qew_create(None, 16, 1, 1.0, 0.1, 0, 1) == -1
    assert lib.qew_advance(None, 5) == -1
    assert lib.qew_observe(None, None, 0, None, None) == -1
    assert lib.qew_disorder_values(5, 0, 1, 0, None, None, 0, None) == -1
    assert lib.qew_philox_words(None, None, -1, None) == -1
    lib.qew_destroy(None)


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1211_7275_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, fn)) as fh:
                    src = fh.read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "liboracle" not in src and "qew_oracle" not in src, fn
