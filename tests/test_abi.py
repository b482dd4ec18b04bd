"""The C ABI library builds, loads without a GPU and exports every symbol the header declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zippir.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^int\s+(zp_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_09190_gb300 import build as b
    b.build()
    import paper_2603_09190_gb300 as zp
    return zp.load_library()


def test_header_and_binding_agree():
    import paper_2603_09190_gb300 as zp
    assert declared_symbols() == sorted(zp.EXPORTS)


def test_library_exports_all(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_and_host_validation(lib):
    import ctypes
    import paper_2603_09190_gb300 as zp
    assert lib.zp_version() == 100
    # host-side validation fails before any device work, so it runs without a GPU
    out = ctypes.c_void_p()
    assert lib.zp_init(0, None, ctypes.byref(out)) == zp.ZP_EINVAL
    P = zp._Params(1024, 2048, 0, 7)
    assert lib.zp_init(0, ctypes.byref(P), ctypes.byref(out)) == zp.ZP_EINVAL
    assert "p_bits" in zp.last_error()
    P = zp._Params(1024, 3072, 0, 8)
    assert lib.zp_init(0, ctypes.byref(P), ctypes.byref(out)) == zp.ZP_EUNSUPPORTED
    P = zp._Params(0, 2048, 0, 8)
    assert lib.zp_init(0, ctypes.byref(P), ctypes.byref(out)) == zp.ZP_EINVAL
    assert lib.zp_answer(None, None, 1, None, None) == zp.ZP_EINVAL
    assert lib.zp_compress(None, None, None, None, 1, None, None) == zp.ZP_EINVAL
