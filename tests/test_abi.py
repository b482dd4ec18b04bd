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


def test_host_validation_of_the_newer_entry_points(lib):
    """Argument checks of the scale option, the keystream, the standalone compression and
    the client-side calls return before any device work (no GPU here)."""
    import ctypes
    import paper_2603_09190_gb300 as zp
    out = ctypes.c_void_p()
    P = zp._Params(1024, 2048, 0, 8, 2)  # scale 2 does not exist
    assert lib.zp_init(0, ctypes.byref(P), ctypes.byref(out)) == zp.ZP_EINVAL
    assert "scale" in zp.last_error()
    key, nonce = ctypes.create_string_buffer(32), ctypes.create_string_buffer(12)
    fake = ctypes.c_void_p(1 << 40)  # never dereferenced: the calls fail first
    # 3 blocks from counter 2^32 - 2 would wrap the 32-bit block counter
    assert lib.zp_prg_chacha20(key, nonce, 2**32 - 2, fake, 33, None) == zp.ZP_EINVAL
    assert lib.zp_prg_chacha20(None, nonce, 0, fake, 16, None) == zp.ZP_EINVAL
    assert lib.zp_prg_chacha20(key, nonce, 0, fake, 0, None) == zp.ZP_OK  # nothing to do
    m = (1 << 2047) + 1
    mw = (ctypes.c_uint32 * 96)(*[(m >> (32 * i)) & 0xFFFFFFFF for i in range(96)])
    assert lib.zp_lc_create(0, 1024, mw, ctypes.byref(out)) == zp.ZP_EUNSUPPORTED
    assert lib.zp_lc_create(0, 3072, mw, ctypes.byref(out)) == zp.ZP_EINVAL  # m has 2048 bits
    even = (ctypes.c_uint32 * 64)(*([0] * 63 + [1 << 31]))
    assert lib.zp_lc_create(0, 2048, even, ctypes.byref(out)) == zp.ZP_EINVAL
    assert lib.zp_lc_compress(None, None, None, 1, 0, 1, None, 0, 0, None, None) == zp.ZP_EINVAL
    assert lib.zp_lc_set_key(None, None, 8, 8, None) == zp.ZP_EINVAL
    assert lib.zp_client_powm(None, None, None, 1, None, 1, None) == zp.ZP_EINVAL
    assert lib.zp_client_decrypt(None, None, None, None, None, 1, None) == zp.ZP_EINVAL
    assert lib.zp_client_expand_ckr(None, key, nonce, 0, None, 1, None) == zp.ZP_EINVAL
    assert lib.zp_db_prepare_fp16(None, None) == zp.ZP_EINVAL
