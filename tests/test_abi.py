"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/tdes.h declares.  No compute call is made (this suite runs without a
GPU); only argument checks that return before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2007_10752_gb300 import build, tdes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdes.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdes_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tdes.load()


def test_header_declares_the_expected_calls():
    assert set(_declared()) == set(tdes.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a():
    build.build()
    log = open(os.path.join(ROOT, "_build", "ptxas.txt")).read()
    assert "for 'sm_103a'" in log
    # the bitsliced kernels keep every plane in registers
    for m in re.finditer(r"Function properties for (\S*tdes_(ecb|ctr)_kernel\S*)\n\s+(\d+) bytes stack "
                         r"frame, (\d+) bytes spill stores", log):
        assert int(m.group(4)) == 0, f"{m.group(1)} spills registers"


def test_gate_count_matches_generator(lib):
    import json
    js = json.load(open(os.path.join(ROOT, "paper_2007_10752_gb300", "gen", "sbox_lop3.json")))
    assert tdes.tdes_sbox_gate_count() == sum(len(s["gates"]) for s in js["sboxes"])


def test_argument_checks_without_device(lib):
    vp = ctypes.c_void_p
    # NULL key schedule
    assert lib.tdes_ecb_encrypt(None, vp(8), vp(8), 8, None) == tdes.TDES_EINVAL
    assert "NULL" in lib.tdes_last_error().decode()
    assert lib.tdes_ctr_crypt(None, 0, 0, vp(8), vp(8), 8, None) == tdes.TDES_EINVAL
    assert lib.tdes_cbc_decrypt(None, 0, vp(8), vp(8), 8, None) == tdes.TDES_EINVAL
    assert lib.tdes_cbc_encrypt(None, 0, vp(8), vp(8), 8, None) == tdes.TDES_EINVAL
    assert lib.tdes_ecb_crypt_host(None, 0, vp(8), vp(8), 8, vp(16), 1 << 20) == tdes.TDES_EINVAL
    assert lib.tdes_key_schedule(None, None, None, None) == tdes.TDES_EINVAL
    assert tdes.tdes_strerror(tdes.TDES_EINVAL) == "invalid argument"


def test_oversized_calls_refused_without_device(lib):
    """A call of 2^31 tiles of 8 KiB (16 TiB) is refused by the host checks,
    before any device query, in every mode.  Run without a GPU: the pointers
    are placeholders that nothing dereferences (the key-schedule handle is a
    zeroed host buffer, never read before the size check), and no kernel can
    launch here."""
    fake_ks = ctypes.create_string_buffer(256)
    ks = ctypes.addressof(fake_ks)
    p, big = ctypes.c_void_p(1 << 20), (1 << 31) * 8192
    calls = {
        "ecb_encrypt": lambda: lib.tdes_ecb_encrypt(ks, p, p, big, None),
        "ecb_decrypt": lambda: lib.tdes_ecb_decrypt(ks, p, p, big, None),
        "ctr": lambda: lib.tdes_ctr_crypt(ks, 0, 0, p, p, big, None),
        "cbc_decrypt": lambda: lib.tdes_cbc_decrypt(ks, 0, p, p, big, None),
        "cbc_encrypt": lambda: lib.tdes_cbc_encrypt(ks, 0, p, p, big, None),
        "cbc_decrypt_noalloc": lambda: lib.tdes_cbc_decrypt_noalloc(ks, 0, p, p, big, None),
    }
    for name, call in calls.items():
        assert call() == tdes.TDES_EINVAL, name
        assert "2^31 tiles" in lib.tdes_last_error().decode(), name
    # the allocation-free call's in-place scratch limit is a host check too
    rc = lib.tdes_cbc_decrypt_noalloc(ks, 0, p, p, tdes.TDES_NOALLOC_MAX_BYTES + 8192, None)
    assert rc == tdes.TDES_EINVAL
    assert "scratch limit" in lib.tdes_last_error().decode()
