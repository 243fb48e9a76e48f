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
