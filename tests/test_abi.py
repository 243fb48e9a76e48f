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


def test_batch_server_and_tuner_calls_refuse_null_arguments(lib):
    """The batch-context, shape, autotuner, server and uniform calls refuse
    NULL handles and pointers with TDES_EINVAL before any device query (this
    suite has no GPU), and the no-result calls accept NULL quietly."""
    vp = ctypes.c_void_p
    t = ctypes.c_uint64()
    h = vp()
    EINVAL = tdes.TDES_EINVAL
    refused = {
        "tdes_ctx_create": lambda: lib.tdes_ctx_create(None, None, ctypes.byref(h)),
        "tdes_batch_submit": lambda: lib.tdes_batch_submit(None, None, 0, ctypes.byref(t)),
        "tdes_batch_submit_plan": lambda: lib.tdes_batch_submit_plan(None, None, ctypes.byref(t)),
        "tdes_batch_poll": lambda: lib.tdes_batch_poll(None, 1, None),
        "tdes_batch_wait": lambda: lib.tdes_batch_wait(None, 1, 1000),
        "tdes_batch_release": lambda: lib.tdes_batch_release(None, 1),
        "tdes_batch_plan": lambda: lib.tdes_batch_plan(None, None, 0, None, ctypes.byref(h)),
        "tdes_batch_set_shape": lambda: lib.tdes_batch_set_shape(None, None),
        "tdes_batch_get_shape": lambda: lib.tdes_batch_get_shape(None, None),
        "tdes_batch_configure": lambda: lib.tdes_batch_configure(None, 8, 0),
        "tdes_batch_info": lambda: lib.tdes_batch_info(None, None),
        "tdes_batch_launch": lambda: lib.tdes_batch_launch(None, None),
        "tdes_batch_autotune": lambda: lib.tdes_batch_autotune(None, 0, 5, None, None),
        "tdes_keytable_create": lambda: lib.tdes_keytable_create(None, 1, ctypes.byref(h)),
        "tdes_server_create": lambda: lib.tdes_server_create(None, None, ctypes.byref(h)),
        "tdes_server_submit": lambda: lib.tdes_server_submit(None, None, ctypes.byref(t)),
        "tdes_server_poll": lambda: lib.tdes_server_poll(None, 1),
        "tdes_server_stats": lambda: lib.tdes_server_stats(None, 0, None),
        "tdes_server_autotune": lambda: lib.tdes_server_autotune(None, None, 0, None),
        "tdes_serve_loadtest": lambda: lib.tdes_serve_loadtest(None, None, None),
        "tdes_uniform_scratch_bytes": lambda: lib.tdes_uniform_scratch_bytes(None, 1, 64, None),
        "tdes_uniform_info": lambda: lib.tdes_uniform_info(None, None),
    }
    for name, call in refused.items():
        assert call() == EINVAL, name
    # calls without a result accept NULL
    lib.tdes_ctx_destroy(None)
    lib.tdes_ctx_config_default(None)
    lib.tdes_batch_free(None)
    lib.tdes_keytable_free(None)
    lib.tdes_server_destroy(None)
    cfg = tdes.CtxConfig()
    lib.tdes_ctx_config_default(ctypes.byref(cfg))
    assert cfg.streams == 2
    # the autotune cache follows TDES_AUTOTUNE_CACHE (set for the test session)
    assert lib.tdes_autotune_cache_path().decode() == os.environ["TDES_AUTOTUNE_CACHE"]
