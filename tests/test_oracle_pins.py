"""Pins for the CPU oracle: what the paper and the mathematics fix, checked
against something other than the oracle itself.

* An independent 3DES implementation run as a black box (the
  ``cryptography`` package's TripleDES, and the OpenSSL command line when
  present) on seeded ECB / CBC inputs, and CTR as that library's ECB applied
  to constructed counter blocks.  This pins every table, the bit order, the
  S-box row reading and the combination order of the halves.
* Closed-form properties the paper states or implies: decryption with the
  round keys reversed inverts encryption (Sec. III-B); EDE3 with K1=K2=K3 is
  single DES (Sec. III-B, backward compatibility); the complementation
  property (E and the round-key XOR are bit selections and XORs); weak keys
  (all round keys equal, so encryption is an involution); parity bits never
  reach PC-1 (Sec. III-A).
* The paper's worked example of S-box addressing (Sec. III-B), stored in
  tests/golden/sbox_worked_example.txt.
* Mutation checks: plausible mistakes planted in copies of the oracle's
  source (never in the CUDA path) must each fail at least one pin.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_2007_10752_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _crypto():
    try:
        from cryptography.hazmat.decrepit.ciphers.algorithms import TripleDES
        from cryptography.hazmat.primitives.ciphers import Cipher, modes
    except Exception:
        return None
    return TripleDES, Cipher, modes


def _lib_ecb(keys, data, decrypt=False):
    TripleDES, Cipher, modes = _crypto()
    c = Cipher(TripleDES(bytes(keys)), modes.ECB())
    op = c.decryptor() if decrypt else c.encryptor()
    return op.update(bytes(data)) + op.finalize()


def _lib_cbc(keys, iv, data, decrypt=False):
    TripleDES, Cipher, modes = _crypto()
    c = Cipher(TripleDES(bytes(keys)), modes.CBC(iv.to_bytes(8, "big")))
    op = c.decryptor() if decrypt else c.encryptor()
    return op.update(bytes(data)) + op.finalize()


def _counter_blocks(nonce, ctr0, n):
    ctr = (np.uint64(ctr0) + np.arange(n, dtype=np.uint64)) & np.uint64(0xFFFFFFFF)
    v = (np.uint64(nonce) << np.uint64(32)) | ctr
    return v.astype(">u8").view(np.uint8)


needs_lib = pytest.mark.skipif(_crypto() is None, reason="cryptography TripleDES not installed")

SIZES = [1, 2, 7, 32, 33, 257]


# --------------------------------------------------------------- pin checks
# Each check takes an Oracle build and raises AssertionError on failure, so the
# same checks run on the real oracle and on the planted mutants below.

def check_library_ecb(o: Oracle):
    for i, n in enumerate(SIZES):
        keys = synth.key_triple(100 + i)
        data = synth.random_bytes(100 + i, 8 * n)
        enc = o.tdes_ecb(keys, data)
        assert enc.tobytes() == _lib_ecb(keys, data), f"ECB encrypt differs, {n} blocks"
        dec = o.tdes_ecb(keys, data, decrypt=True)
        assert dec.tobytes() == _lib_ecb(keys, data, decrypt=True), f"ECB decrypt, {n} blocks"


def check_library_cbc(o: Oracle):
    for i, n in enumerate(SIZES):
        keys = synth.key_triple(200 + i)
        iv = synth.iv64(200 + i)
        data = synth.random_bytes(200 + i, 8 * n)
        assert o.tdes_cbc_encrypt(keys, iv, data).tobytes() == _lib_cbc(keys, iv, data)
        assert o.tdes_cbc_decrypt(keys, iv, data).tobytes() == _lib_cbc(keys, iv, data, True)


def check_library_ctr(o: Oracle):
    for i, (n, ctr0) in enumerate([(1, 0), (33, 5), (16, 0xFFFFFFF0), (257, 123456)]):
        keys = synth.key_triple(300 + i)
        nonce = synth.nonce32(300 + i)
        data = synth.random_bytes(300 + i, 8 * n)
        ks = np.frombuffer(_lib_ecb(keys, _counter_blocks(nonce, ctr0, n)), dtype=np.uint8)
        assert (o.tdes_ctr(keys, nonce, ctr0, data) == (data ^ ks)).all()


def check_library_des(o: Oracle):
    # an 8-byte key makes the library's TripleDES single DES
    for i, n in enumerate(SIZES):
        key = synth.key_triple(250 + i)[:8]
        iv = synth.iv64(250 + i)
        data = synth.random_bytes(250 + i, 8 * n)
        assert o.des_ecb(key, data).tobytes() == _lib_ecb(key, data), f"DES ECB, {n} blocks"
        assert o.des_ecb(key, data, decrypt=True).tobytes() == _lib_ecb(key, data, decrypt=True)
        assert o.des_cbc_encrypt(key, iv, data).tobytes() == _lib_cbc(key, iv, data)
        assert o.des_cbc_decrypt(key, iv, data).tobytes() == _lib_cbc(key, iv, data, True)
        nonce = synth.nonce32(250 + i)
        ks = np.frombuffer(_lib_ecb(key, _counter_blocks(nonce, 3, n)), dtype=np.uint8)
        assert (o.des_ctr(key, nonce, 3, data) == (data ^ ks)).all()


def check_roundtrips(o: Oracle):
    for i, n in enumerate(SIZES):
        keys = synth.key_triple(400 + i)
        data = synth.random_bytes(400 + i, 8 * n)
        assert (o.tdes_ecb(keys, o.tdes_ecb(keys, data), decrypt=True) == data).all()
        assert (o.tdes_ecb(keys, o.tdes_ecb(keys, data, decrypt=True)) == data).all()
        iv = synth.iv64(400 + i)
        assert (o.tdes_cbc_decrypt(keys, iv, o.tdes_cbc_encrypt(keys, iv, data)) == data).all()
        assert (o.tdes_ctr(keys, 7, 9, o.tdes_ctr(keys, 7, 9, data)) == data).all()
        k1 = keys[:8]
        blk = data[:8]
        assert o.des_block(k1, o.des_block(k1, blk), decrypt=True) == blk.tobytes()


def check_ede3_degenerates_to_des(o: Oracle):
    for i in range(8):
        k = synth.key_triple(500 + i)[:8]
        blk = synth.random_bytes(500 + i, 8)
        for dec in (False, True):
            assert o.tdes_block(k * 3, blk, dec) == o.des_block(k, blk, dec)
    # D_K(E_K(x)) = x inside EDE3: K1 = K2 leaves E_K3, K2 = K3 leaves E_K1
    for i in range(4):
        ka, kb = synth.key_triple(510 + i)[:8], synth.key_triple(510 + i)[8:16]
        data = synth.random_bytes(510 + i, 8 * 9)
        for dec in (False, True):
            assert (o.tdes_ecb(ka + ka + kb, data, dec) == o.des_ecb(kb, data, dec)).all()
            assert (o.tdes_ecb(ka + kb + kb, data, dec) == o.des_ecb(ka, data, dec)).all()


def check_des_modes_are_the_block_cipher_in_modes(o: Oracle):
    # the single-DES modes are the EDE3 modes under (K, K, K), and each one
    # is built on des_block the way its definition says
    for i, n in enumerate([1, 5, 33]):
        k = synth.key_triple(520 + i)[:8]
        iv = synth.iv64(520 + i)
        data = synth.random_bytes(520 + i, 8 * n)
        assert (o.des_ecb(k, data) == o.tdes_ecb(k * 3, data)).all()
        assert (o.des_ctr(k, 11, 2, data) == o.tdes_ctr(k * 3, 11, 2, data)).all()
        assert (o.des_cbc_encrypt(k, iv, data) == o.tdes_cbc_encrypt(k * 3, iv, data)).all()
        assert (o.des_cbc_decrypt(k, iv, data) == o.tdes_cbc_decrypt(k * 3, iv, data)).all()
        blocks = [o.des_block(k, data[8 * j:8 * j + 8]) for j in range(n)]
        assert o.des_ecb(k, data).tobytes() == b"".join(blocks)
        assert (o.des_ecb(k, o.des_ecb(k, data), decrypt=True) == data).all()
        assert (o.des_cbc_decrypt(k, iv, o.des_cbc_encrypt(k, iv, data)) == data).all()


def check_complementation(o: Oracle):
    for i in range(8):
        keys = np.frombuffer(synth.key_triple(600 + i), dtype=np.uint8)
        blk = synth.random_bytes(600 + i, 8)
        c = np.frombuffer(o.des_block(keys[:8], blk), dtype=np.uint8)
        cc = np.frombuffer(o.des_block(~keys[:8], ~blk), dtype=np.uint8)
        assert (cc == ~c).all()
        c3 = np.frombuffer(o.tdes_block(keys, blk), dtype=np.uint8)
        cc3 = np.frombuffer(o.tdes_block(~keys, ~blk), dtype=np.uint8)
        assert (cc3 == ~c3).all()


def check_weak_keys(o: Oracle):
    # Keys made only of parity bits (all 0 or all 1 after PC-1) leave every
    # rotated half unchanged, so all 16 round keys are equal and encryption
    # is its own inverse.
    for kb in (b"\x01" * 8, b"\xfe" * 8, b"\x00" * 8, b"\xff" * 8):
        rk = o.des_round_keys(kb)
        assert (rk == rk[0]).all()
        for i in range(4):
            blk = synth.random_bytes(700 + i, 8)
            assert o.des_block(kb, o.des_block(kb, blk)) == blk.tobytes()


def check_parity_ignored(o: Oracle):
    keys = bytearray(synth.key_triple(800))
    blk = synth.random_bytes(800, 8)
    ref = o.tdes_block(bytes(keys), blk)
    for byte in range(24):
        k2 = bytearray(keys)
        k2[byte] ^= 0x01
        assert o.tdes_block(bytes(k2), blk) == ref
    k2 = bytearray(keys)
    k2[3] ^= 0x02  # a non-parity bit must matter
    assert o.tdes_block(bytes(k2), blk) != ref


def _read_worked_example():
    rows = []
    with open(os.path.join(GOLDEN, "sbox_worked_example.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                g, bits, row, col, expected = line.split()
                rows.append((int(g), int(bits, 2), int(row), int(col), int(expected)))
    return rows


def check_worked_example(o: Oracle):
    for g, six, _row, _col, expected in _read_worked_example():
        assert o.sbox(g, six) == expected


def check_sbox_rows_are_permutations(o: Oracle):
    for g in range(8):
        for outer in range(4):
            b1, b6 = outer >> 1, outer & 1
            vals = {o.sbox(g, (b1 << 5) | (mid << 1) | b6) for mid in range(16)}
            assert vals == set(range(16))


LIB_CHECKS = [check_library_ecb, check_library_cbc, check_library_ctr, check_library_des]
PROPERTY_CHECKS = [check_roundtrips, check_ede3_degenerates_to_des,
                   check_des_modes_are_the_block_cipher_in_modes, check_complementation,
                   check_weak_keys, check_parity_ignored, check_worked_example,
                   check_sbox_rows_are_permutations]


# --------------------------------------------------------- the real oracle

@needs_lib
@pytest.mark.parametrize("check", LIB_CHECKS, ids=lambda c: c.__name__)
def test_oracle_matches_independent_library(check):
    check(oracle.default())


@pytest.mark.parametrize("check", PROPERTY_CHECKS, ids=lambda c: c.__name__)
def test_oracle_properties(check):
    check(oracle.default())


@pytest.mark.skipif(shutil.which("openssl") is None, reason="no openssl CLI")
def test_oracle_matches_openssl_cli(tmp_path):
    keys = synth.key_triple(900)
    data = synth.random_bytes(900, 8 * 64)
    src = tmp_path / "p.bin"
    dst = tmp_path / "c.bin"
    src.write_bytes(data.tobytes())
    try:
        subprocess.run(["openssl", "enc", "-des-ede3", "-K", keys.hex(), "-nopad", "-nosalt",
                        "-in", str(src), "-out", str(dst)], check=True, capture_output=True,
                       timeout=60)
    except subprocess.CalledProcessError:
        pytest.skip("openssl has no DES-EDE3 in its default provider here")
    assert dst.read_bytes() == oracle.tdes_ecb(keys, data).tobytes()


def test_golden_vectors_reproduce():
    """The stored vectors (written by tests/golden/make_golden.py) still come out."""
    n = 0
    with open(os.path.join(GOLDEN, "tdes_vectors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            mode, _seed, keys, ivn, ctr0, data, out = line.split()
            keys, data, out = bytes.fromhex(keys), bytes.fromhex(data), bytes.fromhex(out)
            ivn, ctr0 = int(ivn, 16), int(ctr0)
            if mode == "ecb_enc":
                got = oracle.tdes_ecb(keys, data)
            elif mode == "ecb_dec":
                got = oracle.tdes_ecb(keys, data, decrypt=True)
            elif mode == "ctr":
                got = oracle.tdes_ctr(keys, ivn, ctr0, data)
            elif mode == "cbc_enc":
                got = oracle.tdes_cbc_encrypt(keys, ivn, data)
            else:
                got = oracle.tdes_cbc_decrypt(keys, ivn, data)
            assert got.tobytes() == out, line[:40]
            n += 1
    assert n == 15


@needs_lib
def test_golden_vectors_match_library():
    with open(os.path.join(GOLDEN, "tdes_vectors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            mode, _seed, keys, ivn, ctr0, data, out = line.split()
            keys, data, out = bytes.fromhex(keys), bytes.fromhex(data), bytes.fromhex(out)
            ivn, ctr0 = int(ivn, 16), int(ctr0)
            if mode in ("ecb_enc", "ecb_dec"):
                assert _lib_ecb(keys, data, mode == "ecb_dec") == out
            elif mode == "ctr":
                ks = _lib_ecb(keys, _counter_blocks(ivn, ctr0, len(data) // 8))
                assert bytes(a ^ b for a, b in zip(data, ks)) == out
            else:
                assert _lib_cbc(keys, ivn, data, mode == "cbc_dec") == out


def test_ctr_rejects_wrap():
    keys = synth.key_triple(1)
    with pytest.raises(ValueError):
        oracle.tdes_ctr(keys, 0, 0xFFFFFFFF, np.zeros(16, np.uint8))
    oracle.tdes_ctr(keys, 0, 0xFFFFFFFF, np.zeros(8, np.uint8))  # exactly fits


def test_parallel_matches_serial():
    keys = synth.key_triple(2)
    data = synth.random_bytes(2, 8 * 1001)
    for mode in ("ecb_enc", "ecb_dec", "ctr"):
        for th in (1, 3, 8):
            par = oracle.tdes_parallel(keys, data, mode, nonce=5, ctr0=17, threads=th)
            if mode == "ctr":
                ser = oracle.tdes_ctr(keys, 5, 17, data)
            else:
                ser = oracle.tdes_ecb(keys, data, decrypt=(mode == "ecb_dec"))
            assert (par == ser).all()


# ----------------------------------------------------------- planted mistakes
# (name, text in tdes_oracle.c, replacement).  Each is a plausible slip in
# reading the paper; at least one pin must reject every one of them.
MUTANTS = [
    ("row_reading_b6_b1", "int row = 2 * b[1] + b[6];", "int row = 2 * b[6] + b[1];"),
    ("column_bits_reversed", "int col = 8 * b[2] + 4 * b[3] + 2 * b[4] + b[5];",
     "int col = b[2] + 2 * b[3] + 4 * b[4] + 8 * b[5];"),
    ("last_swap_not_undone", "pre[j] = right[j];\n        pre[32 + j] = left[j];",
     "pre[j] = left[j];\n        pre[32 + j] = right[j];"),
    ("decrypt_keys_not_reversed", "round_key[decrypt ? 15 - r : r]", "round_key[r]"),
    ("rotation_not_cumulative", "for (int t = 0; t < shift_keys[r]; ++t) {",
     "for (int t = 0; t < (r == 0 ? 1 : 0); ++t) {"),
    ("lsb_first_bit_order", "int shift = 7 - (i - 1) % 8;\n        bits[i]",
     "int shift = (i - 1) % 8;\n        bits[i]"),
    ("ede_middle_stage_encrypts", "des_block(k->rk[1], 1, a, b);",
     "des_block(k->rk[1], 0, a, b);"),
    ("expansion_entry_swapped", "32, 1,  2,  3,  4,  5,  4,  5,", "1, 32,  2,  3,  4,  5,  4,  5,"),
    ("pc2_entry_swapped", "14, 17, 11, 24, 1,  5,", "17, 14, 11, 24, 1,  5,"),
    ("per_entry_swapped", "{16, 7,  20, 21,", "{7, 16,  20, 21,"),
    ("sbox_entry_swapped", "{14, 4, 13, 1, 2, 15,", "{4, 14, 13, 1, 2, 15,"),
    ("ctr_counter_low_half_first",
     "uint64_t counter = ((uint64_t)nonce << 32) | (uint32_t)(ctr0 + (uint32_t)i);",
     "uint64_t counter = ((uint64_t)(uint32_t)(ctr0 + (uint32_t)i) << 32) | nonce;"),
    ("cbc_dec_chains_plaintext", "memcpy(prev, cur, 8);", "memcpy(prev, out + 8 * i, 8);"),
    ("single_des_ignores_direction", "des_block(k->rk[0], decrypt, in, out);",
     "des_block(k->rk[0], 0, in, out);"),
]


def _run_all_checks(o: Oracle):
    failed = []
    for check in (LIB_CHECKS if _crypto() else []) + PROPERTY_CHECKS:
        try:
            check(o)
        except AssertionError:
            failed.append(check.__name__)
    return failed


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, mutant_dir):
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = os.path.join(mutant_dir, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.compile_oracle(path, os.path.join(mutant_dir, f"lib{name}.so"))
    failed = _run_all_checks(Oracle(lib))
    assert failed, f"mutant {name} passed every pin"


def test_real_oracle_passes_every_check():
    assert _run_all_checks(oracle.default()) == []


@pytest.mark.parametrize("threads", [1, 4])
def test_messages_entry_equals_per_message_calls(threads):
    """oracle_tdes_messages is a loop over the pinned mode functions: every
    message equals the same mode function called on it alone, whatever the
    thread split; bytes between messages are copied through."""
    rng = np.random.default_rng(41)
    keys = synth.key_triples(41, 5)
    n = 300
    nblocks = rng.integers(0, 12, n).astype(np.uint64)
    gaps = rng.integers(0, 3, n) * 8
    offset = np.concatenate([[0], np.cumsum(8 * nblocks + gaps)])[:-1].astype(np.uint64)
    data = synth.random_bytes(41, int(offset[-1] + 8 * nblocks[-1]) + 16)
    key_index = rng.integers(0, 5, n).astype(np.uint32)
    mode = rng.integers(0, 5, n).astype(np.uint8)
    iv = synth.u64s(41, n, synth.STREAM_IV)
    iv[mode == 2] &= np.uint64(0xFFFFFFFF000FFFFF)
    got = oracle.tdes_messages(keys, key_index, mode, iv, offset, nblocks, data, threads)
    want = data.copy()
    for i in range(n):
        k, s = keys[key_index[i]].tobytes(), slice(int(offset[i]), int(offset[i] + 8 * nblocks[i]))
        v, d = int(iv[i]), data[s]
        want[s] = [lambda: oracle.tdes_ecb(k, d), lambda: oracle.tdes_ecb(k, d, decrypt=True),
                   lambda: oracle.tdes_ctr(k, v >> 32, v & 0xFFFFFFFF, d),
                   lambda: oracle.tdes_cbc_decrypt(k, v, d),
                   lambda: oracle.tdes_cbc_encrypt(k, v, d)][int(mode[i])]()
    assert (got == want).all()


def test_messages_entry_rejects_bad_messages():
    keys = synth.key_triples(42, 2)
    data = synth.random_bytes(42, 64)
    one = dict(offset=[0], nblocks=[8], data=data)
    with pytest.raises(ValueError):
        oracle.tdes_messages(keys, [2], [0], [0], **one)             # key index out of range
    with pytest.raises(ValueError):
        oracle.tdes_messages(keys, [0], [5], [0], **one)             # no such mode
    with pytest.raises(ValueError):
        oracle.tdes_messages(keys, [0], [2], [0xFFFFFFFC], **one)    # counter passes 2^32
    with pytest.raises(ValueError):
        oracle.tdes_messages(keys, [0], [0], [0], [8], [8], data)    # past the buffer
