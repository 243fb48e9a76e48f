"""ctypes front end of the C oracle (test infrastructure only).

Builds ``oracle/libtdes_oracle.so`` with gcc on first use (or via
``build()``), then exposes numpy-in/numpy-out wrappers.  Byte buffers are
``numpy.uint8`` arrays whose length is a multiple of 8; keys are 24-byte
K1||K2||K3 strings.

``Oracle(path)`` loads any build of ``tdes_oracle.c``; the test suite uses it
to load deliberately mutated copies and check that the pins catch them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "tdes_oracle.c")
HEADER = os.path.join(_HERE, "tdes_oracle.h")
_LIB = os.path.join(_HERE, "libtdes_oracle.so")
_lock = threading.Lock()
_default = None


def compile_oracle(src: str, out: str) -> str:
    """gcc -O2, plain C11, no target-specific flags (same on x86_64 and aarch64)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-I", _HERE,
                           "-o", tmp, src, "-lpthread"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(SOURCE), os.path.getmtime(HEADER))
    if force or stale:
        compile_oracle(SOURCE, _LIB)
    return _LIB


_u8p = ctypes.POINTER(ctypes.c_uint8)


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_u8p)


def _keys(keys) -> np.ndarray:
    k = _u8(keys).reshape(-1)
    if k.size != 24:
        raise ValueError("a key triple is 24 bytes (K1||K2||K3)")
    return k


def _key8(key) -> np.ndarray:
    k = _u8(key).reshape(-1)
    if k.size != 8:
        raise ValueError("a DES key is 8 bytes")
    return k


def _blocks(data) -> np.ndarray:
    d = _u8(data).reshape(-1)
    if d.size % 8:
        raise ValueError("buffers hold whole 8-byte blocks")
    return d


class Oracle:
    """One loaded build of the C oracle."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u8p = _u8p
        lib.oracle_des_round_keys.argtypes = [u8p, u8p]
        lib.oracle_sbox.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_sbox.restype = ctypes.c_int
        lib.oracle_des_block.argtypes = [u8p, ctypes.c_int, u8p, u8p]
        lib.oracle_tdes_block.argtypes = [u8p, ctypes.c_int, u8p, u8p]
        lib.oracle_tdes_ecb.argtypes = [u8p, ctypes.c_int, u8p, u8p, ctypes.c_uint64]
        lib.oracle_tdes_ctr.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint32, u8p, u8p,
                                        ctypes.c_uint64]
        lib.oracle_tdes_ctr.restype = ctypes.c_int
        lib.oracle_tdes_cbc_encrypt.argtypes = [u8p, ctypes.c_uint64, u8p, u8p, ctypes.c_uint64]
        lib.oracle_tdes_cbc_decrypt.argtypes = [u8p, ctypes.c_uint64, u8p, u8p, ctypes.c_uint64]
        lib.oracle_des_ecb.argtypes = [u8p, ctypes.c_int, u8p, u8p, ctypes.c_uint64]
        lib.oracle_des_ctr.argtypes = [u8p, ctypes.c_uint32, ctypes.c_uint32, u8p, u8p,
                                       ctypes.c_uint64]
        lib.oracle_des_ctr.restype = ctypes.c_int
        lib.oracle_des_cbc_encrypt.argtypes = [u8p, ctypes.c_uint64, u8p, u8p, ctypes.c_uint64]
        lib.oracle_des_cbc_decrypt.argtypes = [u8p, ctypes.c_uint64, u8p, u8p, ctypes.c_uint64]
        lib.oracle_tdes_parallel.argtypes = [u8p, ctypes.c_int, ctypes.c_uint32,
                                             ctypes.c_uint32, u8p, u8p, ctypes.c_uint64,
                                             ctypes.c_int]
        lib.oracle_tdes_parallel.restype = ctypes.c_int
        vp = ctypes.c_void_p
        lib.oracle_tdes_messages.argtypes = [vp, ctypes.c_uint32, vp, vp, vp, vp, vp, vp, vp,
                                             ctypes.c_uint64, ctypes.c_int]
        lib.oracle_tdes_messages.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    # Sec. III-A
    def des_round_keys(self, key) -> np.ndarray:
        """16 x 48 round-key bits (one uint8 per bit) of one 8-byte key."""
        k = _u8(key).reshape(-1)
        if k.size != 8:
            raise ValueError("a DES key is 8 bytes")
        out = np.zeros((16, 48), dtype=np.uint8)
        self.lib.oracle_des_round_keys(_ptr(k), _ptr(out))
        return out

    # Sec. III-B, S-box step
    def sbox(self, g: int, six: int) -> int:
        return int(self.lib.oracle_sbox(int(g), int(six)))

    # Sec. III-B
    def des_block(self, key, block, decrypt: bool = False) -> bytes:
        k, b = _u8(key).reshape(-1), _u8(block).reshape(-1)
        if k.size != 8 or b.size != 8:
            raise ValueError("key and block are 8 bytes each")
        out = np.zeros(8, dtype=np.uint8)
        self.lib.oracle_des_block(_ptr(k), int(decrypt), _ptr(b), _ptr(out))
        return out.tobytes()

    # Sec. III-B, 3DES equations
    def tdes_block(self, keys, block, decrypt: bool = False) -> bytes:
        k, b = _keys(keys), _u8(block).reshape(-1)
        if b.size != 8:
            raise ValueError("a block is 8 bytes")
        out = np.zeros(8, dtype=np.uint8)
        self.lib.oracle_tdes_block(_ptr(k), int(decrypt), _ptr(b), _ptr(out))
        return out.tobytes()

    def tdes_ecb(self, keys, data, decrypt: bool = False) -> np.ndarray:
        k, d = _keys(keys), _blocks(data)
        out = np.empty_like(d)
        self.lib.oracle_tdes_ecb(_ptr(k), int(decrypt), _ptr(d), _ptr(out), d.size // 8)
        return out

    def tdes_ctr(self, keys, nonce: int, ctr0: int, data) -> np.ndarray:
        k, d = _keys(keys), _blocks(data)
        out = np.empty_like(d)
        rc = self.lib.oracle_tdes_ctr(_ptr(k), nonce & 0xFFFFFFFF, ctr0 & 0xFFFFFFFF, _ptr(d),
                                      _ptr(out), d.size // 8)
        if rc != 0:
            raise ValueError("CTR counter would wrap past 2^32")
        return out

    def tdes_cbc_encrypt(self, keys, iv: int, data) -> np.ndarray:
        k, d = _keys(keys), _blocks(data)
        out = np.empty_like(d)
        self.lib.oracle_tdes_cbc_encrypt(_ptr(k), iv & (2**64 - 1), _ptr(d), _ptr(out),
                                         d.size // 8)
        return out

    def tdes_cbc_decrypt(self, keys, iv: int, data) -> np.ndarray:
        k, d = _keys(keys), _blocks(data)
        out = np.empty_like(d)
        self.lib.oracle_tdes_cbc_decrypt(_ptr(k), iv & (2**64 - 1), _ptr(d), _ptr(out),
                                         d.size // 8)
        return out

    # single DES (one pass of Sec. III-B) in the same modes
    def des_ecb(self, key, data, decrypt: bool = False) -> np.ndarray:
        k, d = _key8(key), _blocks(data)
        out = np.empty_like(d)
        self.lib.oracle_des_ecb(_ptr(k), int(decrypt), _ptr(d), _ptr(out), d.size // 8)
        return out

    def des_ctr(self, key, nonce: int, ctr0: int, data) -> np.ndarray:
        k, d = _key8(key), _blocks(data)
        out = np.empty_like(d)
        rc = self.lib.oracle_des_ctr(_ptr(k), nonce & 0xFFFFFFFF, ctr0 & 0xFFFFFFFF, _ptr(d),
                                     _ptr(out), d.size // 8)
        if rc != 0:
            raise ValueError("CTR counter would wrap past 2^32")
        return out

    def des_cbc_encrypt(self, key, iv: int, data) -> np.ndarray:
        k, d = _key8(key), _blocks(data)
        out = np.empty_like(d)
        self.lib.oracle_des_cbc_encrypt(_ptr(k), iv & (2**64 - 1), _ptr(d), _ptr(out),
                                        d.size // 8)
        return out

    def des_cbc_decrypt(self, key, iv: int, data) -> np.ndarray:
        k, d = _key8(key), _blocks(data)
        out = np.empty_like(d)
        self.lib.oracle_des_cbc_decrypt(_ptr(k), iv & (2**64 - 1), _ptr(d), _ptr(out),
                                        d.size // 8)
        return out

    def tdes_parallel(self, keys, data, mode: str = "ecb_enc", nonce: int = 0, ctr0: int = 0,
                      threads: int = 1) -> np.ndarray:
        """ECB/CTR split over ``threads`` host threads (CPU-baseline timing only)."""
        k, d = _keys(keys), _blocks(data)
        out = np.empty_like(d)
        m = {"ecb_enc": 0, "ecb_dec": 1, "ctr": 2}[mode]
        rc = self.lib.oracle_tdes_parallel(_ptr(k), m, nonce & 0xFFFFFFFF, ctr0 & 0xFFFFFFFF,
                                           _ptr(d), _ptr(out), d.size // 8, int(threads))
        if rc != 0:
            raise ValueError("bad arguments to oracle_tdes_parallel")
        return out


    def tdes_messages(self, keys, key_index, mode, iv_or_ctr, offset, nblocks, data,
                      threads: int = 1) -> np.ndarray:
        """Independent messages under their own triples and modes (see
        oracle_tdes_messages); returns a copy of ``data`` with every message
        replaced by its result."""
        k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint8).reshape(-1, 24))
        ki = np.ascontiguousarray(key_index, dtype=np.uint32)
        md = np.ascontiguousarray(mode, dtype=np.uint8)
        iv = np.ascontiguousarray(np.asarray(iv_or_ctr).astype(np.uint64))
        off = np.ascontiguousarray(offset, dtype=np.uint64)
        nb = np.ascontiguousarray(nblocks, dtype=np.uint64)
        d = np.ascontiguousarray(data, dtype=np.uint8)
        n = ki.size
        if not (md.size == iv.size == off.size == nb.size == n):
            raise ValueError("one key index, mode, IV, offset and length per message")
        if n and int((off + 8 * nb).max()) > d.size:
            raise ValueError("a message extends past the buffer")
        out = d.copy()
        rc = self.lib.oracle_tdes_messages(k.ctypes.data, k.shape[0], ki.ctypes.data,
                                           md.ctypes.data, iv.ctypes.data, off.ctypes.data,
                                           nb.ctypes.data, d.ctypes.data, out.ctypes.data, n,
                                           int(threads))
        if rc != 0:
            raise ValueError("bad message for oracle_tdes_messages")
        return out


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def des_round_keys(key):
    return default().des_round_keys(key)


def sbox(g, six):
    return default().sbox(g, six)


def des_block(key, block, decrypt=False):
    return default().des_block(key, block, decrypt)


def tdes_block(keys, block, decrypt=False):
    return default().tdes_block(keys, block, decrypt)


def tdes_ecb(keys, data, decrypt=False):
    return default().tdes_ecb(keys, data, decrypt)


def tdes_ctr(keys, nonce, ctr0, data):
    return default().tdes_ctr(keys, nonce, ctr0, data)


def tdes_cbc_encrypt(keys, iv, data):
    return default().tdes_cbc_encrypt(keys, iv, data)


def tdes_cbc_decrypt(keys, iv, data):
    return default().tdes_cbc_decrypt(keys, iv, data)


def tdes_parallel(keys, data, mode="ecb_enc", nonce=0, ctr0=0, threads=1):
    return default().tdes_parallel(keys, data, mode, nonce, ctr0, threads)


def tdes_messages(keys, key_index, mode, iv_or_ctr, offset, nblocks, data, threads=1):
    return default().tdes_messages(keys, key_index, mode, iv_or_ctr, offset, nblocks, data,
                                   threads)


def des_ecb(key, data, decrypt=False):
    return default().des_ecb(key, data, decrypt)


def des_ctr(key, nonce, ctr0, data):
    return default().des_ctr(key, nonce, ctr0, data)


def des_cbc_encrypt(key, iv, data):
    return default().des_cbc_encrypt(key, iv, data)


def des_cbc_decrypt(key, iv, data):
    return default().des_cbc_decrypt(key, iv, data)
