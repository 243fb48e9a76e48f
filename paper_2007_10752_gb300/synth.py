"""Seeded synthetic inputs for 3DES-EDE3 workloads.

This module holds no cipher arithmetic: it only draws bytes, keys, IVs,
nonces, message lengths and modes.  Both the CUDA path's tests/benchmark and
the CPU oracle's tests take their inputs from here, so the same seed gives
the same bytes on both sides and on every machine.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in its counter form: the
i-th output of the stream with seed ``s`` is ``mix(s + (i + 1) * gamma)``
with gamma = 0x9E3779B97F4A7C15 and the published two-multiply finaliser.
Being counter-based, any word of a stream can be regenerated on its own,
which is how full-size buffers are sampled without keeping a copy.

Byte order: a byte buffer is the concatenation of its 64-bit words stored
little-endian (word i covers bytes 8i..8i+7).  A cipher block is an 8-byte
big-endian string, so the block value is the byte-swapped word; nothing here
cares, the bytes are the input.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

# Stream labels: each kind of draw uses its own substream of the seed.
STREAM_PAYLOAD = 1
STREAM_KEYS = 2
STREAM_IV = 3
STREAM_LENGTH = 4
STREAM_MODE = 5
STREAM_KEYPICK = 6
STREAM_ARRIVAL = 7
STREAM_SIZECLASS = 8


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, index) -> np.ndarray:
    """Outputs ``index`` (scalar or array of uint64) of the stream seeded ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + (idx + np.uint64(1)) * GAMMA
        return _mix(np.asarray(z, dtype=np.uint64))


def substream(seed: int, label: int) -> int:
    """Seed of the substream ``label`` of ``seed`` (itself a SplitMix64 output)."""
    return int(splitmix64_at(seed, np.uint64(label)))


def words(seed: int, start: int, count: int, stream: int = STREAM_PAYLOAD) -> np.ndarray:
    """``count`` consecutive uint64 words starting at word ``start``."""
    s = substream(seed, stream)
    idx = np.arange(start, start + count, dtype=np.uint64)
    return splitmix64_at(s, idx)


def random_bytes(seed: int, nbytes: int, stream: int = STREAM_PAYLOAD,
                 start_byte: int = 0, out: np.ndarray | None = None,
                 chunk_words: int = 1 << 22) -> np.ndarray:
    """Uniform random bytes [start_byte, start_byte + nbytes) of a payload stream.

    ``start_byte`` and ``nbytes`` are multiples of 8.  Generated in chunks so
    that a 1 GiB buffer needs no temporaries beyond a few tens of MiB.
    """
    if nbytes % 8 or start_byte % 8:
        raise ValueError("payload streams are drawn in whole 8-byte words")
    if out is None:
        out = np.empty(nbytes, dtype=np.uint8)
    w = out.view("<u8") if nbytes else np.empty(0, "<u8")
    s = substream(seed, stream)
    first = start_byte // 8
    n = nbytes // 8
    for c0 in range(0, n, chunk_words):
        c1 = min(n, c0 + chunk_words)
        idx = np.arange(first + c0, first + c1, dtype=np.uint64)
        w[c0:c1] = splitmix64_at(s, idx)
    return out


def blocks_at(seed: int, block_indices, stream: int = STREAM_PAYLOAD,
              start_byte: int = 0) -> np.ndarray:
    """The 8-byte blocks at ``block_indices`` of ``random_bytes(seed, ..)``, as (k, 8) uint8."""
    s = substream(seed, stream)
    idx = np.asarray(block_indices, dtype=np.uint64) + np.uint64(start_byte // 8)
    w = splitmix64_at(s, idx).astype("<u8")
    return w.view(np.uint8).reshape(-1, 8)


def _odd_parity(b: np.ndarray) -> np.ndarray:
    """Set each byte's least significant bit so that the byte has odd parity."""
    hi = b & np.uint8(0xFE)
    ones = np.unpackbits(hi[..., None], axis=-1).sum(axis=-1)
    return hi | ((ones + 1) % 2).astype(np.uint8)


def key_triples(seed: int, count: int, first: int = 0) -> np.ndarray:
    """``count`` key triples (K1||K2||K3, 24 bytes each) as a (count, 24) uint8 array.

    Each key is a uniform 64-bit word with every byte's low bit set for odd
    parity (the parity bits are ignored by the cipher's PC-1).
    """
    w = words(seed, 3 * first, 3 * count, STREAM_KEYS).astype("<u8")
    b = w.view(np.uint8).reshape(count, 24)
    return _odd_parity(b)


def key_triple(seed: int, index: int = 0) -> bytes:
    return key_triples(seed, 1, index)[0].tobytes()


def u64s(seed: int, count: int, stream: int, first: int = 0) -> np.ndarray:
    return words(seed, first, count, stream)


def uniform01(seed: int, count: int, stream: int, first: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each word."""
    w = words(seed, first, count, stream)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def iv64(seed: int, index: int = 0) -> int:
    return int(words(seed, index, 1, STREAM_IV)[0])


def nonce32(seed: int, index: int = 0) -> int:
    return int(words(seed, index, 1, STREAM_IV)[0] >> np.uint64(32))


def log_uniform_lengths(seed: int, count: int, lo: int, hi: int, stream: int = STREAM_LENGTH,
                        first: int = 0) -> np.ndarray:
    """Lengths exp(U(ln lo, ln hi)) rounded down to a multiple of 8, at least ``lo``."""
    u = uniform01(seed, count, stream, first)
    x = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    n = (np.floor(x).astype(np.int64) // 8) * 8
    return np.clip(n, lo, hi).astype(np.int64)


def categorical(seed: int, count: int, probs, stream: int, first: int = 0) -> np.ndarray:
    """Indices drawn with the given probabilities (inverse CDF of a uniform draw)."""
    p = np.asarray(probs, dtype=np.float64)
    cdf = np.cumsum(p / p.sum())
    u = uniform01(seed, count, stream, first)
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(p) - 1).astype(np.int64)


def fill_device(tensor, seed: int, stream: int = STREAM_PAYLOAD, start_byte: int = 0) -> None:
    """Fill a CUDA uint8 tensor with ``random_bytes(seed, tensor.numel(), stream, start_byte)``.

    Runs the same SplitMix64 words on the GPU (libtdes_tools.so) for inputs
    too large to draw on the host; asynchronous on the current torch stream.
    """
    import ctypes
    import os

    import torch
    n = tensor.numel()
    if n % 8 or start_byte % 8:
        raise ValueError("payload streams are drawn in whole 8-byte words")
    lib = ctypes.CDLL(os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtdes_tools.so"))
    lib.tdes_tools_fill_splitmix64.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.c_void_p]
    rc = lib.tdes_tools_fill_splitmix64(tensor.data_ptr(), n // 8, substream(seed, stream),
                                        start_byte // 8, torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise RuntimeError(f"device fill failed: {rc}")
