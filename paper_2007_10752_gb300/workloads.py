"""Seeded synthetic workloads of the benchmark and the tests, as device
buffers plus batch descriptors (no cipher arithmetic here).

* ``build_batched``: 4096 messages, lengths log-uniform 64 B .. 4 MiB
  (multiples of 8), own key triple each, modes ECB 40% / CTR 30% /
  CBC-decrypt 20% / CBC-encrypt 10%, seeded IVs; out of place.
* ``build_streaming``: one 32 GiB buffer processed in place: a 16 GiB
  single-key CTR stream at offset 0, then 2^20 messages of 64 bytes under
  65536 key triples with the same mode mix.  The payload is drawn on the
  device with the same SplitMix64 words as ``synth.random_bytes``.
* ``uniform_arrays_device``: per-message key index, mode and IV arrays for
  the second 16 GiB of that buffer read as 2^28 messages of 64 bytes, drawn
  on the device with the same words as the host draws above (message i gets
  word i of each stream, so the first 2^20 match ``build_streaming``).
"""
from __future__ import annotations

import numpy as np

from . import synth

BATCH_SEED = 3
STREAM_SEED = 5
STREAM_TOTAL = 32 << 30
STREAM_BYTES = 16 << 30
STREAM_N_SMALL = 1 << 20
STREAM_N_KEYS = 65536
STREAM_N_UNIFORM = 1 << 28  # the second 16 GiB as 64-byte messages
MODE_MIX = (0.4, 0.3, 0.2, 0.1)  # ECB encrypt, CTR, CBC-decrypt, CBC-encrypt


def _modes(seed, n):
    return np.array([0, 2, 3, 4], dtype=np.uint32)[
        synth.categorical(seed, n, list(MODE_MIX), synth.STREAM_MODE)]


def build_batched(torch, tdes, seed=BATCH_SEED, n=4096):
    """Returns (src, dst, key table, descriptor array, lengths, modes)."""
    lens = synth.log_uniform_lengths(seed, n, 64, 4 << 20)
    modes = _modes(seed, n)
    keys = synth.key_triples(seed, n)
    ivs = synth.u64s(seed, n, synth.STREAM_IV)
    offs = np.concatenate([[0], np.cumsum((lens + 15) // 16 * 16)])[:-1].astype(np.uint64)
    total = int(offs[-1]) + int(lens[-1]) + 16
    src = torch.from_numpy(synth.random_bytes(seed, (total + 7) // 8 * 8)).cuda()
    dst = torch.empty_like(src)
    d = np.zeros(n, dtype=tdes.DESC_DTYPE)
    d["mode"] = modes
    d["key_index"] = np.arange(n, dtype=np.uint32)
    d["iv_or_ctr"] = np.where(modes == 2, ivs & np.uint64(0xFFFFFFFF00000000), ivs)
    d["in_ptr"] = np.uint64(src.data_ptr()) + offs
    d["out_ptr"] = np.uint64(dst.data_ptr()) + offs
    d["nbytes"] = lens.astype(np.uint64)
    return src, dst, tdes.KeyTable(keys), d, lens, modes


def build_streaming(torch, tdes, seed=STREAM_SEED, total=STREAM_TOTAL, stream_bytes=STREAM_BYTES,
                    n_small=STREAM_N_SMALL, n_keys=STREAM_N_KEYS):
    """Returns (buffer, key table, descriptor array, keys, CTR nonce)."""
    buf = torch.empty(total, dtype=torch.uint8, device="cuda")
    synth.fill_device(buf, seed)
    keys = synth.key_triples(seed, n_keys + 1)  # the last triple keys the CTR stream
    kt = tdes.KeyTable(keys)
    base = buf.data_ptr()
    d = np.zeros(n_small + 1, dtype=tdes.DESC_DTYPE)
    nonce = synth.nonce32(seed)
    d[0] = (tdes.MODE_CTR, n_keys, nonce << 32, base, base, stream_bytes)
    offs = stream_bytes + 64 * np.arange(n_small, dtype=np.uint64)
    modes = _modes(seed, n_small)
    ivs = synth.u64s(seed, n_small, synth.STREAM_IV)
    d["mode"][1:] = modes
    d["key_index"][1:] = (synth.u64s(seed, n_small, synth.STREAM_KEYPICK)
                          % np.uint64(n_keys)).astype(np.uint32)
    d["iv_or_ctr"][1:] = np.where(modes == 2, ivs & np.uint64(0xFFFFFFFF00000000), ivs)
    d["in_ptr"][1:] = np.uint64(base) + offs
    d["out_ptr"][1:] = np.uint64(base) + offs
    d["nbytes"][1:] = 64
    return buf, kt, d, keys, nonce


def uniform_arrays_device(torch, seed, n, n_keys, first=0):
    """(key_index int32, mode uint8, iv_or_ctr int64) CUDA tensors for messages
    first .. first + n - 1: key pick = word % n_keys (n_keys a power of two,
    so the low bits of the word), mode from MODE_MIX by the inverse CDF of the
    word's top 53 bits (as ``synth.categorical``), IV = the word of the IV
    stream (CTR keeps its nonce half, counter 0)."""
    if n_keys & (n_keys - 1):
        raise ValueError("device key picks need a power-of-two key count")

    def words(stream):
        w = torch.empty(n, dtype=torch.int64, device="cuda")
        synth.fill_device(w.view(torch.uint8), seed, stream, 8 * first)
        return w

    key_index = uniform_key_index(torch, words(synth.STREAM_KEYPICK), n_keys)
    mode = uniform_mode(torch, words(synth.STREAM_MODE))
    return key_index, mode, uniform_iv(torch, words(synth.STREAM_IV), mode)


def uniform_key_index(torch, w, n_keys):
    return (w & (n_keys - 1)).to(torch.int32)


def uniform_mode(torch, w):
    u = ((w >> 11) & ((1 << 53) - 1)).to(torch.float64) * (1.0 / (1 << 53))
    p = np.asarray(MODE_MIX, dtype=np.float64)
    idx = torch.zeros(w.shape[0], dtype=torch.int64, device=w.device)
    for c in np.cumsum(p / p.sum()):
        idx += (u >= float(c)).to(torch.int64)
    del u
    idx.clamp_(max=len(p) - 1)
    return torch.tensor([0, 2, 3, 4], dtype=torch.uint8, device=w.device)[idx]


def uniform_iv(torch, w, mode):
    return torch.where(mode == 2, w & -(1 << 32), w)


def uniform_expected_fields(seed, i, n_keys):
    """Host copy of message i's (key index, mode, iv_or_ctr) as drawn by
    uniform_arrays_device."""
    k, m, v = uniform_expected_arrays(seed, np.array([i], dtype=np.uint64), n_keys)
    return int(k[0]), int(m[0]), int(v[0])


def uniform_expected_arrays(seed, idx, n_keys):
    """(key index, mode, iv_or_ctr) arrays of the messages at indices ``idx``
    (any order), as drawn by uniform_arrays_device: word idx of each stream."""
    idx = np.asarray(idx, dtype=np.uint64)
    key = (synth.splitmix64_at(synth.substream(seed, synth.STREAM_KEYPICK), idx)
           % np.uint64(n_keys)).astype(np.uint32)
    u = (synth.splitmix64_at(synth.substream(seed, synth.STREAM_MODE), idx)
         >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    p = np.asarray(MODE_MIX, dtype=np.float64)
    cat = np.minimum(np.searchsorted(np.cumsum(p / p.sum()), u, side="right"), len(p) - 1)
    mode = np.array([0, 2, 3, 4], dtype=np.uint8)[cat]
    iv = synth.splitmix64_at(synth.substream(seed, synth.STREAM_IV), idx)
    iv = np.where(mode == 2, iv & np.uint64(0xFFFFFFFF00000000), iv)
    return key, mode, iv

