"""Large streaming, processed in place in one persistent launch: a 32 GiB
seeded buffer whose first 16 GiB is one single-key CTR stream and whose next
64 MiB are 2^20 messages of 64 bytes under 65536 key triples (modes
ECB 40% / CTR 30% / CBC-decrypt 20% / CBC-encrypt 10%).  Every message, and
2^20 seeded random blocks plus windows of the CTR stream, are recomputed by
the oracle (on all host cores) from inputs regenerated by the counter-based
generator; bytes outside the processed ranges are unchanged."""
import os

import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2007_10752_gb300.workloads import (STREAM_BYTES, STREAM_N_KEYS as N_KEYS,
                                              STREAM_N_SMALL as N_SMALL, STREAM_SEED as SEED,
                                              STREAM_TOTAL as TOTAL, build_streaming)


def _oracle(mode, keys, iv, data):
    if mode == 0:
        return oracle.tdes_ecb(keys, data)
    if mode == 2:
        return oracle.tdes_ctr(keys, iv >> 32, iv & 0xFFFFFFFF, data)
    if mode == 3:
        return oracle.tdes_cbc_decrypt(keys, iv, data)
    return oracle.tdes_cbc_encrypt(keys, iv, data)


def test_device_fill_matches_host_generator(cuda_lib):
    t = torch.empty(8 * 100003, dtype=torch.uint8, device="cuda")
    synth.fill_device(t, 77, start_byte=8 * 12345)
    torch.cuda.synchronize()
    assert (t.cpu().numpy() == synth.random_bytes(77, t.numel(), start_byte=8 * 12345)).all()


def test_large_streaming_every_message(cuda_lib):
    T = cuda_lib
    import torch as _t
    buf, kt, d, keys, nonce = build_streaming(_t, T)
    b = T.Batch(kt, d)
    assert (b.status == 0).all()
    b.launch_graph()
    torch.cuda.synchronize()
    rng = np.random.default_rng(SEED)
    threads = max(1, min(64, os.cpu_count() or 1))
    # every 64-byte message
    e = d[1:]
    got = buf[STREAM_BYTES:STREAM_BYTES + 64 * N_SMALL].cpu().numpy()
    want = oracle.tdes_messages(keys, e["key_index"], e["mode"].astype(np.uint8),
                                e["iv_or_ctr"], 64 * np.arange(N_SMALL, dtype=np.uint64),
                                np.full(N_SMALL, 8, dtype=np.uint64),
                                synth.random_bytes(SEED, 64 * N_SMALL, start_byte=STREAM_BYTES),
                                threads)
    bad = np.nonzero((got != want).reshape(N_SMALL, 64).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} messages differ, first {bad[:5]}"
    # 2^20 seeded random blocks of the CTR stream, each a one-block CTR message
    nblk = STREAM_BYTES // 8
    pos = np.unique(rng.integers(0, nblk, 1 << 20, dtype=np.uint64))
    gotb = buf.view(torch.int64)[torch.from_numpy(pos.astype(np.int64)).cuda()].cpu().numpy()
    wantb = oracle.tdes_messages(keys, np.full(pos.size, N_KEYS, dtype=np.uint32),
                                 np.full(pos.size, 2, dtype=np.uint8),
                                 (np.uint64(nonce) << np.uint64(32)) | pos,
                                 8 * np.arange(pos.size, dtype=np.uint64),
                                 np.ones(pos.size, dtype=np.uint64),
                                 synth.blocks_at(SEED, pos).reshape(-1), threads)
    assert (gotb.view(np.uint8) == wantb).all(), "CTR stream block"
    # CTR stream windows (counter = block index from 0)
    kctr = keys[N_KEYS].tobytes()
    nblk = STREAM_BYTES // 8
    for s in [0, nblk - 512] + [int(x) for x in rng.integers(0, nblk - 512, 30)]:
        data = synth.random_bytes(SEED, 4096, start_byte=8 * s)
        want = oracle.tdes_ctr(kctr, nonce, s, data)
        assert (buf[8 * s:8 * s + 4096].cpu().numpy() == want).all(), f"CTR window {s}"
    # untouched beyond the processed ranges
    tail = STREAM_BYTES + 64 * N_SMALL
    assert (buf[tail:tail + 4096].cpu().numpy() ==
            synth.random_bytes(SEED, 4096, start_byte=tail)).all()
    assert (buf[TOTAL - 4096:].cpu().numpy() ==
            synth.random_bytes(SEED, 4096, start_byte=TOTAL - 4096)).all()
    del buf
    torch.cuda.empty_cache()
