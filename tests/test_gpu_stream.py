"""Large streaming, processed in place in one persistent launch: a 32 GiB
seeded buffer whose first 16 GiB is one single-key CTR stream and whose next
64 MiB are 2^20 messages of 64 bytes under 65536 key triples (modes
ECB 40% / CTR 30% / CBC-decrypt 20% / CBC-encrypt 10%).  Sampled messages
and CTR windows are recomputed by the oracle from inputs regenerated by the
counter-based generator; bytes outside the processed ranges are unchanged."""
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


def test_large_streaming_sampled(cuda_lib):
    T = cuda_lib
    import torch as _t
    buf, kt, d, keys, nonce = build_streaming(_t, T)
    b = T.Batch(kt, d)
    assert (b.status == 0).all()
    b.launch_graph()
    torch.cuda.synchronize()
    rng = np.random.default_rng(SEED)
    # 64-byte messages
    pick = np.sort(rng.choice(N_SMALL, 3000, replace=False))
    got = buf[STREAM_BYTES:STREAM_BYTES + 64 * N_SMALL].view(-1, 64)[torch.from_numpy(pick).cuda()]
    got = got.cpu().numpy()
    for row, i in enumerate(pick):
        e = d[1 + i]
        data = synth.random_bytes(SEED, 64, start_byte=STREAM_BYTES + 64 * int(i))
        want = _oracle(int(e["mode"]), keys[int(e["key_index"])].tobytes(), int(e["iv_or_ctr"]), data)
        assert (got[row] == want).all(), f"message {i} mode {e['mode']}"
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
