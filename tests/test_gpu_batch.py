"""Batches through the C ABI: every message of a mixed batch (own key triple,
own mode, uneven length, some in place, some only 8-byte aligned) equals the
CPU oracle on that message alone, bit for bit, and equals the same message
run alone on the GPU (alone vs in the mix); graph replay and every launch
shape give identical bytes; invalid descriptors are rejected and skipped."""
import os

import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCPU = max(1, min(16, os.cpu_count() or 1))
MODES = ["ecb_enc", "ecb_dec", "ctr", "cbc_dec", "cbc_enc"]


def oracle_msg(mode, keys, iv, data):
    if mode == 0:
        return oracle.tdes_ecb(keys, data)
    if mode == 1:
        return oracle.tdes_ecb(keys, data, decrypt=True)
    if mode == 2:
        return oracle.tdes_ctr(keys, iv >> 32, iv & 0xFFFFFFFF, data)
    if mode == 3:
        return oracle.tdes_cbc_decrypt(keys, iv, data)
    return oracle.tdes_cbc_encrypt(keys, iv, data)


def build_mix(seed, n_msgs, n_keys, max_blocks, in_place_frac=0.3):
    """Messages laid out in one device arena; returns (arena, msgs, keys)."""
    rng = np.random.default_rng(seed)
    keys = synth.key_triples(seed, n_keys)
    sizes = []
    for i in range(n_msgs):
        r = rng.random()
        if r < 0.35:
            nb = int(rng.integers(0, 33))          # small: scalar path (0 = empty)
        elif r < 0.8:
            nb = int(rng.integers(33, 3000))       # one to three tiles, ragged
        else:
            nb = int(rng.integers(3000, max_blocks))
        sizes.append(nb)
    msgs, off = [], 0
    for i, nb in enumerate(sizes):
        mode = int(rng.integers(0, 5))
        key = int(rng.integers(0, n_keys))
        iv = int(synth.words(seed, i, 1, synth.STREAM_IV)[0])
        if mode == 2:
            iv = (iv & 0xFFFFFFFF00000000) | int(rng.integers(0, 1 << 20))
        in_place = rng.random() < in_place_frac
        align = 8 if rng.random() < 0.3 else 16
        off = (off + 15) // 16 * 16 + (8 if align == 8 else 0)
        in_off = off
        off += 8 * nb + 16
        out_off = in_off if in_place else (off + 15) // 16 * 16 + (8 if align == 8 else 0)
        if not in_place:
            off = out_off + 8 * nb + 16
        data = synth.random_bytes(seed * 1000 + i, 8 * nb)
        msgs.append(dict(mode=mode, key=key, iv=iv, nb=nb, in_off=in_off, out_off=out_off,
                         data=data))
    arena = torch.zeros(off + 64, dtype=torch.uint8, device="cuda")
    for m in msgs:
        if m["nb"]:
            arena[m["in_off"]:m["in_off"] + 8 * m["nb"]].copy_(torch.from_numpy(m["data"]))
    return arena, msgs, keys


def entries_for(arena, msgs):
    base = arena.data_ptr()
    return [(m["mode"], m["key"], m["iv"], base + m["in_off"], base + m["out_off"], 8 * m["nb"])
            for m in msgs]


def outputs(arena, msgs):
    torch.cuda.synchronize()
    h = arena.cpu().numpy()
    return [h[m["out_off"]:m["out_off"] + 8 * m["nb"]] for m in msgs]


def restage(arena, msgs):
    for m in msgs:
        if m["nb"]:
            arena[m["in_off"]:m["in_off"] + 8 * m["nb"]].copy_(torch.from_numpy(m["data"]))


@pytest.fixture(scope="module")
def mix(cuda_lib):
    arena, msgs, keys = build_mix(11, 180, 23, 20000)
    kt = cuda_lib.KeyTable(keys)
    want = [oracle_msg(m["mode"], keys[m["key"]].tobytes(), m["iv"], m["data"]) for m in msgs]
    return cuda_lib, arena, msgs, keys, kt, want


def test_mixed_batch_matches_oracle(mix):
    T, arena, msgs, keys, kt, want = mix
    b = T.Batch(kt, entries_for(arena, msgs))
    assert (b.status == 0).all()
    info = b.info()
    assert info["n_cbc_enc_messages"] > 0 and info["n_tiles"] > 0 and info["n_small_items"] > 0
    b.launch()
    for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
        m = msgs[i]
        assert (got == w).all(), f"message {i}: mode {m['mode']} {m['nb']} blocks"


def test_graph_and_launch_shapes_identical(mix):
    T, arena, msgs, keys, kt, want = mix
    b = T.Batch(kt, entries_for(arena, msgs))
    for shape in [(8, 0), (4, 1), (8, 1), (2, 0)]:
        restage(arena, msgs)
        b.configure(*shape)
        b.launch_graph()
        for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
            assert (got == w).all(), f"shape {shape}, message {i}"
    # a second replay of the same graph on restaged inputs gives the same bytes
    restage(arena, msgs)
    b.launch_graph()
    for got, w in zip(outputs(arena, msgs), want):
        assert (got == w).all()


def test_alone_equals_in_the_mix(mix):
    T, arena, msgs, keys, kt, want = mix
    restage(arena, msgs)
    T.Batch(kt, entries_for(arena, msgs)).launch()
    mixed = [o.copy() for o in outputs(arena, msgs)]
    base = arena.data_ptr()
    for i in range(0, len(msgs), 7):
        m = msgs[i]
        restage(arena, [m])
        T.Batch(kt, [(m["mode"], m["key"], m["iv"], base + m["in_off"], base + m["out_off"],
                      8 * m["nb"])]).launch()
        alone = outputs(arena, [m])[0]
        assert (alone == mixed[i]).all(), f"message {i} differs alone vs in the mix"
        # and equals the single-message entry points
        if m["nb"] and m["mode"] in (0, 1, 2, 3):
            ks = T.KeySchedule.from_triple(keys[m["key"]].tobytes())
            x = torch.from_numpy(m["data"]).cuda()
            if m["mode"] == 0:
                y = T.tdes_ecb_encrypt(ks, x)
            elif m["mode"] == 1:
                y = T.tdes_ecb_decrypt(ks, x)
            elif m["mode"] == 2:
                y = T.tdes_ctr_crypt(ks, m["iv"] >> 32, m["iv"] & 0xFFFFFFFF, x)
            else:
                y = T.tdes_cbc_decrypt(ks, m["iv"], x)
            torch.cuda.synchronize()
            assert (y.cpu().numpy() == alone).all()


def test_invalid_descriptors_are_skipped(cuda_lib):
    T = cuda_lib
    keys = synth.key_triples(5, 3)
    kt = T.KeyTable(keys)
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    data = synth.random_bytes(5, 4096)
    buf[:4096].copy_(torch.from_numpy(data))
    base = buf.data_ptr()
    entries = [
        (0, 0, 0, base, base + 8192, 4096),          # valid
        (7, 0, 0, base, base + 16384, 4096),         # bad mode
        (0, 3, 0, base, base + 16384, 4096),         # bad key index
        (0, 0, 0, base, base + 16384, 4095),         # not whole blocks
        (0, 0, 0, base + 4, base + 16384, 4096),     # 4-byte aligned
        (0, 0, 0, base, base + 8, 4096),             # partial overlap
        (2, 0, 0xFFFFFFF0, base, base + 16384, 4096),  # CTR counter would wrap
        (1, 1, 0, base, base + 24576, 0),            # empty: fine, nothing done
    ]
    b = T.Batch(kt, entries)
    assert list(b.status) == [0, -1, -1, -1, -1, -1, -1, 0]
    b.launch()
    torch.cuda.synchronize()
    got = buf[8192:8192 + 4096].cpu().numpy()
    assert (got == oracle.tdes_ecb(keys[0].tobytes(), data)).all()
    assert (buf[16384:16384 + 4096] == 0).all()


def test_config3_every_byte(cuda_lib):
    """4096 messages, log-uniform 64 B .. 4 MiB, modes 40/30/20/10, own keys:
    every byte of every message against the oracle (all host cores)."""
    T = cuda_lib
    seed = 3
    n = 4096
    lens = synth.log_uniform_lengths(seed, n, 64, 4 << 20)
    modes = np.array([0, 2, 3, 4])[synth.categorical(seed, n, [0.4, 0.3, 0.2, 0.1],
                                                     synth.STREAM_MODE)]
    keys = synth.key_triples(seed, n)
    ivs = synth.u64s(seed, n, synth.STREAM_IV)
    total = int(lens.sum())
    offs = np.concatenate([[0], np.cumsum((lens + 15) // 16 * 16)])[:-1]
    src = torch.from_numpy(synth.random_bytes(seed, (total + 15) // 16 * 16 + 16 * n)).cuda()
    dst = torch.zeros_like(src)
    kt = T.KeyTable(keys)
    ents = []
    for i in range(n):
        iv = int(ivs[i])
        if modes[i] == 2:
            iv &= 0xFFFFFFFF00000000
        ents.append((int(modes[i]), i, iv, src.data_ptr() + int(offs[i]),
                     dst.data_ptr() + int(offs[i]), int(lens[i])))
    b = T.Batch(kt, ents)
    assert (b.status == 0).all()
    b.launch()
    torch.cuda.synchronize()
    hs, hd = src.cpu().numpy(), dst.cpu().numpy()
    ivw = np.array([e[2] for e in ents], dtype=np.uint64)
    want = oracle.tdes_messages(keys, np.arange(n, dtype=np.uint32), modes.astype(np.uint8), ivw,
                                offs.astype(np.uint64), (lens // 8).astype(np.uint64), hs, NCPU)
    for i in range(n):
        o, nb = int(offs[i]), int(lens[i])
        assert (hd[o:o + nb] == want[o:o + nb]).all(), f"message {i} mode {modes[i]}"


def test_plans_with_different_shapes_coexist(mix):
    """Each plan keeps its own launch shape; configuring a small plan must not
    stop a larger-shaped plan from launching afterwards."""
    T, arena, msgs, keys, kt, want = mix
    big = T.Batch(kt, entries_for(arena, msgs))
    small = T.Batch(kt, entries_for(arena, msgs))
    big.configure(8, 0)
    small.configure(2, 1)
    for b in (big, small, big):
        restage(arena, msgs)
        b.launch()
        for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
            assert (got == w).all(), f"message {i}"


def test_key_tables_with_single_des_triples(cuda_lib):
    """Triples with K1 = K2 or K2 = K3 (parity bits ignored) get single-DES
    tables in a key table; every path of the batch kernel (bitsliced tiles,
    small messages, packed and one-per-warp CBC-encryption chains) gives the
    oracle's EDE3 result for them, next to ordinary triples."""
    T = cuda_lib
    t = synth.key_triples(31, 3)
    a, b, c = t[0].tobytes()[:8], t[1].tobytes()[8:16], t[2].tobytes()[16:]
    flip = bytes(x ^ 1 for x in a)
    triples = [a + a + b, a + b + b, c + c + c, a + flip + c, a + b + c, t[1].tobytes()]
    keys = np.frombuffer(b"".join(triples), dtype=np.uint8).reshape(-1, 24).copy()
    kt = T.KeyTable(keys)
    msgs, off = [], 0
    for k in range(len(triples)):
        for mode in range(5):
            for nb in (20, 700, 1500 + 7 * k):
                data = synth.random_bytes(3100 + 97 * k + 13 * mode + nb, 8 * nb)
                iv = int(synth.words(31, 100 * k + 10 * mode + nb % 7, 1, synth.STREAM_IV)[0])
                if mode == 2:
                    iv &= 0xFFFFFFFF00000000
                msgs.append(dict(mode=mode, key=k, iv=iv, nb=nb, in_off=off, out_off=off + 8 * nb,
                                 data=data))
                off += 16 * nb
    arena = torch.zeros(off + 64, dtype=torch.uint8, device="cuda")
    restage(arena, msgs)
    b = T.Batch(kt, entries_for(arena, msgs))
    assert (b.status == 0).all()
    b.launch()
    for i, (got, m) in enumerate(zip(outputs(arena, msgs), msgs)):
        want = oracle_msg(m["mode"], triples[m["key"]], m["iv"], m["data"])
        assert (got == want).all(), f"message {i}: key {m['key']} mode {m['mode']} {m['nb']} blocks"


def test_many_small_messages_share_mixed_key_tiles(cuda_lib):
    """A batch with more than 8192 blocks of small (<= 32-block) messages
    packs them into bitsliced tiles whose 32 bit positions carry different
    key triples and directions: every message equals the oracle, for every
    mode, ragged sizes, repeated and single-DES-reducing keys, in-place and
    8-byte-aligned buffers."""
    T = cuda_lib
    rng = np.random.default_rng(41)
    t = synth.key_triples(41, 40)
    a = t[0].tobytes()[:8]
    triples = [x.tobytes() for x in t]
    triples[1] = a + a + t[1].tobytes()[16:]      # K1 = K2: single DES under K3
    triples[2] = t[2].tobytes()[:8] * 3           # K1 = K2 = K3
    keys = np.frombuffer(b"".join(triples), dtype=np.uint8).reshape(-1, 24).copy()
    kt = T.KeyTable(keys)
    msgs, off = [], 0
    for i in range(1400):
        nb = int(rng.integers(1, 33))
        mode = int(rng.integers(0, 5))
        key = int(rng.integers(0, len(triples)))
        iv = int(synth.words(41, i, 1, synth.STREAM_IV)[0])
        if mode == 2:
            iv = (iv & 0xFFFFFFFF00000000) | int(rng.integers(0, 1 << 20))
        in_place = rng.random() < 0.3
        off = (off + 15) // 16 * 16 + (8 if rng.random() < 0.3 else 0)
        in_off = off
        off += 8 * nb
        out_off = in_off if in_place else (off + 15) // 16 * 16
        if not in_place:
            off = out_off + 8 * nb
        msgs.append(dict(mode=mode, key=key, iv=iv, nb=nb, in_off=in_off, out_off=out_off,
                         data=synth.random_bytes(4100 + i, 8 * nb)))
    arena = torch.zeros(off + 64, dtype=torch.uint8, device="cuda")
    restage(arena, msgs)
    b = T.Batch(kt, entries_for(arena, msgs))
    assert (b.status == 0).all()
    info = b.info()
    assert info["n_mixed_tiles"] > 0 and info["n_small_items"] == 0
    for shape in [(8, 0), (4, 0)]:
        restage(arena, msgs)
        b.configure(*shape)
        b.launch_graph()
        for i, (got, m) in enumerate(zip(outputs(arena, msgs), msgs)):
            want = oracle_msg(m["mode"], triples[m["key"]], m["iv"], m["data"])
            assert (got == want).all(), f"{shape} message {i}: mode {m['mode']} {m['nb']} blocks"


def test_large_messages_run_direct(cuda_lib):
    """Messages of 64 MiB or more (ECB both ways, CTR, out-of-place CBC
    decryption) run through the single-key kernels inside the batch launch;
    in-place CBC decryption and CBC encryption stay in the batch kernel.
    Sampled windows of every large message against the oracle (a single-DES
    triple included), every byte of the small ones, and graph replays equal
    the plain launch."""
    T = cuda_lib
    seed, big = 31, 64 << 20
    keys = synth.key_triples(seed, 4).copy()
    keys[2, 8:16] = keys[2, 0:8]  # K1 = K2: one DES pass
    specs = [(0, 0, big), (1, 1, big), (2, 2, big), (3, 3, big), (3, 0, big), (0, 1, 4096),
             (2, 3, 8 * 1000), (4, 2, 8 * 300)]
    inplace = {4}
    ivs = synth.u64s(seed, len(specs), synth.STREAM_IV)
    bufs, ents = [], []
    for i, (mode, key, n) in enumerate(specs):
        x = torch.from_numpy(synth.random_bytes(seed + i, n)).cuda()
        y = x if i in inplace else torch.zeros_like(x)
        iv = int(ivs[i]) & (0xFFFFFFFF00000000 if mode == 2 else 0xFFFFFFFFFFFFFFFF)
        bufs.append((x.cpu().numpy() if i in inplace else None, x, y))
        ents.append((mode, key, iv, x.data_ptr(), y.data_ptr(), n))
    kt = T.KeyTable(keys)
    b = T.Batch(kt, ents)
    assert (b.status == 0).all()
    assert b.info()["n_direct_messages"] == 4
    b.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    outs = []
    for i, ((mode, key, n), (host_in, x, y)) in enumerate(zip(specs, bufs)):
        hin = host_in if host_in is not None else x.cpu().numpy()
        hy = y.cpu().numpy()
        outs.append(hy.copy())
        k, iv, nblk = keys[key].tobytes(), ents[i][2], n // 8
        w = min(nblk, 1024)
        for s in sorted({0, nblk - w, int(rng.integers(0, nblk - w + 1))}):
            xs = hin[8 * s:8 * (s + w)]
            if mode in (0, 1):
                want = oracle.tdes_ecb(k, xs, decrypt=(mode == 1))
            elif mode == 2:
                want = oracle.tdes_ctr(k, iv >> 32, (iv & 0xFFFFFFFF) + s, xs)
            elif mode == 3:
                prev = iv if s == 0 else int.from_bytes(hin[8 * s - 8:8 * s].tobytes(), "big")
                want = oracle.tdes_cbc_decrypt(k, prev, xs)
            else:
                prev = iv if s == 0 else int.from_bytes(hy[8 * s - 8:8 * s].tobytes(), "big")
                want = oracle.tdes_cbc_encrypt(k, prev, xs)
            assert (hy[8 * s:8 * (s + w)] == want).all(), f"message {i} mode {mode} window {s}"
    # graph replays give the same bytes (the in-place message is restored first)
    bufs[4][1].copy_(torch.from_numpy(bufs[4][0]).cuda())
    b.launch_graph()
    torch.cuda.synchronize()
    for i, (_, x, y) in enumerate(bufs):
        assert (y.cpu().numpy() == outs[i]).all(), f"message {i} graph replay"
