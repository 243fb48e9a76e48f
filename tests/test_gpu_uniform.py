"""Uniform messages (tdes_uniform_crypt) through the C ABI: every message of
a seeded set (own key triple from a key table, own mode, own IV) equals the
CPU oracle on that message alone, bit for bit, at message sizes from one
block to 32 blocks (odd sizes split a lane's block pair across messages),
in place and out of place, with few keys (single-key tiles) and many keys
(mixed-key tiles), and for CBC encryption in both tile shapes.  The device
plan's tile and slice counts equal those worked out here from the counts per
(mode, key).  Skipped messages are counted and left untouched; the
call replays from a CUDA graph; bad arguments are refused.  At full size,
2^28 messages of 64 bytes (16 GiB), sampled messages are checked."""
import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX5 = (0.25, 0.15, 0.2, 0.2, 0.2)  # ECB enc, ECB dec, CTR, CBC dec, CBC enc


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


def make_case(seed, n, msg_bytes, n_keys, mix=MIX5, reducing_key0=False):
    keys = synth.key_triples(seed, n_keys).copy()
    if reducing_key0:  # K1 = K2: one DES pass under K3
        keys[0, 8:16] = keys[0, 0:8]
    key_index = (synth.u64s(seed, n, synth.STREAM_KEYPICK) % np.uint64(n_keys)).astype(np.uint32)
    mode = synth.categorical(seed, n, list(mix), synth.STREAM_MODE).astype(np.uint8)
    iv = synth.u64s(seed, n, synth.STREAM_IV)
    ctr = mode == 2
    iv[ctr] = (iv[ctr] & np.uint64(0xFFFFFFFF00000000)) | (iv[ctr] & np.uint64(0xFFFF))
    data = synth.random_bytes(seed, n * msg_bytes)
    return keys, key_index, mode, iv, data


def expected(keys, key_index, mode, iv, data, msg_bytes):
    out = np.empty_like(data)
    for i in range(key_index.size):
        s = slice(i * msg_bytes, (i + 1) * msg_bytes)
        out[s] = oracle_msg(int(mode[i]), keys[key_index[i]].tobytes(), int(iv[i]), data[s])
    return out


def expected_plan(key_index, mode, n_keys, m):
    """Tiles and slices the planner must make: per (mode, key) group, whole
    single-key tiles of 1024 // m messages (1024 chains for CBC encryption),
    and slices of 32 // m messages (32 chains) for the rest."""
    counts = np.bincount(mode.astype(np.int64) * n_keys + key_index, minlength=5 * n_keys)
    plan = {}
    for name, c, per_tile, per_slice in (("", counts[:4 * n_keys], 1024 // m, 32 // m),
                                         ("chain_", counts[4 * n_keys:], 1024, 32)):
        u, r = np.divmod(c, per_tile)
        plan[name + "key_tiles"] = int(u.sum())
        plan[(name + "slices") if name else "mixed_slices"] = int((-(-r // per_slice)).sum())
    return plan


def run(T, kt, key_index, mode, iv, data, msg_bytes, in_place, out_fill=None, stream=None):
    k = torch.from_numpy(key_index.view(np.int32)).cuda()
    md = torch.from_numpy(mode).cuda()
    v = torch.from_numpy(iv.view(np.int64)).cuda()
    x = torch.from_numpy(data).cuda()
    if in_place:
        y = x
    else:
        y = torch.full_like(x, 0) if out_fill is None else torch.from_numpy(out_fill).cuda()
    skipped = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    scratch = T.tdes_uniform_crypt(kt, k, md, v, x, y, msg_bytes, skipped=skipped, stream=stream)
    torch.cuda.synchronize()
    return y.cpu().numpy(), int(skipped.item()), T.tdes_uniform_info(scratch)


CASES = [
    # (msg_bytes, n, n_keys): few keys -> single-key tiles; many -> mixed-key tiles
    (64, 6000, 3),
    (64, 3000, 700),
    (8, 12000, 2),
    (24, 6000, 3),
    (16, 6000, 2),  # two blocks: one pair of chain passes per message
    (200, 1500, 4),
    (256, 1200, 3),
]


@pytest.mark.parametrize("in_place", [False, True], ids=["out_of_place", "in_place"])
@pytest.mark.parametrize("msg_bytes,n,n_keys", CASES)
def test_uniform_parity(cuda_lib, msg_bytes, n, n_keys, in_place):
    seed = 9000 + msg_bytes + n_keys
    keys, key_index, mode, iv, data = make_case(seed, n, msg_bytes, n_keys, reducing_key0=True)
    kt = cuda_lib.KeyTable(keys)
    got, skipped, info = run(cuda_lib, kt, key_index, mode, iv, data, msg_bytes, in_place)
    want = expected(keys, key_index, mode, iv, data, msg_bytes)
    bad = np.nonzero((got != want).reshape(n, msg_bytes).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} messages differ, first {bad[:5]} modes {mode[bad[:5]]}"
    assert skipped == 0
    plan = expected_plan(key_index, mode, n_keys, msg_bytes // 8)
    assert {k: info[k] for k in plan} == plan
    if n_keys <= 5:
        assert info["key_tiles"] > 0 and info["mixed_slices"] > 0
    else:
        assert info["mixed_slices"] > 0


@pytest.mark.parametrize("msg_bytes", [8, 64, 136])
def test_uniform_cbc_encrypt_key_tiles(cuda_lib, msg_bytes):
    """CBC encryption only, two keys (key 0 reduces to single DES: the one-pass
    table): 1024-chain single-key tiles plus chain slices."""
    n, n_keys, seed = 2600, 2, 9100 + msg_bytes
    keys, key_index, mode, iv, data = make_case(seed, n, msg_bytes, n_keys,
                                                mix=(0, 0, 0, 0, 1.0), reducing_key0=True)
    kt = cuda_lib.KeyTable(keys)
    for in_place in (False, True):
        got, skipped, info = run(cuda_lib, kt, key_index, mode, iv, data, msg_bytes, in_place)
        assert (got == expected(keys, key_index, mode, iv, data, msg_bytes)).all()
        assert info["chain_key_tiles"] == 2 and info["chain_slices"] > 0
        assert info["key_tiles"] == 0 and info["mixed_slices"] == 0


@pytest.mark.parametrize("msg_bytes,n_keys,mix", [
    (64, 2, (0, 0, 0, 0, 1.0)),  # 1024-chain single-key tiles and chain slices
    (64, 300, MIX5),             # mixed-key slices of every mode
    (16, 3, MIX5),
], ids=["cbc_enc_key_tiles", "mixed_keys", "two_blocks"])
def test_uniform_8_byte_aligned_buffers(cuda_lib, msg_bytes, n_keys, mix):
    """Buffers 8 bytes past a 16-byte boundary: messages of an even number of
    blocks then take the 8-byte loads and stores (CBC-encryption chains one
    block per pass; block tiles without the 16-byte path)."""
    n, seed = 2600, 9150 + msg_bytes + n_keys
    keys, key_index, mode, iv, data = make_case(seed, n, msg_bytes, n_keys, mix=mix)
    kt = cuda_lib.KeyTable(keys)
    want = expected(keys, key_index, mode, iv, data, msg_bytes)
    k = torch.from_numpy(key_index.view(np.int32)).cuda()
    md = torch.from_numpy(mode).cuda()
    v = torch.from_numpy(iv.view(np.int64)).cuda()
    for in_place in (False, True):
        xb = torch.zeros(n * msg_bytes + 32, dtype=torch.uint8, device="cuda")
        x = xb[8 + (-xb.data_ptr()) % 16:][:n * msg_bytes]
        assert x.data_ptr() % 16 == 8
        x.copy_(torch.from_numpy(data))
        if in_place:
            y = x
        else:
            yb = torch.zeros_like(xb)
            y = yb[8 + (-yb.data_ptr()) % 16:][:n * msg_bytes]
        cuda_lib.tdes_uniform_crypt(kt, k, md, v, x, y, msg_bytes)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        bad = np.nonzero((got != want).reshape(n, msg_bytes).any(axis=1))[0]
        assert bad.size == 0, f"{bad.size} messages differ, first {bad[:5]} (modes {mode[bad[:5]]})"


def test_uniform_one_key_skewed(cuda_lib):
    """Every message under one key: a handful of large groups (the planner's
    per-group atomics are shared per warp), CBC-encryption key tiles of 1024
    chains, and ECB messages checked as one concatenated ECB call."""
    n, mb, seed = 100_000, 64, 9600
    keys, key_index, mode, iv, data = make_case(seed, n, mb, 1)
    kt = cuda_lib.KeyTable(keys)
    got, skipped, info = run(cuda_lib, kt, key_index, mode, iv, data, mb, True)
    assert skipped == 0
    assert {k: info[k] for k in expected_plan(key_index, mode, 1, mb // 8)} == \
        expected_plan(key_index, mode, 1, mb // 8)
    assert info["chain_key_tiles"] > 0
    k = keys[0].tobytes()
    g = got.reshape(n, mb)
    d = data.reshape(n, mb)
    for md in (0, 1):
        sel = np.nonzero(mode == md)[0]
        want = oracle.tdes_ecb(k, d[sel].reshape(-1), decrypt=(md == 1)).reshape(-1, mb)
        assert (g[sel] == want).all(), f"mode {md}"
    for i in np.nonzero(mode >= 2)[0]:
        assert (g[i] == oracle_msg(int(mode[i]), k, int(iv[i]), d[i])).all(), i


def test_uniform_million_keys(cuda_lib):
    """A key table of 2^20 triples: 5 x 2^20 groups, so the planner's scan of
    block sums runs over more than one CTA-wide chunk; every message against
    the oracle."""
    import os
    n, mb, n_keys, seed = 20000, 64, 1 << 20, 9700
    keys, key_index, mode, iv, data = make_case(seed, n, mb, n_keys)
    kt = cuda_lib.KeyTable(keys)
    got, skipped, info = run(cuda_lib, kt, key_index, mode, iv, data, mb, False)
    assert skipped == 0
    assert {k: info[k] for k in expected_plan(key_index, mode, n_keys, mb // 8)} == \
        expected_plan(key_index, mode, n_keys, mb // 8)
    want = oracle.tdes_messages(keys, key_index, mode, iv, mb * np.arange(n, dtype=np.uint64),
                                np.full(n, mb // 8, dtype=np.uint64), data,
                                max(1, min(64, os.cpu_count() or 1)))
    assert (got == want).all()
    del kt
    torch.cuda.empty_cache()


def test_uniform_single_message_and_empty(cuda_lib):
    keys = synth.key_triples(9200, 4)
    kt = cuda_lib.KeyTable(keys)
    for md in range(5):
        key_index = np.array([3], dtype=np.uint32)
        mode = np.array([md], dtype=np.uint8)
        iv = np.array([0x0123456789ABCDEF if md != 2 else 0x01234567_00000005], dtype=np.uint64)
        data = synth.random_bytes(9200 + md, 40)
        got, skipped, _ = run(cuda_lib, kt, key_index, mode, iv, data, 40, False)
        assert (got == expected(keys, key_index, mode, iv, data, 40)).all(), md
        assert skipped == 0
    # no messages: nothing runs, skipped = 0
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    skipped = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    scratch = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    cuda_lib.tdes_uniform_crypt(kt, e, e.to(torch.uint8), e.to(torch.int64), x, x, 64,
                                scratch=scratch, skipped=skipped, n_msgs=0)
    torch.cuda.synchronize()
    assert skipped.item() == 0 and (x == 0).all()


def test_uniform_skips_bad_messages(cuda_lib):
    n, mb, n_keys, seed = 3000, 64, 4, 9300
    keys, key_index, mode, iv, data = make_case(seed, n, mb, n_keys)
    rng = np.random.default_rng(seed)
    bad_key = rng.choice(n, 40, replace=False)
    key_index[bad_key] = n_keys + rng.integers(0, 1000, 40).astype(np.uint32)
    rest = np.setdiff1d(np.arange(n), bad_key)
    bad_mode = rng.choice(rest, 30, replace=False)
    mode[bad_mode] = rng.integers(5, 256, 30).astype(np.uint8)
    rest = np.setdiff1d(rest, bad_mode)
    bad_ctr = rng.choice(rest, 20, replace=False)
    mode[bad_ctr] = 2
    iv[bad_ctr] = (iv[bad_ctr] & np.uint64(0xFFFFFFFF00000000)) | np.uint64(0xFFFFFFFC)  # +8 > 2^32
    ok_ctr = rng.choice(np.setdiff1d(rest, bad_ctr), 10, replace=False)
    mode[ok_ctr] = 2
    iv[ok_ctr] = (iv[ok_ctr] & np.uint64(0xFFFFFFFF00000000)) | np.uint64(0xFFFFFFF8)  # ends at 2^32
    fill = np.full_like(data, 0xA5)
    kt = cuda_lib.KeyTable(keys)
    got, skipped, info = run(cuda_lib, kt, key_index, mode, iv, data, mb, False, out_fill=fill)
    skip = np.zeros(n, dtype=bool)
    skip[bad_key] = skip[bad_mode] = skip[bad_ctr] = True
    assert skipped == skip.sum() == info["skipped"]
    g = got.reshape(n, mb)
    assert (g[skip] == 0xA5).all()
    idx = np.nonzero(~skip)[0]
    for i in idx:
        s = slice(i * mb, (i + 1) * mb)
        want = oracle_msg(int(mode[i]), keys[key_index[i]].tobytes(), int(iv[i]), data[s])
        assert (got[s] == want).all(), i
    del kt


def test_uniform_graph_replay(cuda_lib):
    n, mb, n_keys, seed = 4000, 64, 6, 9400
    keys, key_index, mode, iv, data = make_case(seed, n, mb, n_keys)
    kt = cuda_lib.KeyTable(keys)
    k = torch.from_numpy(key_index.view(np.int32)).cuda()
    md = torch.from_numpy(mode).cuda()
    v = torch.from_numpy(iv.view(np.int64)).cuda()
    x = torch.from_numpy(data).cuda()
    y = torch.zeros_like(x)
    need = cuda_lib.tdes_uniform_scratch_bytes(kt, n, mb)
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    cuda_lib.tdes_uniform_crypt(kt, k, md, v, x, y, mb, scratch=scratch)  # outside capture first
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cuda_lib.tdes_uniform_crypt(kt, k, md, v, x, y, mb, scratch=scratch)
    want = expected(keys, key_index, mode, iv, data, mb)
    for _ in range(3):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert (y.cpu().numpy() == want).all()


def test_uniform_argument_errors(cuda_lib):
    kt = cuda_lib.KeyTable(synth.key_triples(9500, 2))
    T = cuda_lib
    for mb in (0, 4, 12, 264):
        with pytest.raises(T.TdesError):
            T.tdes_uniform_scratch_bytes(kt, 10, mb)
    with pytest.raises(T.TdesError):
        T.tdes_uniform_scratch_bytes(kt, (1 << 31) + 1, 64)
    n, mb = 100, 64
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    md = torch.zeros(n, dtype=torch.uint8, device="cuda")
    v = torch.zeros(n, dtype=torch.int64, device="cuda")
    buf = torch.zeros(n * mb + 64, dtype=torch.uint8, device="cuda")
    need = T.tdes_uniform_scratch_bytes(kt, n, mb)
    scratch = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = scratch[(-scratch.data_ptr()) % 256:]
    with pytest.raises(T.TdesError):  # partial overlap
        T.tdes_uniform_crypt(kt, k, md, v, buf[:n * mb], buf[8:8 + n * mb], mb, scratch=base)
    with pytest.raises(T.TdesError):  # misaligned buffer
        T.tdes_uniform_crypt(kt, k, md, v, buf[4:4 + n * mb], buf[4:4 + n * mb], mb,
                             scratch=base)
    with pytest.raises(T.TdesError):  # scratch too small
        T.tdes_uniform_crypt(kt, k, md, v, buf[:n * mb], buf[:n * mb], mb,
                             scratch=base[:need - 256])
    with pytest.raises(T.TdesError):  # misaligned scratch
        T.tdes_uniform_crypt(kt, k, md, v, buf[:n * mb], buf[:n * mb], mb, scratch=base[16:])
    lib = T.load()
    assert lib.tdes_uniform_crypt(None, 0, 0, 0, 0, 0, 64, 1, 0, 0, None, None) == T.TDES_EINVAL
    assert lib.tdes_uniform_info(None, None) == T.TDES_EINVAL


def test_uniform_full_size_sampled(cuda_lib):
    """The second 16 GiB of the streaming workload read as 2^28 messages of 64
    bytes under 65536 key triples (device-drawn arrays), in place; 2^20
    seeded random messages (and the first and last) against the oracle."""
    import os
    seed, n, n_keys, mb = workloads.STREAM_SEED, workloads.STREAM_N_UNIFORM, 65536, 64
    keys = synth.key_triples(seed, n_keys)
    kt = cuda_lib.KeyTable(keys)
    buf = torch.empty(n * mb, dtype=torch.uint8, device="cuda")
    start = workloads.STREAM_BYTES  # the buffer's bytes are those at 16 GiB of the workload
    synth.fill_device(buf, seed, start_byte=start)
    k, md, v = workloads.uniform_arrays_device(torch, seed, n, n_keys)
    skipped = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    scratch = cuda_lib.tdes_uniform_crypt(kt, k, md, v, buf, buf, mb, skipped=skipped)
    torch.cuda.synchronize()
    assert skipped.item() == 0
    info = cuda_lib.tdes_uniform_info(scratch)
    assert info["key_tiles"] > 0 and info["mixed_slices"] > 0 and info["chain_slices"] > 0
    del k, md, v, scratch
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 1 << 20)])).astype(np.uint64)
    key, mode, iv = workloads.uniform_expected_arrays(seed, idx, n_keys)
    got = buf.view(-1, mb)[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    blocks = (np.uint64(start // 8) + np.uint64(8) * idx)[:, None] + np.arange(8, dtype=np.uint64)
    data = synth.blocks_at(seed, blocks.reshape(-1)).reshape(-1)
    want = oracle.tdes_messages(keys, key, mode, iv, mb * np.arange(idx.size, dtype=np.uint64),
                                np.full(idx.size, 8, dtype=np.uint64), data,
                                max(1, min(64, os.cpu_count() or 1)))
    bad = np.nonzero((got.reshape(-1) != want).reshape(-1, mb).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} messages differ, first {idx[bad[:5]]} modes {mode[bad[:5]]}"
    del buf
    torch.cuda.empty_cache()
