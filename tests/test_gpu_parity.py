"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Bit-exact comparison (tolerance 0: the cipher is integer work) on seeded
inputs: sizes that hit the empty case, one block, ragged lane groups,
exactly one and just past one warp tile, many tiles across the wide
launch geometry, 8-byte-aligned (not 16) buffers, in-place calls, and the
1 GiB single-key workload in the launch configuration the benchmark times,
checked on sampled windows the oracle recomputes.  Sizes small calls can
take run on both single-key paths (bitsliced tiles, and one block per
thread), forced with the small-call cutoff.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
NCPU = max(1, min(16, os.cpu_count() or 1))

SIZES = [0, 1, 2, 31, 32, 33, 1023, 1024, 1025, 3 * 1024 + 517, 40 * 1024 + 3]


def _dev(data: np.ndarray, offset: int = 0):
    """Device copy of data starting `offset` bytes into a fresh allocation."""
    buf = torch.empty(data.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + data.size]
    if data.size:
        view.copy_(torch.from_numpy(data))
    return view


def _host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _ref(mode, keys, data, iv=0, nonce=0, ctr0=0):
    if mode == "ecb_enc":
        return oracle.tdes_parallel(keys, data, "ecb_enc", threads=NCPU)
    if mode == "ecb_dec":
        return oracle.tdes_parallel(keys, data, "ecb_dec", threads=NCPU)
    if mode == "ctr":
        return oracle.tdes_parallel(keys, data, "ctr", nonce=nonce, ctr0=ctr0, threads=NCPU)
    if mode == "cbc_dec":
        return oracle.tdes_cbc_decrypt(keys, iv, data)
    return oracle.tdes_cbc_encrypt(keys, iv, data)


def _gpu(T, mode, ks, x, out, iv=0, nonce=0, ctr0=0):
    if mode == "ecb_enc":
        T.tdes_ecb_encrypt(ks, x, out)
    elif mode == "ecb_dec":
        T.tdes_ecb_decrypt(ks, x, out)
    elif mode == "ctr":
        T.tdes_ctr_crypt(ks, nonce, ctr0, x, out)
    elif mode == "cbc_dec":
        T.tdes_cbc_decrypt(ks, iv, x, out)
    else:
        T.tdes_cbc_encrypt(ks, iv, x, out)
    return out


MODES = ["ecb_enc", "ecb_dec", "ctr", "cbc_dec", "cbc_enc"]
PATHS = {"bitsliced": 0, "per_thread": 1 << 40}  # small-call cutoff forcing each path


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nblocks", SIZES)
def test_parity_sizes(cuda_lib, mode, nblocks, path):
    if mode == "cbc_enc" and nblocks > 5000:
        nblocks = 5000  # serial chain: keep the test quick
    seed = 1000 + nblocks
    keys = synth.key_triple(seed)
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce, ctr0 = synth.iv64(seed), synth.nonce32(seed), 17
    ks = cuda_lib.KeySchedule.from_triple(keys)
    x = _dev(data)
    out = _dev(np.zeros_like(data))
    with cuda_lib.small_cutoff(PATHS[path]):
        got = _host(_gpu(cuda_lib, mode, ks, x, out, iv, nonce, ctr0))
    want = _ref(mode, keys, data, iv, nonce, ctr0)
    assert (got == want).all(), f"{mode} {nblocks}: first diff at byte {np.argmax(got != want)}"


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("offset", [8, 24])
@pytest.mark.parametrize("nblocks", [2 * 1024 + 77, 1000])
def test_parity_8byte_aligned_and_in_place(cuda_lib, mode, offset, path, nblocks):
    """Both sizes run in place on the per-thread path: up to 1024 blocks as one
    CTA, above that the bitsliced kernels take in-place CBC decryption."""
    if mode == "cbc_enc":
        nblocks = 700
    seed = 2000 + offset
    keys = synth.key_triple(seed)
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce = synth.iv64(seed), synth.nonce32(seed)
    ks = cuda_lib.KeySchedule.from_triple(keys)
    want = _ref(mode, keys, data, iv, nonce, 0)
    with cuda_lib.small_cutoff(PATHS[path]):
        x = _dev(data, offset)           # 8-byte aligned, not 16
        out = _dev(np.zeros_like(data), offset)
        assert (_host(_gpu(cuda_lib, mode, ks, x, out, iv, nonce, 0)) == want).all()
        y = _dev(data, offset)           # in place
        assert (_host(_gpu(cuda_lib, mode, ks, y, y, iv, nonce, 0)) == want).all()
        z = _dev(data, 0)                # in place, 16-byte aligned
        assert (_host(_gpu(cuda_lib, mode, ks, z, z, iv, nonce, 0)) == want).all()


@pytest.mark.parametrize("mode", ["ecb_enc", "ecb_dec", "ctr", "cbc_dec"])
def test_parity_wide_geometry(cuda_lib, mode):
    """More tiles than the small-input geometry covers: 8-warp CTAs striding."""
    nblocks = (1 << 21) + 77  # 16 MiB + a ragged tile
    seed = 3000
    keys = synth.key_triple(seed)
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce = synth.iv64(seed), synth.nonce32(seed)
    ks = cuda_lib.KeySchedule.from_triple(keys)
    x = _dev(data)
    got = _host(_gpu(cuda_lib, mode, ks, x, _dev(np.zeros_like(data)), iv, nonce, 5))
    if mode == "cbc_dec":  # parallel reference: windows with their own IV
        want = np.empty_like(data)
        step = 8 * 65536
        for s in range(0, data.size, step):
            ivw = iv if s == 0 else int.from_bytes(data[s - 8:s].tobytes(), "big")
            want[s:s + step] = oracle.tdes_cbc_decrypt(keys, ivw, data[s:s + step])
    else:
        want = _ref(mode, keys, data, iv, nonce, 5)
    assert (got == want).all()
    # the in-place CBC decryption takes the halo snapshot path
    if mode == "cbc_dec":
        _gpu(cuda_lib, mode, ks, x, x, iv)
        assert (_host(x) == want).all()


def test_golden_vectors(cuda_lib):
    n = 0
    for line in open(os.path.join(HERE, "golden", "tdes_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        mode, _seed, keys, ivn, ctr0, data, out = line.split()
        keys = bytes.fromhex(keys)
        data = np.frombuffer(bytes.fromhex(data), dtype=np.uint8).copy()
        ks = cuda_lib.KeySchedule.from_triple(keys)
        x = _dev(data)
        got = _host(_gpu(cuda_lib, mode, ks, x, _dev(np.zeros_like(data)), int(ivn, 16),
                         int(ivn, 16), int(ctr0)))
        assert got.tobytes().hex() == out, line[:30]
        n += 1
    assert n == 15


def test_roundtrips_and_determinism(cuda_lib):
    keys = synth.key_triple(4000)
    data = synth.random_bytes(4000, 8 * (5 * 1024 + 9))
    ks = cuda_lib.KeySchedule.from_triple(keys)
    x = _dev(data)
    c1 = cuda_lib.tdes_ecb_encrypt(ks, x)
    c2 = cuda_lib.tdes_ecb_encrypt(ks, x)
    assert torch.equal(c1, c2)
    assert (_host(cuda_lib.tdes_ecb_decrypt(ks, c1)) == data).all()
    iv = synth.iv64(4000)
    ce = cuda_lib.tdes_cbc_encrypt(ks, iv, x)
    assert (_host(cuda_lib.tdes_cbc_decrypt(ks, iv, ce)) == data).all()
    k = cuda_lib.tdes_ctr_crypt(ks, 9, 0, x)
    assert (_host(cuda_lib.tdes_ctr_crypt(ks, 9, 0, k)) == data).all()
    # EDE3 with K1 = K2 = K3 is single DES (Sec. III-B)
    k1 = keys[:8]
    ks1 = cuda_lib.KeySchedule(k1, k1, k1)
    blk = data[:8 * 64]
    got = _host(cuda_lib.tdes_ecb_encrypt(ks1, _dev(blk)))
    want = b"".join(oracle.des_block(k1, blk[i:i + 8]) for i in range(0, blk.size, 8))
    assert got.tobytes() == want


def test_argument_errors(cuda_lib):
    keys = synth.key_triple(5000)
    ks = cuda_lib.KeySchedule.from_triple(keys)
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    E = cuda_lib.TdesError
    with pytest.raises(E) as e:   # partial overlap
        cuda_lib.tdes_ecb_encrypt(ks, buf[:4096], buf[8:4104])
    assert e.value.status == cuda_lib.TDES_EINVAL
    with pytest.raises(E):        # 4-byte aligned
        cuda_lib.tdes_ecb_encrypt(ks, buf[4:4100], buf[8192:12288])
    with pytest.raises(E):        # not whole blocks
        cuda_lib.tdes_ecb_encrypt(ks, buf[:4096], buf[8192:12288], nbytes=4095)
    with pytest.raises(E):        # counter would wrap
        cuda_lib.tdes_ctr_crypt(ks, 0, 0xFFFFFFFF, buf[:16], buf[8192:8208])
    cuda_lib.tdes_ctr_crypt(ks, 0, 0xFFFFFFFF, buf[:8], buf[8192:8200])  # exactly fits
    cuda_lib.tdes_ecb_encrypt(ks, buf[:0], buf[8192:8192])                # empty is fine
    torch.cuda.synchronize()


@pytest.mark.parametrize("kind", ["pinned", "pageable", "pinned_4_bytes_off"])
def test_host_buffer_pipeline(cuda_lib, kind):
    """Host buffers in and out, pinned, pageable, and pinned but off an 8-byte
    boundary: each streams through the device buffer in several chunks."""
    nblocks = (1 << 20) + 333  # 8 MiB + ragged, several chunks of a 1 MiB device buffer
    keys = synth.key_triple(6000)
    data = synth.random_bytes(6000, 8 * nblocks)
    ks = cuda_lib.KeySchedule.from_triple(keys)
    if kind == "pageable":
        hin, hout = data.copy(), np.empty_like(data)
    else:
        off = 4 if kind == "pinned_4_bytes_off" else 0
        a = torch.empty(data.size + 8, dtype=torch.uint8).pin_memory()
        b = torch.empty(data.size + 8, dtype=torch.uint8).pin_memory()
        hin, hout = a[off:off + data.size], b[off:off + data.size]
        hin.copy_(torch.from_numpy(data))
    dev_buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    cuda_lib.tdes_ecb_crypt_host(ks, False, hin, hout, dev_buf)
    want = oracle.tdes_parallel(keys, data, "ecb_enc", threads=NCPU)
    got = hout if kind == "pageable" else hout.numpy()
    assert (got == want).all()
    cuda_lib.tdes_ecb_crypt_host(ks, True, hout, hout, dev_buf)  # in place, host side
    got = hout if kind == "pageable" else hout.numpy()
    assert (got == data).all()


def test_full_size_1gib(cuda_lib):
    """The 1 GiB single-key workload, in the benchmark's launch configuration:
    every byte of the ECB encryption against the oracle (all host cores),
    CTR windows against the oracle, and decryption restores the input
    everywhere."""
    nbytes = 1 << 30
    seed = 2
    keys = synth.key_triple(seed)
    nonce = synth.nonce32(seed)
    host = synth.random_bytes(seed, nbytes)
    ks = cuda_lib.KeySchedule.from_triple(keys)
    x = torch.from_numpy(host).cuda()
    y = torch.empty_like(x)
    rng = np.random.default_rng(seed)
    nblk = nbytes // 8
    starts = np.concatenate([[0, nblk - 1024], rng.integers(0, nblk - 1024, 30)]).astype(np.int64)
    cuda_lib.tdes_ecb_encrypt(ks, x, y)
    yh = _host(y)
    want = oracle.tdes_parallel(keys, host, "ecb_enc", threads=NCPU)
    bad = np.nonzero((yh != want).reshape(-1, 8).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} ECB blocks differ, first {bad[:5]}"
    del want
    cuda_lib.tdes_ecb_decrypt(ks, y, y)
    assert torch.equal(y, x)
    cuda_lib.tdes_ctr_crypt(ks, nonce, 0, x, y)
    yh = _host(y)
    for s in starts:
        w = slice(8 * s, 8 * (s + 1024))
        assert (yh[w] == oracle.tdes_ctr(keys, nonce, int(s), host[w])).all(), f"CTR at {s}"
    del x, y
    torch.cuda.empty_cache()


def test_pinned_host_buffers_zero_copy(cuda_lib):
    """The kernels read and write page-locked host memory directly over the
    host link; pageable memory is refused before any launch."""
    keys = synth.key_triple(7000)
    data = synth.random_bytes(7000, 8 * (3 * 1024 + 77))
    ks = cuda_lib.KeySchedule.from_triple(keys)
    hin = torch.from_numpy(data).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    cuda_lib.tdes_ecb_encrypt(ks, hin, hout)
    cuda_lib.tdes_ctr_crypt(ks, 5, 0, hout, hout)  # in place, host to host
    torch.cuda.synchronize()
    want = oracle.tdes_ctr(keys, 5, 0, oracle.tdes_ecb(keys, data))
    assert (hout.numpy() == want).all()
    pageable = np.zeros_like(data)
    with pytest.raises(cuda_lib.TdesError) as e:
        cuda_lib.tdes_ecb_encrypt(ks, pageable, pageable)
    assert e.value.status == cuda_lib.TDES_EINVAL
