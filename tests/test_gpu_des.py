"""Single-DES schedules through the C ABI, against the CPU oracle.

EDE3 under (K, K, K) is single DES under K, and more generally K1 = K2
leaves E_K3 while K2 = K3 leaves E_K1 (Sec. III-B: decryption with the
same key undoes encryption).  The library runs such schedules as one
16-round pass: tdes_des_key_schedule() asks for it directly, and
tdes_key_schedule() picks it for a triple that reduces.  Every mode is
compared bit for bit with the oracle's single-DES and EDE3 functions, at
sizes that cover the empty case, ragged lane groups, one tile and many
tiles of the wide geometry, 8-byte-aligned and in-place buffers; two-key
3DES (K1 = K3) keeps three passes.
"""
import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [0, 1, 33, 1024, 1025, 3 * 1024 + 517]
MODES = ["ecb_enc", "ecb_dec", "ctr", "cbc_dec", "cbc_enc"]


def _dev(data: np.ndarray, offset: int = 0):
    buf = torch.empty(data.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + data.size]
    if data.size:
        view.copy_(torch.from_numpy(data))
    return view


def _host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy()


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


def _des_ref(mode, key, data, iv=0, nonce=0, ctr0=0):
    if mode in ("ecb_enc", "ecb_dec"):
        return oracle.des_ecb(key, data, decrypt=(mode == "ecb_dec"))
    if mode == "ctr":
        return oracle.des_ctr(key, nonce, ctr0, data)
    if mode == "cbc_dec":
        return oracle.des_cbc_decrypt(key, iv, data)
    return oracle.des_cbc_encrypt(key, iv, data)


def _tdes_ref(mode, keys, data, iv=0, nonce=0, ctr0=0):
    if mode in ("ecb_enc", "ecb_dec"):
        return oracle.tdes_ecb(keys, data, decrypt=(mode == "ecb_dec"))
    if mode == "ctr":
        return oracle.tdes_ctr(keys, nonce, ctr0, data)
    if mode == "cbc_dec":
        return oracle.tdes_cbc_decrypt(keys, iv, data)
    return oracle.tdes_cbc_encrypt(keys, iv, data)


@pytest.mark.parametrize("cutoff", [0, 1 << 40], ids=["bitsliced", "per_thread"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nblocks", SIZES)
def test_des_schedule_parity(cuda_lib, mode, nblocks, cutoff):
    seed = 8000 + nblocks
    key = synth.key_triple(seed)[:8]
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce = synth.iv64(seed), synth.nonce32(seed)
    ks = cuda_lib.KeySchedule.des(key)
    assert ks.stages == 1
    with cuda_lib.small_cutoff(cutoff):
        got = _host(_gpu(cuda_lib, mode, ks, _dev(data), _dev(np.zeros_like(data)), iv, nonce, 7))
    want = _des_ref(mode, key, data, iv, nonce, 7)
    assert (got == want).all(), f"{mode} {nblocks}: first diff at byte {np.argmax(got != want)}"


@pytest.mark.parametrize("cutoff", [0, 1 << 40], ids=["bitsliced", "per_thread"])
@pytest.mark.parametrize("mode", MODES)
def test_des_unaligned_and_in_place(cuda_lib, mode, cutoff):
    nblocks = 1000 if mode != "cbc_enc" else 600
    seed = 8100
    key = synth.key_triple(seed)[:8]
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce = synth.iv64(seed), synth.nonce32(seed)
    ks = cuda_lib.KeySchedule.des(key)
    want = _des_ref(mode, key, data, iv, nonce, 0)
    with cuda_lib.small_cutoff(cutoff):
        x = _dev(data, 8)                 # 8-byte aligned, not 16
        out = _dev(np.zeros_like(data), 8)
        assert (_host(_gpu(cuda_lib, mode, ks, x, out, iv, nonce, 0)) == want).all()
        z = _dev(data, 0)                 # in place
        assert (_host(_gpu(cuda_lib, mode, ks, z, z, iv, nonce, 0)) == want).all()


@pytest.mark.parametrize("mode", ["ecb_enc", "ecb_dec", "ctr", "cbc_dec"])
def test_des_wide_geometry(cuda_lib, mode):
    nblocks = (1 << 20) + 77  # 8 MiB + a ragged tile: 8-warp CTAs striding
    seed = 8200
    key = synth.key_triple(seed)[:8]
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce = synth.iv64(seed), synth.nonce32(seed)
    ks = cuda_lib.KeySchedule.des(key)
    x = _dev(data)
    got = _host(_gpu(cuda_lib, mode, ks, x, _dev(np.zeros_like(data)), iv, nonce, 3))
    assert (got == _des_ref(mode, key, data, iv, nonce, 3)).all()
    if mode == "cbc_dec":  # in place: the halo snapshot path
        _gpu(cuda_lib, mode, ks, x, x, iv)
        assert (_host(x) == got).all()


def _variant(key: bytes, flip: int) -> bytes:
    """`key` with the parity bit of every byte flipped when flip is set:
    the same 56 key bits, different bytes."""
    return bytes(b ^ 1 for b in key) if flip else key


@pytest.mark.parametrize("cutoff", [0, 1 << 40], ids=["bitsliced", "per_thread"])
@pytest.mark.parametrize("shape", ["k1=k2", "k2=k3", "k1=k2=k3", "k1=k2 parity differs"])
@pytest.mark.parametrize("mode", MODES)
def test_reducing_triples_run_one_pass(cuda_lib, shape, mode, cutoff):
    seed = 8300 + len(shape)
    t = synth.key_triple(seed)
    a, b = t[:8], t[8:16]
    keys = {"k1=k2": a + a + b, "k2=k3": a + b + b, "k1=k2=k3": a + a + a,
            "k1=k2 parity differs": a + _variant(a, 1) + b}[shape]
    ks = cuda_lib.KeySchedule.from_triple(keys)
    assert ks.stages == 1
    nblocks = 1024 + 300 if mode != "cbc_enc" else 300
    data = synth.random_bytes(seed, 8 * nblocks)
    iv, nonce = synth.iv64(seed), synth.nonce32(seed)
    with cuda_lib.small_cutoff(cutoff):
        got = _host(_gpu(cuda_lib, mode, ks, _dev(data), _dev(np.zeros_like(data)), iv, nonce, 1))
    assert (got == _tdes_ref(mode, keys, data, iv, nonce, 1)).all()


def test_two_key_and_general_triples_keep_three_passes(cuda_lib):
    t = synth.key_triple(8400)
    k1, k2 = t[:8], t[8:16]
    data = synth.random_bytes(8400, 8 * (2048 + 5))
    ks2 = cuda_lib.KeySchedule.two_key(k1, k2)
    assert ks2.stages == 3
    got = _host(cuda_lib.tdes_ecb_encrypt(ks2, _dev(data)))
    assert (got == oracle.tdes_ecb(k1 + k2 + k1, data)).all()
    assert cuda_lib.KeySchedule.from_triple(t).stages == 3
    # a key that differs from its neighbour in one non-parity bit does not reduce
    k2b = bytes([k1[0] ^ 0x02]) + k1[1:]
    ks3 = cuda_lib.KeySchedule(k1, k2b, t[16:])
    assert ks3.stages == 3
    got = _host(cuda_lib.tdes_ecb_encrypt(ks3, _dev(data)))
    assert (got == oracle.tdes_ecb(k1 + k2b + t[16:], data)).all()


def test_des_noalloc_and_host_pipeline(cuda_lib):
    key = synth.key_triple(8500)[:8]
    ks = cuda_lib.KeySchedule.des(key)
    nblocks = 5 * 1024 + 11
    data = synth.random_bytes(8500, 8 * nblocks)
    iv = synth.iv64(8500)
    x = _dev(data)
    cuda_lib.tdes_cbc_decrypt_noalloc(ks, iv, x, x)
    assert (_host(x) == oracle.des_cbc_decrypt(key, iv, data)).all()
    big = synth.random_bytes(8501, 8 * ((1 << 19) + 333))
    hin = torch.from_numpy(big).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    dev_buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    cuda_lib.tdes_ecb_crypt_host(ks, False, hin, hout, dev_buf)
    assert (hout.numpy() == oracle.des_ecb(key, big)).all()


def test_des_full_size_1gib_sampled(cuda_lib):
    """1 GiB under a single-DES schedule in the benchmark's launch shape:
    sampled windows against the oracle, and decryption restores the input."""
    nbytes = 1 << 30
    seed = 3
    key = synth.key_triple(seed)[:8]
    host = synth.random_bytes(seed, nbytes)
    ks = cuda_lib.KeySchedule.des(key)
    x = torch.from_numpy(host).cuda()
    y = torch.empty_like(x)
    rng = np.random.default_rng(seed)
    nblk = nbytes // 8
    starts = np.concatenate([[0, nblk - 1024], rng.integers(0, nblk - 1024, 20)]).astype(np.int64)
    cuda_lib.tdes_ecb_encrypt(ks, x, y)
    yh = _host(y)
    for s in starts:
        w = slice(8 * s, 8 * (s + 1024))
        assert (yh[w] == oracle.des_ecb(key, host[w])).all(), f"DES ECB window at block {s}"
    cuda_lib.tdes_ecb_decrypt(ks, y, y)
    assert torch.equal(y, x)
    del x, y
    torch.cuda.empty_cache()


def test_des_schedule_argument_errors(cuda_lib):
    with pytest.raises(ValueError):
        cuda_lib.KeySchedule.des(b"\x00" * 7)
    lib = cuda_lib.load()
    assert lib.tdes_key_schedule_stages(None) == cuda_lib.TDES_EINVAL
