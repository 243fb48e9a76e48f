"""The allocation-free CBC decryption entry point, checked against the CPU
oracle and the allocating entry point.

tdes_cbc_decrypt_noalloc exists for callers that cannot let the library
allocate device memory (a server whose pool owns the GPU, a plugin handed
fixed buffers).  Its in-place calls keep the per-tile halo in a fixed scratch
array inside the library instead of a temporary allocation.  Every result
here is compared byte for byte with the oracle's CBC decryption of the same
seeded input and with tdes_cbc_decrypt's: several tiles with a ragged one
(the scratch path), a single tile in place (no scratch), 8-byte-aligned
buffers, and out of place, each twice in a row so that the second call runs
on the scratch the first left.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # (name, blocks, byte offset of the buffer from a 16-byte boundary)
    ("multi_tile_ragged", 5 * 1024 + 321, 0),
    ("single_tile", 1000, 0),
    ("exactly_one_tile", 1024, 0),
    ("aligned_8", 3 * 1024 + 77, 8),
]


def _dev(data: np.ndarray, offset: int) -> "torch.Tensor":
    """A device copy of `data` starting `offset` bytes past a 16-byte boundary."""
    buf = torch.empty(data.size + 16, dtype=torch.uint8, device="cuda")
    assert buf.data_ptr() % 16 == 0
    view = buf[offset:offset + data.size]
    view.copy_(torch.from_numpy(data))
    return view


@pytest.mark.parametrize("name,nblocks,offset", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_twice(cuda_lib, name, nblocks, offset):
    T = cuda_lib
    for call, seed in enumerate((9101, 9102)):  # two calls in a row share the scratch
        keys = synth.key_triple(seed + nblocks)
        iv = synth.iv64(seed)
        data = synth.random_bytes(seed + nblocks, 8 * nblocks)
        want = oracle.tdes_cbc_decrypt(keys, iv, data)
        ks = T.KeySchedule.from_triple(keys)
        x = _dev(data, offset)
        T.tdes_cbc_decrypt_noalloc(ks, iv, x, x)             # in place
        src = _dev(data, offset)
        y = T.tdes_cbc_decrypt_noalloc(ks, iv, src)           # out of place
        z = _dev(data, offset)
        T.tdes_cbc_decrypt(ks, iv, z, z)                      # the allocating entry point
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), want), f"{name}: in-place call {call} differs"
        assert np.array_equal(y.cpu().numpy(), want), f"{name}: out-of-place call {call} differs"
        assert np.array_equal(z.cpu().numpy(), want), f"{name}: regular entry point differs"
        assert np.array_equal(src.cpu().numpy(), data), f"{name}: input changed"
        ks.free()


def test_noalloc_rejects_oversize_in_place(cuda_lib):
    """An in-place call one tile past the scratch limit is refused.  The
    buffer is really that large, so even a call that slipped past the check
    would stay inside its own memory."""
    T = cuda_lib
    ks = T.KeySchedule.from_triple(synth.key_triple(9103))
    n = T.TDES_NOALLOC_MAX_BYTES + 8192
    buf = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TdesError) as e:
        T.tdes_cbc_decrypt_noalloc(ks, 0, buf, buf)
    assert e.value.status == T.TDES_EINVAL
    assert "scratch limit" in str(e.value)
    del buf
    torch.cuda.empty_cache()
    ks.free()
