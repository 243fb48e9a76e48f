"""The allocation-free CBC decryption entry point, checked against the
regular one.

tdes_cbc_decrypt_noalloc exists for callers that cannot let the library
allocate device memory (a server whose pool owns the GPU, a plugin handed
fixed buffers).  Its in-place calls use a fixed scratch array inside the
library instead of a temporary allocation.  This file is collected last so
that a failure here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(data: np.ndarray) -> "torch.Tensor":
    return torch.from_numpy(data).cuda()


def test_noalloc_matches_regular_entry_point_twice(cuda_lib):
    T = cuda_lib
    # several tiles plus a ragged one, so the in-place path saves tile halos
    nblocks = 5 * 1024 + 321
    for call, seed in enumerate((9101, 9102)):  # two calls in a row share the scratch
        keys = synth.key_triple(seed)
        iv = synth.iv64(seed)
        data = synth.random_bytes(seed, 8 * nblocks)
        ks = T.KeySchedule.from_triple(keys)
        want = T.tdes_cbc_decrypt(ks, iv, _dev(data))           # regular entry, out of place
        x = _dev(data)
        T.tdes_cbc_decrypt_noalloc(ks, iv, x, x)                 # new entry, in place
        y = T.tdes_cbc_decrypt_noalloc(ks, iv, _dev(data))       # new entry, out of place
        torch.cuda.synchronize()
        assert torch.equal(x, want), f"in-place call {call} differs"
        assert torch.equal(y, want), f"out-of-place call {call} differs"


def test_noalloc_rejects_oversize_in_place(cuda_lib):
    T = cuda_lib
    ks = T.KeySchedule.from_triple(synth.key_triple(9103))
    buf = torch.zeros(8192, dtype=torch.uint8, device="cuda")
    # rejected by the size check before any launch or memory access
    with pytest.raises(T.TdesError) as e:
        T.tdes_cbc_decrypt_noalloc(ks, 0, buf, buf, nbytes=T.TDES_NOALLOC_MAX_BYTES + 8192)
    assert e.value.status == T.TDES_EINVAL
    assert "scratch limit" in str(e.value)
