"""The paper's own one-thread-per-bit design, rebuilt on GB300 as the
benchmark's context point, gives the oracle's bytes too."""
import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import paper_design, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nblocks", [4, 1024, 8192 + 3])
@pytest.mark.parametrize("decrypt", [False, True])
def test_paper_design_matches_oracle(cuda_lib, nblocks, decrypt):
    keys = synth.key_triple(70 + nblocks)
    data = synth.random_bytes(70 + nblocks, 8 * nblocks)
    x = torch.from_numpy(data).cuda()
    y = torch.empty_like(x)
    ms = paper_design.paper_ecb(keys, x, y, decrypt)
    assert ms > 0
    assert (y.cpu().numpy() == oracle.tdes_ecb(keys, data, decrypt=decrypt)).all()
