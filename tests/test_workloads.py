"""The device-side draws of the uniform-message workload (key pick, mode,
IV per message) equal the host draws of ``synth`` word for word: the same
tensor arithmetic is run here on CPU tensors built from the host words."""
import numpy as np
import pytest

from paper_2007_10752_gb300 import synth, workloads

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("first", [0, 1 << 20, (1 << 28) - 5000])
def test_uniform_draws_match_host(first):
    seed, n, n_keys = workloads.STREAM_SEED, 5000, workloads.STREAM_N_KEYS
    kw = torch.from_numpy(synth.u64s(seed, n, synth.STREAM_KEYPICK, first).view(np.int64).copy())
    mw = torch.from_numpy(synth.u64s(seed, n, synth.STREAM_MODE, first).view(np.int64).copy())
    iw = torch.from_numpy(synth.u64s(seed, n, synth.STREAM_IV, first).view(np.int64).copy())
    key = workloads.uniform_key_index(torch, kw, n_keys).numpy().view(np.uint32)
    mode = workloads.uniform_mode(torch, mw)
    iv = workloads.uniform_iv(torch, iw, mode).numpy().view(np.uint64)
    mode = mode.numpy()
    want_key = (synth.u64s(seed, n, synth.STREAM_KEYPICK, first) % np.uint64(n_keys))
    want_mode = np.array([0, 2, 3, 4])[synth.categorical(seed, n, list(workloads.MODE_MIX),
                                                         synth.STREAM_MODE, first)]
    assert (key == want_key).all()
    assert (mode == want_mode).all()
    for i in (0, 1, n // 2, n - 1):
        assert workloads.uniform_expected_fields(seed, first + i, n_keys) == (
            int(key[i]), int(mode[i]), int(iv[i]))
    ctr = mode == 2
    assert (iv[ctr] & np.uint64(0xFFFFFFFF) == 0).all()
    assert (iv[~ctr] == synth.u64s(seed, n, synth.STREAM_IV, first)[~ctr]).all()
    # the mix is roughly the configured one
    frac = np.bincount(want_mode, minlength=5)[[0, 2, 3, 4]] / n
    assert np.allclose(frac, workloads.MODE_MIX, atol=0.03)


def test_first_messages_match_the_batch_workload():
    """Message i of the uniform reading draws what message i of the 2^20-message
    batch reading draws (same streams, same word index)."""
    seed, n_keys = workloads.STREAM_SEED, workloads.STREAM_N_KEYS
    n = 1000
    keys = synth.u64s(seed, n, synth.STREAM_KEYPICK) % np.uint64(n_keys)
    modes = workloads._modes(seed, n)
    for i in (0, 17, 999):
        k, m, _ = workloads.uniform_expected_fields(seed, i, n_keys)
        assert (k, m) == (int(keys[i]), int(modes[i]))
