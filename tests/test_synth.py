"""The seeded input generator: counter form of SplitMix64 against the
sequential definition, random access, and the shapes of the draws."""
import numpy as np

from paper_2007_10752_gb300 import synth


def _splitmix64_sequential(seed, n):
    """SplitMix64 written the sequential way (state += gamma; mix(state))."""
    mask = (1 << 64) - 1
    state = seed & mask
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_counter_form_equals_sequential_definition():
    for seed in (0, 1, 1234567, 2**63 + 5):
        got = [int(x) for x in synth.splitmix64_at(seed, np.arange(50, dtype=np.uint64))]
        assert got == _splitmix64_sequential(seed, 50)


def test_random_access_agrees_with_bulk():
    full = synth.random_bytes(7, 8 * 5000, chunk_words=333)
    assert (synth.random_bytes(7, 8 * 100, start_byte=8 * 1234) == full[8 * 1234:8 * 1334]).all()
    idx = np.array([0, 1, 999, 4999])
    assert (synth.blocks_at(7, idx) == full.reshape(-1, 8)[idx]).all()


def test_streams_and_seeds_differ():
    a = synth.random_bytes(1, 64)
    assert not (a == synth.random_bytes(2, 64)).all()
    assert not (a == synth.random_bytes(1, 64, stream=synth.STREAM_KEYS)).all()


def test_keys_have_odd_parity():
    k = synth.key_triples(3, 100)
    assert k.shape == (100, 24)
    ones = np.unpackbits(k[..., None], axis=-1).sum(axis=-1)
    assert (ones % 2 == 1).all()


def test_log_uniform_lengths():
    n = synth.log_uniform_lengths(4, 20000, 64, 4 << 20)
    assert (n % 8 == 0).all() and n.min() >= 64 and n.max() <= 4 << 20
    med = np.median(n)
    assert 0.7 * np.sqrt(64 * (4 << 20)) < med < 1.3 * np.sqrt(64 * (4 << 20))


def test_categorical_frequencies():
    m = synth.categorical(5, 40000, [0.4, 0.3, 0.2, 0.1], synth.STREAM_MODE)
    f = np.bincount(m, minlength=4) / m.size
    assert np.allclose(f, [0.4, 0.3, 0.2, 0.1], atol=0.01)
