"""The launch-shape autotuner through the C ABI: tuning a batch leaves its
results bit-exact (every shape the search can pick, including the compact
round loop and multi-tile claims, gives the oracle's bytes), the choice is
written to the cache file under the batch's workload class, and a later plan
of the same class starts in the tuned shape without timing; shapes outside
the documented ranges are refused.  The server's tuner stores a
configuration that tdes_server_config_default then returns."""
import json

import pytest

from paper_2007_10752_gb300 import synth
from test_gpu_batch import build_mix, entries_for, oracle_msg, outputs, restage

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "autotune.jsonl"
    monkeypatch.setenv("TDES_AUTOTUNE_CACHE", str(path))
    return path


def test_every_shape_gives_the_oracle_bytes(cuda_lib, cache):
    T = cuda_lib
    arena, msgs, keys = build_mix(61, 150, 19, 40000, in_place_frac=0.0)
    kt = T.KeyTable(keys)
    want = [oracle_msg(m["mode"], keys[m["key"]].tobytes(), m["iv"], m["data"]) for m in msgs]
    b = T.Batch(kt, entries_for(arena, msgs))
    shapes = [(8, 0, 0, T.ROUNDS_PER_PASS), (8, 0, 0, T.ROUNDS_COMPACT),
              (4, 0, 2, T.ROUNDS_PER_PASS), (4, 3, 8, T.ROUNDS_COMPACT),
              (8, 1, 1, T.ROUNDS_COMPACT), (6, 0, 1024, T.ROUNDS_PER_PASS)]
    for shape in shapes:
        restage(arena, msgs)
        b.set_shape(*shape)
        got_shape = b.shape()
        assert got_shape["warps_per_cta"] == shape[0] and got_shape["round_form"] == shape[3]
        b.launch_graph()
        for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
            assert (got == w).all(), f"shape {shape}, message {i}"
    for bad in [(0, 0, 0, 0), (9, 0, 0, 0), (8, 0, -1, 0), (8, 0, 1025, 0), (8, 0, 0, 2)]:
        with pytest.raises(T.TdesError):
            b.set_shape(*bad)


def test_autotune_stores_and_later_plans_use_it(cuda_lib, cache):
    T = cuda_lib
    arena, msgs, keys = build_mix(62, 200, 23, 60000, in_place_frac=0.0)
    kt = T.KeyTable(keys)
    want = [oracle_msg(m["mode"], keys[m["key"]].tobytes(), m["iv"], m["data"]) for m in msgs]
    ents = entries_for(arena, msgs)
    b = T.Batch(kt, ents)
    assert not b.info()["tuned"]
    r = b.autotune(reps=2)
    assert not r["from_cache"] and r["candidates"] >= 5
    assert r["best_ms"] > 0 and r["baseline_ms"] > 0
    assert r["best_ms"] <= r["baseline_ms"] * 1.0000001 or r["best"] == r["baseline"]
    assert b.info()["tuned"]
    # the tuning runs rewrote the outputs from intact inputs: still the oracle's bytes
    for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
        assert (got == w).all(), f"message {i} after tuning"
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert lines[-1]["key"] == r["key"] and r["key"].startswith("sm")
    assert lines[-1]["warps_per_cta"] == r["best"]["warps_per_cta"]
    # a new plan of the same class starts in the tuned shape
    b2 = T.Batch(kt, ents)
    info = b2.info()
    assert info["tuned"]
    s2 = b2.shape()
    for k in ("warps_per_cta", "tiles_per_claim", "round_form"):
        assert s2[k] == r["best"][k], k
    r2 = b2.autotune()
    assert r2["from_cache"] and r2["candidates"] == 0
    restage(arena, msgs)
    b2.launch()
    for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
        assert (got == w).all(), f"message {i} in the tuned shape"
    # a batch context picks the tuned shape up too, and gets the same bytes
    ctx = T.Ctx(kt)
    restage(arena, msgs)
    torch.cuda.synchronize()
    t = ctx.submit(ents)
    assert ctx.wait(t, 60.0) == 0
    for i, (got, w) in enumerate(zip(outputs(arena, msgs), want)):
        assert (got == w).all(), f"message {i} through the context"
    ctx.close()


def test_server_autotune_feeds_the_default_config(cuda_lib, cache):
    T = cuda_lib
    kt = T.KeyTable(synth.key_triples(63, 64))
    pool = torch.from_numpy(synth.random_bytes(63, 32 << 20)).cuda()
    out = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    r = T.tdes_server_autotune(kt, pool, out, 400, large=(64 << 10, 1 << 20))
    assert not r["from_cache"] and r["candidates"] >= 4 and r["best_gbps"] > 0
    srv = T.Server(kt)  # default configuration: now the tuned one
    for k in ("warps_per_cta", "reserve_ctas_per_sm", "slots", "round_form"):
        assert srv.config[k] == r["best"][k], k
    res = srv.loadtest(pool, out, 300, 0.0, large=(64 << 10, 1 << 20))
    assert res["gbps"] > 0
    srv.close()
    again = T.tdes_server_autotune(kt, pool, out, 400, large=(64 << 10, 1 << 20))
    assert again["from_cache"] and again["best"]["slots"] == r["best"]["slots"]
