"""The continuous-batching server through the C ABI: every request's result
equals the oracle and the same request run alone; requests submitted while
others run are batched separately and overlap; the HBM budget queues work
instead of failing it; waits are bounded; the load generator reports sane
latency statistics."""
import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle(mode, keys, iv, data):
    if mode == 0:
        return oracle.tdes_ecb(keys, data)
    if mode == 2:
        return oracle.tdes_ctr(keys, iv >> 32, iv & 0xFFFFFFFF, data)
    return oracle.tdes_cbc_decrypt(keys, iv, data)


def _requests(seed, n, n_keys, big_every=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        if big_every and i % big_every == 0:
            nb = int(rng.integers(8192, 2 * 8192 + 5))      # 64-128 KiB
        elif rng.random() < 0.8:
            nb = int(rng.integers(8, 513))                   # 64 B .. 4 KiB
        else:
            nb = int(rng.integers(513, 6000))
        mode = int(rng.choice([0, 2, 3]))
        iv = int(synth.words(seed, i, 1, synth.STREAM_IV)[0])
        if mode == 2:
            iv &= 0xFFFFFFFF00000000
        reqs.append(dict(mode=mode, key=int(rng.integers(0, n_keys)), iv=iv,
                         data=synth.random_bytes(seed * 7919 + i, 8 * nb)))
    return reqs


def _run(T, srv, reqs, keys):
    ins = [torch.from_numpy(r["data"]).cuda() for r in reqs]
    outs = [torch.empty_like(x) for x in ins]
    torch.cuda.synchronize()
    tickets = [srv.submit(r["mode"], r["key"], r["iv"], x, y) for r, x, y in zip(reqs, ins, outs)]
    for t in tickets:
        assert srv.wait(t, 60.0) == 0
    return [y.cpu().numpy() for y in outs]


def test_server_results_match_oracle_and_alone(cuda_lib):
    """16384 resident key triples, as in the serving workload."""
    T = cuda_lib
    keys = synth.key_triples(21, 16384)
    kt = T.KeyTable(keys)
    srv = T.Server(kt)
    reqs = _requests(21, 400, 16384, big_every=37)
    got = _run(T, srv, reqs, keys)
    for i, (r, g) in enumerate(zip(reqs, got)):
        want = _oracle(r["mode"], keys[r["key"]].tobytes(), r["iv"], r["data"])
        assert (g == want).all(), f"request {i}"
    # the same requests one at a time (each alone in its batch) give the same bytes
    for i in range(0, len(reqs), 23):
        alone = _run(T, srv, [reqs[i]], keys)[0]
        assert (alone == got[i]).all(), f"request {i} alone vs in the mix"
    srv.close()


def test_group_submit_poll_wait(cuda_lib):
    """A group of requests under one ticket: per-request statuses, the group
    completes as a whole and every result equals the oracle; a group with one
    bad descriptor is refused whole, before anything is queued."""
    T = cuda_lib
    keys = synth.key_triples(23, 16)
    kt = T.KeyTable(keys)
    srv = T.Server(kt)
    reqs = _requests(23, 120, 16, big_every=17)
    ins = [torch.from_numpy(r["data"]).cuda() for r in reqs]
    outs = [torch.empty_like(x) for x in ins]
    empty = torch.empty(0, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    entries = [(r["mode"], r["key"], r["iv"], x, y, x.numel()) for r, x, y in zip(reqs, ins, outs)]
    entries.append((0, 0, 0, empty, empty, 0))  # an empty request completes at once
    group = srv.submit_group(entries)
    assert group[1] == len(reqs) + 1
    assert srv.wait_group(group, 60.0) == 0
    status, per = srv.poll_group(group)
    assert status == 0 and (per == 0).all()
    for i, (r, y) in enumerate(zip(reqs, outs)):
        want = _oracle(r["mode"], keys[r["key"]].tobytes(), r["iv"], r["data"])
        assert (y.cpu().numpy() == want).all(), f"request {i}"
    # one invalid descriptor (key index out of range): the whole group is refused
    bad = entries[:3] + [(0, 999, 0, ins[0], outs[0], ins[0].numel())]
    with pytest.raises(T.TdesError):
        srv.submit_group(bad)
    # the next group still works, and its tickets follow on
    g2 = srv.submit_group(entries[:5])
    assert g2[0] == group[0] + group[1]
    assert srv.wait_group(g2, 60.0) == 0
    srv.close()


def test_budget_queues_instead_of_failing(cuda_lib):
    T = cuda_lib
    keys = synth.key_triples(22, 8)
    kt = T.KeyTable(keys)
    srv = T.Server(kt, budget_bytes=256 << 10, slots=2)  # far below the total submitted
    reqs = _requests(22, 120, 8, big_every=10)
    got = _run(T, srv, reqs, keys)
    for r, g in zip(reqs, got):
        assert (g == _oracle(r["mode"], keys[r["key"]].tobytes(), r["iv"], r["data"])).all()
    big = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TdesError):  # larger than the whole budget
        srv.submit(0, 0, 0, big, torch.empty_like(big))
    srv.close()


def test_bounded_wait_and_bad_requests(cuda_lib):
    T = cuda_lib
    kt = T.KeyTable(synth.key_triples(23, 2))
    srv = T.Server(kt)
    # a ticket that was never issued stays pending: the wait gives up
    assert srv.wait(10 ** 9, 0.01) == T.TDES_ETIMEDOUT
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TdesError):
        srv.submit(0, 5, 0, buf, torch.empty_like(buf))        # key index out of range
    with pytest.raises(T.TdesError):
        srv.submit(9, 0, 0, buf, torch.empty_like(buf))        # bad mode
    t = srv.submit(0, 0, 0, buf[:0], buf[:0])                  # empty request completes
    assert srv.poll(t) == 0
    srv.close()


def test_loadtest_reports(cuda_lib):
    T = cuda_lib
    kt = T.KeyTable(synth.key_triples(24, 256))
    srv = T.Server(kt)
    pool = torch.from_numpy(synth.random_bytes(24, 64 << 20)).cuda()
    out = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    r = srv.loadtest(pool, out, 3000, 20.0, large=(64 << 10, 4 << 20))
    assert r["requests"] == 3000 and r["batches"] >= 1
    assert 0 < r["p50_ms"] <= r["p99_ms"] <= r["max_ms"]
    assert r["gbps"] > 0
    sat = srv.loadtest(pool, out, 3000, 0.0, large=(64 << 10, 4 << 20))
    assert sat["gbps"] > 0
    # at saturation the slots fill: batches are in flight and on the device together
    assert sat["max_slots_busy"] >= 2 and sat["max_device_overlap"] >= 2, sat
    assert 0.0 < sat["device_overlap_frac"] <= 1.0, sat
    srv.close()


@pytest.mark.parametrize("staged", [False, True], ids=["zero_copy", "staged"])
def test_server_host_payloads(cuda_lib, staged):
    """Requests whose buffers are pinned host memory: the kernels work on them
    over the host link, or (staged) the large ones are copied through the
    slot's device staging and processed there; pageable host buffers are
    refused at submit."""
    T = cuda_lib
    keys = synth.key_triples(25, 16)
    kt = T.KeyTable(keys)
    srv = T.Server(kt, stage_bytes=(1 << 20) if staged else 0, stage_min_bytes=64 << 10)
    reqs = _requests(25, 120, 16, big_every=40)
    ins = [torch.from_numpy(r["data"]).pin_memory() for r in reqs]
    outs = [torch.empty_like(x).pin_memory() for x in ins]
    tickets = [srv.submit(r["mode"], r["key"], r["iv"], x, y) for r, x, y in zip(reqs, ins, outs)]
    for t in tickets:
        assert srv.wait(t, 60.0) == 0
    for r, y in zip(reqs, outs):
        assert (y.numpy() == _oracle(r["mode"], keys[r["key"]].tobytes(), r["iv"], r["data"])).all()
    page = np.zeros(4096, dtype=np.uint8)
    with pytest.raises(T.TdesError):
        srv.submit(0, 0, 0, page, page)
    srv.close()


def test_requests_overlap_on_the_device(cuda_lib):
    """Continuous batching: a large request (4 MiB of CBC encryption, one
    serial chain of 2^19 blocks, about half a second) is submitted first and
    200 small requests after it.  The small ones are dispatched into other
    slots while the large one runs: all of them complete before it, at least
    two batches are in flight and on the device at once (device intervals
    from CUDA events), and every result equals the oracle.  Keys are drawn
    from 16384 resident triples."""
    T = cuda_lib
    keys = synth.key_triples(24, 16384)
    kt = T.KeyTable(keys)
    srv = T.Server(kt, slots=4)
    big_data = synth.random_bytes(2400, 4 << 20)
    bx = torch.from_numpy(big_data).cuda()
    by = torch.zeros_like(bx)
    big_iv = synth.iv64(2400)
    small = _requests(25, 200, 16384)
    small = [r for r in small if r["data"].size <= 4096][:150]
    ins = [torch.from_numpy(r["data"]).cuda() for r in small]
    outs = [torch.empty_like(x) for x in ins]
    torch.cuda.synchronize()
    srv.stats(reset=True)
    tb = srv.submit(4, 1234, big_iv, bx, by)
    ts = [srv.submit(r["mode"], r["key"], r["iv"], x, y) for r, x, y in zip(small, ins, outs)]
    for t in ts:
        assert srv.wait(t, 30.0) == 0
    assert srv.poll(tb) == 1, "the small requests waited for the large one"
    assert srv.wait(tb, 60.0) == 0
    st = srv.stats()
    assert st["max_slots_busy"] >= 2, st
    assert st["max_device_overlap"] >= 2, st
    assert st["device_overlap_ms"] > 0.0, st
    assert st["untimed_batches"] == 0, st
    for r, y in zip(small, outs):
        want = _oracle(r["mode"], keys[r["key"]].tobytes(), r["iv"], r["data"])
        assert (y.cpu().numpy() == want).all()
    want = oracle.tdes_cbc_encrypt(keys[1234].tobytes(), big_iv, big_data)
    assert (by.cpu().numpy() == want).all()
    srv.close()


def test_idle_server_sleeps(cuda_lib):
    """With nothing queued and nothing in flight the dispatcher sleeps on a
    condition variable: an idle server uses almost no CPU time."""
    import resource
    import time
    T = cuda_lib
    kt = T.KeyTable(synth.key_triples(26, 4))
    srv = T.Server(kt)
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    assert srv.wait(srv.submit(0, 0, 0, buf, torch.empty_like(buf)), 10.0) == 0
    time.sleep(0.05)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    time.sleep(0.5)
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    wall = time.perf_counter() - t0
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    assert cpu < 0.2 * wall, f"{cpu:.3f} s of CPU in {wall:.3f} s idle"
    srv.close()
