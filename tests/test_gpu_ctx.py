"""Batch contexts through the C ABI (tdes_ctx_create, tdes_batch_submit,
tdes_batch_poll, tdes_batch_wait, tdes_batch_release): a mixed batch in the
shape of the 4096-message workload -- own key triple per message, log-uniform
lengths, ECB / CTR / CBC-decrypt / CBC-encrypt -- is submitted as
descriptors, its per-descriptor statuses are polled, and every byte of every
message equals the CPU oracle; rejected descriptors are reported and skipped;
waits are bounded (a wait on a ticket not issued yet, and a short wait on a
long CBC-encryption chain, run out with TDES_ETIMEDOUT and leave the
context usable); several tickets are in flight at once; a planned batch gets
a ticket too."""
import ctypes
import gc
import os

import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NCPU = max(1, min(16, os.cpu_count() or 1))


def mixed_workload(seed, n, max_len, n_keys):
    """Config-3-style messages packed in one source arena (16-byte aligned)."""
    lens = synth.log_uniform_lengths(seed, n, 64, max_len)
    modes = np.array([0, 2, 3, 4])[synth.categorical(seed, n, [0.4, 0.3, 0.2, 0.1],
                                                     synth.STREAM_MODE)]
    kidx = (synth.u64s(seed, n, synth.STREAM_KEYPICK) % np.uint64(n_keys)).astype(np.uint32)
    ivs = synth.u64s(seed, n, synth.STREAM_IV)
    ivs = np.where(modes == 2, ivs & np.uint64(0xFFFFFFFF00000000), ivs).astype(np.uint64)
    offs = np.concatenate([[0], np.cumsum((lens + 15) // 16 * 16)])[:-1].astype(np.uint64)
    total = int(offs[-1] + lens[-1]) + 16
    data = synth.random_bytes(seed, total)
    return lens, modes, kidx, ivs, offs, data


def expected(keys, lens, modes, kidx, ivs, offs, data):
    return oracle.tdes_messages(keys, kidx, modes.astype(np.uint8), ivs, offs,
                                (lens // 8).astype(np.uint64), data, NCPU)


def raw_descs(T, lens, modes, kidx, ivs, offs, src, dst):
    arr = (T.Desc * len(lens))()
    for i in range(len(lens)):
        arr[i] = T.Desc(int(modes[i]), int(kidx[i]), int(ivs[i]), src.data_ptr() + int(offs[i]),
                        dst.data_ptr() + int(offs[i]), int(lens[i]))
    return arr


def test_submit_poll_wait_every_byte(cuda_lib):
    T = cuda_lib
    lib = T.load()
    seed, n, n_keys = 41, 1500, 97
    keys = synth.key_triples(seed, n_keys)
    lens, modes, kidx, ivs, offs, data = mixed_workload(seed, n, 1 << 20, n_keys)
    kt = T.KeyTable(keys)
    src = torch.from_numpy(data).cuda()
    dst = torch.zeros_like(src)
    descs = raw_descs(T, lens, modes, kidx, ivs, offs, src, dst)
    # three rejected descriptors at the end: bad key index, bad mode, CTR counter wrap
    bad = (T.Desc * 3)(T.Desc(0, n_keys, 0, src.data_ptr(), dst.data_ptr(), 64),
                       T.Desc(9, 0, 0, src.data_ptr(), dst.data_ptr(), 64),
                       T.Desc(2, 0, 0xFFFFFFFF, src.data_ptr(), dst.data_ptr(), 64))
    allc = (T.Desc * (n + 3))(*descs, *bad)
    torch.cuda.synchronize()  # the context's streams do not wait for torch's
    ctx = ctypes.c_void_p()
    cfg = T.CtxConfig()
    lib.tdes_ctx_config_default(ctypes.byref(cfg))
    assert lib.tdes_ctx_create(kt.handle, ctypes.byref(cfg), ctypes.byref(ctx)) == 0
    ticket = ctypes.c_uint64()
    assert lib.tdes_batch_submit(ctx, ctypes.addressof(allc), n + 3, ctypes.byref(ticket)) == 0
    per = np.full(n + 3, 7, dtype=np.int32)
    r = lib.tdes_batch_poll(ctx, ticket.value, per.ctypes.data)
    assert r in (1, T.TDES_EINVAL)
    assert set(np.unique(per[:n])) <= {0, 1}            # valid ones: done or pending
    assert (per[n:] == T.TDES_EINVAL).all()             # rejected at submission
    assert lib.tdes_batch_wait(ctx, ticket.value, 60 * 10**9) == T.TDES_EINVAL
    assert lib.tdes_batch_poll(ctx, ticket.value, per.ctypes.data) == T.TDES_EINVAL
    assert (per[:n] == 0).all() and (per[n:] == T.TDES_EINVAL).all()
    want = expected(keys, lens, modes, kidx, ivs, offs, src.cpu().numpy())
    got = dst.cpu().numpy()
    for i in range(n):
        o, nb = int(offs[i]), int(lens[i])
        assert (got[o:o + nb] == want[o:o + nb]).all(), f"message {i} mode {modes[i]}"
    assert lib.tdes_batch_release(ctx, ticket.value) == 0
    assert lib.tdes_batch_poll(ctx, ticket.value, None) == T.TDES_EINVAL  # released
    lib.tdes_ctx_destroy(ctx)


def test_bounded_waits(cuda_lib):
    """A ticket not issued yet reads as pending and its wait runs out; a short
    wait on a batch holding a long serial CBC-encryption chain (2^18 blocks,
    about a quarter of a second) runs out too, and a long wait then returns
    the batch's status, with the chain equal to the oracle's."""
    T = cuda_lib
    keys = synth.key_triples(43, 2)
    kt = T.KeyTable(keys)
    ctx = T.Ctx(kt)
    assert ctx.wait(10**6, 0.005) == T.TDES_ETIMEDOUT       # never issued
    assert ctx.poll(10**6, 0)[0] == 1
    nb = 1 << 18
    data = synth.random_bytes(43, 8 * nb)
    x = torch.from_numpy(data).cuda()
    y = torch.zeros_like(x)
    iv = synth.iv64(43)
    torch.cuda.synchronize()
    t = ctx.submit([(4, 1, iv, x, y, 8 * nb)])
    assert ctx.wait(t, 0.001) == T.TDES_ETIMEDOUT
    assert ctx.release(t) == T.TDES_EBUSY                   # still pending
    assert ctx.wait(t, 60.0) == 0
    r, per = ctx.poll(t)
    assert r == 0 and (per == 0).all()
    want = oracle.tdes_cbc_encrypt(keys[1].tobytes(), iv, data)
    assert (y.cpu().numpy() == want).all()
    # the context is still usable: an empty batch completes at once
    t2 = ctx.submit([])
    assert ctx.wait(t2, 1.0) == 0
    ctx.close()


def test_tickets_in_flight_together_and_planned_batch(cuda_lib):
    """Eight batches submitted back to back without waiting (two streams),
    collected in reverse order; then a batch planned with tdes_batch_plan is
    submitted twice under tickets (its graph replayed on a context stream).
    Every message against the oracle."""
    T = cuda_lib
    seed, n_keys = 47, 31
    keys = synth.key_triples(seed, n_keys)
    kt = T.KeyTable(keys)
    ctx = T.Ctx(kt, streams=2)
    jobs = []
    for j in range(8):
        lens, modes, kidx, ivs, offs, data = mixed_workload(seed + j, 120, 64 << 10, n_keys)
        src = torch.from_numpy(data).cuda()
        dst = torch.zeros_like(src)
        ents = [(int(modes[i]), int(kidx[i]), int(ivs[i]), src.data_ptr() + int(offs[i]),
                 dst.data_ptr() + int(offs[i]), int(lens[i])) for i in range(len(lens))]
        torch.cuda.synchronize()
        jobs.append((ctx.submit(ents), (lens, modes, kidx, ivs, offs, data), src, dst))
    tickets = [j[0] for j in jobs]
    assert tickets == list(range(tickets[0], tickets[0] + 8))
    for t, w, src, dst in reversed(jobs):
        assert ctx.wait(t, 60.0) == 0
        lens, modes, kidx, ivs, offs, data = w
        want = expected(keys, lens, modes, kidx, ivs, offs, data)
        got = dst.cpu().numpy()
        for i in range(len(lens)):
            o, nb = int(offs[i]), int(lens[i])
            assert (got[o:o + nb] == want[o:o + nb]).all(), f"ticket {t} message {i}"
    # a planned batch under tickets
    lens, modes, kidx, ivs, offs, data = mixed_workload(seed + 99, 200, 256 << 10, n_keys)
    src = torch.from_numpy(data).cuda()
    dst = torch.zeros_like(src)
    ents = [(int(modes[i]), int(kidx[i]), int(ivs[i]), src.data_ptr() + int(offs[i]),
             dst.data_ptr() + int(offs[i]), int(lens[i])) for i in range(len(lens))]
    b = T.Batch(kt, ents)
    want = expected(keys, lens, modes, kidx, ivs, offs, data)
    for _ in range(2):
        dst.zero_()
        torch.cuda.synchronize()
        t = ctx.submit_plan(b)
        assert ctx.wait(t, 60.0) == 0
        r, per = ctx.poll(t)
        assert r == 0 and len(per) == len(lens) and (per == 0).all()
        got = dst.cpu().numpy()
        for i in range(len(lens)):
            o, nb = int(offs[i]), int(lens[i])
            assert (got[o:o + nb] == want[o:o + nb]).all(), f"planned message {i}"
    ctx.close()


def test_many_submissions_with_host_heap_churn(cuda_lib):
    """Thirty batches submitted back to back while the host allocates and
    frees memory between submissions: a plan's host image must stay intact
    until its copy to the device has run (on a GPU that reads host memory
    directly the copy may run after the call returns).  Every message against
    the oracle."""
    T = cuda_lib
    seed, n_keys = 53, 17
    keys = synth.key_triples(seed, n_keys)
    kt = T.KeyTable(keys)
    ctx = T.Ctx(kt, streams=3)
    jobs, junk = [], []
    for j in range(30):
        lens, modes, kidx, ivs, offs, data = mixed_workload(seed + j, 60, 32 << 10, n_keys)
        src = torch.from_numpy(data).cuda()
        dst = torch.zeros_like(src)
        ents = [(int(modes[i]), int(kidx[i]), int(ivs[i]), src.data_ptr() + int(offs[i]),
                 dst.data_ptr() + int(offs[i]), int(lens[i])) for i in range(len(lens))]
        torch.cuda.synchronize()
        # src and dst stay referenced until the ticket completes: the context's
        # streams are not ordered with torch's, whose allocator would hand a
        # freed input to the next tensor while the batch still reads it
        jobs.append((ctx.submit(ents), (lens, modes, kidx, ivs, offs, data), src, dst))
        junk = [bytearray(b"\xa5" * (4096 + 64 * k)) for k in range(64)]  # reuse freed chunks
    del junk
    for t, w, src, dst in jobs:
        assert ctx.wait(t, 60.0) == 0
        lens, modes, kidx, ivs, offs, data = w
        want = expected(keys, lens, modes, kidx, ivs, offs, data)
        got = dst.cpu().numpy()
        for i in range(len(lens)):
            o, nb = int(offs[i]), int(lens[i])
            assert (got[o:o + nb] == want[o:o + nb]).all(), f"ticket {t} message {i}"
    ctx.close()


def test_in_place_halo_and_direct_messages(cuda_lib):
    """A context batch with in-place CBC decryption over several tiles (the
    per-tile snapshot runs first), a 64 MiB ECB message and a 64 MiB CTR
    message (run by the single-key kernels inside the batch) and small
    messages, in place and out of place: every byte against the oracle (the
    large ones on 2^16 sampled blocks and their first and last tiles)."""
    T = cuda_lib
    keys = synth.key_triples(59, 5)
    kt = T.KeyTable(keys)
    ctx = T.Ctx(kt)
    big = 64 << 20
    plan = [(3, 0, 6000 * 8, True), (3, 1, 1025 * 8, True), (0, 2, big, False), (2, 3, big, True),
            (1, 4, 4096, True), (4, 0, 700 * 8, False), (0, 1, 24, True)]
    bufs, ents, datas = [], [], []
    for j, (mode, key, nbytes, in_place) in enumerate(plan):
        data = synth.random_bytes(5900 + j, nbytes)
        iv = int(synth.words(59, j, 1, synth.STREAM_IV)[0])
        if mode == 2:
            iv &= 0xFFFFFFFF00000000
        x = torch.from_numpy(data).cuda()
        y = x if in_place else torch.zeros_like(x)
        bufs.append((x, y))
        datas.append((mode, key, iv, data))
        ents.append((mode, key, iv, x, y, nbytes))
    torch.cuda.synchronize()
    t = ctx.submit(ents)
    assert ctx.wait(t, 60.0) == 0
    rng = np.random.default_rng(59)
    for (x, y), (mode, key, iv, data) in zip(bufs, datas):
        k = keys[key].tobytes()
        got = y.cpu().numpy()
        if data.size <= (1 << 20):
            want = {0: lambda: oracle.tdes_ecb(k, data),
                    1: lambda: oracle.tdes_ecb(k, data, decrypt=True),
                    2: lambda: oracle.tdes_ctr(k, iv >> 32, iv & 0xFFFFFFFF, data),
                    3: lambda: oracle.tdes_cbc_decrypt(k, iv, data),
                    4: lambda: oracle.tdes_cbc_encrypt(k, iv, data)}[mode]()
            assert (got == want).all(), f"mode {mode}, {data.size} bytes"
            continue
        nb = data.size // 8
        blocks = np.concatenate([np.arange(1024), np.arange(nb - 1024, nb),
                                 rng.integers(0, nb, 1 << 16)])
        for b in np.unique(blocks)[::7]:
            blk = data[8 * b:8 * b + 8]
            if mode == 0:
                w = oracle.tdes_ecb(k, blk)
            else:
                w = oracle.tdes_ctr(k, iv >> 32, (iv & 0xFFFFFFFF) + int(b), blk)
            assert (got[8 * b:8 * b + 8] == w).all(), f"mode {mode} block {b}"
    ctx.close()


def test_resubmitted_plan_runs_in_order(cuda_lib):
    """One in-place plan (ECB both ways, CTR, CBC decryption over several
    tiles) submitted three times back to back on a two-stream context, then
    waited on.  Each run reads what the run before it wrote, so the bytes
    must equal the oracle applied three times in a row: two runs of one plan
    overlapping on two streams would share its claim counter and halo
    snapshot and skip or repeat tiles.  The caller drops its Batch right
    after submitting: the context holds the plan until the tickets are
    released."""
    T = cuda_lib
    seed, n, n_keys = 61, 48, 11
    keys = synth.key_triples(seed, n_keys)
    lens = synth.log_uniform_lengths(seed, n, 64, 1 << 20)
    modes = synth.categorical(seed, n, [0.3, 0.2, 0.2, 0.3], synth.STREAM_MODE).astype(np.uint8)
    kidx = (synth.u64s(seed, n, synth.STREAM_KEYPICK) % np.uint64(n_keys)).astype(np.uint32)
    ivs = synth.u64s(seed, n, synth.STREAM_IV)
    ivs = np.where(modes == 2, ivs & np.uint64(0xFFFFFFFF00000000), ivs).astype(np.uint64)
    offs = np.concatenate([[0], np.cumsum((lens + 15) // 16 * 16)])[:-1].astype(np.uint64)
    data = synth.random_bytes(seed, int(offs[-1] + lens[-1]) + 16)
    kt = T.KeyTable(keys)
    ctx = T.Ctx(kt, streams=2)
    x = torch.from_numpy(data).cuda()
    ents = [(int(modes[i]), int(kidx[i]), int(ivs[i]), x.data_ptr() + int(offs[i]),
             x.data_ptr() + int(offs[i]), int(lens[i])) for i in range(n)]
    b = T.Batch(kt, ents)
    torch.cuda.synchronize()
    tickets = [ctx.submit_plan(b) for _ in range(3)]
    del b  # the context keeps the plan until its tickets are released
    gc.collect()
    for t in tickets:
        assert ctx.wait(t, 60.0) == 0
    for t in tickets:
        assert ctx.release(t) == 0
    want = data
    for _ in range(3):
        want = expected(keys, lens, modes, kidx, ivs, offs, want)
    got = x.cpu().numpy()
    for i in range(n):
        o, nb = int(offs[i]), int(lens[i])
        assert (got[o:o + nb] == want[o:o + nb]).all(), f"message {i} (mode {modes[i]})"
    ctx.close()
