#!/usr/bin/env python
"""3DES-EDE3 benchmark on GB300: GB/s of the 1 GiB single-key ECB workload.

Workload (one step): ECB encryption of a 1 GiB buffer (2^27 big-endian
64-bit blocks) of seeded uniform-random bytes under one seeded key triple,
input and output resident in HBM, one launch of the bitsliced ECB kernel
through the C ABI (tdes_ecb_encrypt).  The input (1 GiB) is larger than the
129 MB L2, so no flush is needed between steps.

Reported beside it: the same pass decrypting and in CTR mode, the 1 MiB
single-launch latency, the key-schedule time, an end-to-end number through
the host-buffer entry point (tdes_ecb_crypt_host, pinned host memory, every
byte copied host->device and back inside the timed region), the ALU
roofline of the dominant kernel against a live LOP3-throughput probe, and
the CPU oracle's throughput on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) every rank encrypts its own 1 GiB
(replicas: the cipher needs no exchange between GPUs); value = all bytes /
the slowest rank's time.  --impl reference times the CPU oracle (the plain
reference implementation of the paper's method) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3DES GB/s: 1 GiB ECB and batched serve (p50/p99 ms) vs plain ECB, bit-exact"
WORKLOAD = ("3DES-EDE3 ECB encrypt of 1 GiB (2^27 big-endian 64-bit blocks) of seeded "
            "uniform random bytes, one seeded key triple with odd-parity bytes")
NBYTES = 1 << 30
SEED = 2
HBM_FALLBACK_GBS = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def start_clock_sampler(device_id: str | None):
    cmd = ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
           "-lms", "100"]
    if device_id:
        cmd.insert(1, f"--id={device_id}")
    try:
        return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def stop_clock_sampler(p):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out, _ = p.communicate()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
            "reasons": sorted(reasons)}


def gpu_id_for_smi(torch, dev: int):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# --------------------------------------------------------------- CPU oracle
def cpu_baseline(keys: bytes, seconds: float = 12.0):
    """The oracle as it stands, single-threaded and over all host cores."""
    import oracle
    from paper_2007_10752_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    # calibrate on 64 KiB, then size each sample for about seconds/2
    probe = synth.random_bytes(SEED, 1 << 16)
    t = time.perf_counter()
    oracle.tdes_parallel(keys, probe, "ecb_enc", threads=1)
    rate1 = (1 << 16) / max(time.perf_counter() - t, 1e-6)
    n1 = int(min(max(rate1 * seconds / 2, 1 << 16), 64 << 20)) // 8 * 8
    n_mt = int(min(max(rate1 * cores * seconds / 2, 1 << 16), 512 << 20)) // 8 * 8
    s1 = synth.random_bytes(SEED, n1)
    t = time.perf_counter()
    oracle.tdes_parallel(keys, s1, "ecb_enc", threads=1)
    g1 = n1 / (time.perf_counter() - t) / 1e9
    smt = synth.random_bytes(SEED, n_mt)
    t = time.perf_counter()
    oracle.tdes_parallel(keys, smt, "ecb_enc", threads=cores)
    gmt = n_mt / (time.perf_counter() - t) / 1e9
    return {"value": gmt, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": (f"ECB encrypt of the first {n_mt} bytes of the 1 GiB workload over "
                       f"{cores} threads; single-thread: {g1:.6f} GB/s on the first {n1} bytes"),
            "single_thread_gbs": g1}


def openssl_reference(keys: bytes, data, gpu_out, seconds: float = 6.0):
    """OpenSSL's DES-EDE3 ECB (libcrypto EVP) on the host cores, if the library
    is there: a practical CPU implementation for context (not the oracle).  Its
    output on the first MiB is compared with the GPU's output of the timed step."""
    import ctypes
    import ctypes.util
    import threading
    name = ctypes.util.find_library("crypto")
    if not name:
        return {"unavailable": "libcrypto not found on this host"}
    lib = ctypes.CDLL(name)
    vp, cp, ip = ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)
    lib.EVP_CIPHER_CTX_new.restype = vp
    lib.EVP_des_ede3_ecb.restype = vp
    lib.EVP_EncryptInit_ex.argtypes = [vp, vp, vp, cp, cp]
    lib.EVP_CIPHER_CTX_set_padding.argtypes = [vp, ctypes.c_int]
    lib.EVP_EncryptUpdate.argtypes = [vp, vp, ip, vp, ctypes.c_int]
    lib.EVP_CIPHER_CTX_free.argtypes = [vp]
    cipher = lib.EVP_des_ede3_ecb()
    if not cipher:
        return {"unavailable": "DES-EDE3 not offered by this libcrypto"}

    def run(src, dst):
        ctx = lib.EVP_CIPHER_CTX_new()
        lib.EVP_EncryptInit_ex(ctx, cipher, None, keys, None)
        lib.EVP_CIPHER_CTX_set_padding(ctx, 0)
        outl = ctypes.c_int(0)
        chunk = 1 << 24
        for off in range(0, len(src), chunk):
            n = min(chunk, len(src) - off)
            lib.EVP_EncryptUpdate(ctx, ctypes.c_void_p(dst.ctypes.data + off), ctypes.byref(outl),
                                  ctypes.c_void_p(src.ctypes.data + off), n)
        lib.EVP_CIPHER_CTX_free(ctx)

    import numpy as np
    head = data[: 1 << 20]
    out = np.empty_like(head)
    run(head, out)
    agrees = bool((out == gpu_out[: 1 << 20]).all())
    t = time.perf_counter()
    run(head, out)
    rate1 = head.size / max(time.perf_counter() - t, 1e-6)
    n1 = int(min(max(rate1 * seconds / 2, 1 << 20), data.size)) // 8 * 8
    buf = np.empty(n1, dtype=np.uint8)
    t = time.perf_counter()
    run(data[:n1], buf)
    g1 = n1 / (time.perf_counter() - t) / 1e9
    cores = os.cpu_count() or 1
    per = n1 // cores // 8 * 8
    outs = [np.empty(per, dtype=np.uint8) for _ in range(cores)]
    ths = [threading.Thread(target=run, args=(data[i * per:(i + 1) * per], outs[i]))
           for i in range(cores)]
    t = time.perf_counter()
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    gn = per * cores / (time.perf_counter() - t) / 1e9
    return {"kind": "openssl EVP des-ede3-ecb", "version": int(lib.OpenSSL_version_num()),
            "gbs_1_thread": round(g1, 4), "gbs_all_threads": round(gn, 4), "threads": cores,
            "sample_bytes": n1, "agrees_with_gpu_on_first_mib": agrees}


# ---------------------------------------------------------------- roofline
def alg_ops_per_32_blocks(stages: int = 3) -> int:
    """Logic-pipe operations the bitsliced ECB algorithm needs per 32 blocks.

    16 x stages rounds (48 for EDE3, 16 for single DES) x (8 S-box circuits
    of G LOP3 in total + 32 fused XOR updates), 4 bit-matrix transposes x 256
    operations, and (stages + 1) x 32 key-mask XORs (prologue, re-keyings,
    epilogue, one half each).  The 16 doubled expansion inputs per round are
    XORed on the integer multiply-add pipe and not counted.
    """
    with open(os.path.join(ROOT, "paper_2007_10752_gb300", "gen", "sbox_lop3.json")) as f:
        g = sum(len(s["gates"]) for s in json.load(f)["sboxes"])
    return 16 * stages * (g + 32) + 4 * 256 + (stages + 1) * 32


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_10752_gb300", "csrc")
    for rel in ("tdes_kernels.cu", "tdes_bitslice.cuh", "generated/tdes_generated.cuh"):
        with open(os.path.join(csrc, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per ECB launch from the committed ncu summary, if it is for this kernel."""
    path = os.path.join(ROOT, "profiles", "tdes_ecb_kernel_256mib.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def probe_alu_peak():
    import ctypes
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2007_10752_gb300", "libtdes_tools.so"))
    lib.tdes_tools_lop3_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_float)]
    best = 0.0
    for ctas in (4, 8):
        ops, ms = ctypes.c_double(), ctypes.c_float()
        rc = lib.tdes_tools_lop3_rate(ctas, 256, 4000, ctypes.byref(ops), ctypes.byref(ms))
        if rc == 0:
            best = max(best, ops.value)
    return best


# ------------------------------------------------------------- multi-rank
def reduce_max(x: float, device: str) -> float:
    """Max of x over all ranks of the default process group (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_rank: int, world: int, slowest_s: float) -> float:
    """Whole-job GB/s: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank / slowest_s / 1e9


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2007_10752_gb300 import build as b
    from paper_2007_10752_gb300 import synth, tdes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    b.build()
    tdes.load()
    dev = torch.cuda.current_device()

    keys = synth.key_triple(SEED)
    host = synth.random_bytes(SEED, NBYTES)
    x = torch.from_numpy(host).to(f"cuda:{dev}")
    y = torch.empty_like(x)
    t0 = time.perf_counter()
    ks = tdes.KeySchedule.from_triple(keys)
    keysched_ms = (time.perf_counter() - t0) * 1e3
    stream = torch.cuda.current_stream()

    def ecb_step():
        tdes.tdes_ecb_encrypt(ks, x, y)

    for _ in range(args.warmup):
        ecb_step()
    torch.cuda.synchronize()
    alu_peak = probe_alu_peak() if rank == 0 else 0.0

    # ---- timed region: K ECB launches, an event pair around each
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = start_clock_sampler(gpu_id_for_smi(torch, dev))
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for e0, e1 in evs:
        e0.record(stream)
        ecb_step()
        e1.record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = stop_clock_sampler(sampler)
    total_ms = start.elapsed_time(end)
    if world > 1:
        total_ms = reduce_max(total_ms, f"cuda:{dev}")
    per_launch_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
    ms_per_step = total_ms / args.steps
    value = job_throughput(NBYTES, world, ms_per_step * 1e-3)

    # the timed output decrypts back to the input (parity with the oracle is
    # the test suite's job)
    z = torch.empty_like(y)
    tdes.tdes_ecb_decrypt(ks, y, z)
    torch.cuda.synchronize()
    assert torch.equal(z, x), "ECB decrypt(encrypt(x)) != x"
    ecb_out = y[: 1 << 20].cpu().numpy()  # checked against OpenSSL on the host below
    del z

    # ---- other modes of the same workload, and the 1 MiB single launch
    def time_fn(fn, n):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    nonce = synth.nonce32(SEED)
    dec_ms = time_fn(lambda: tdes.tdes_ecb_decrypt(ks, x, y), 50)
    ctr_ms = time_fn(lambda: tdes.tdes_ctr_crypt(ks, nonce, 0, x, y), 50)
    cbc_dec_ms = time_fn(lambda: tdes.tdes_cbc_decrypt(ks, synth.iv64(SEED), x, y), 50)
    small_in, small_out = x[: 1 << 20], y[: 1 << 20]
    small_us = graph_call_ms(torch, lambda: tdes.tdes_ecb_encrypt(ks, small_in, small_out)) * 1e3
    small_call_us = time_fn(lambda: tdes.tdes_ecb_encrypt(ks, small_in, small_out), 200) * 1e3

    # ---- one serial CBC-encryption chain through the single-message call
    n_chain = 1 << 16
    chain_ms = time_fn(lambda: tdes.tdes_cbc_encrypt(ks, 5, x[: 8 * n_chain], y[: 8 * n_chain]), 2)

    # ---- single DES (a DES schedule, or a triple that reduces): one pass
    kd = tdes.KeySchedule.des(keys[:8])
    des_ms = time_fn(lambda: tdes.tdes_ecb_encrypt(kd, x, y), 50)
    kd.free()

    # ---- batched: 4096 messages with their own keys and modes, one launch
    batched = None if args.no_batch else run_batched(torch, tdes, synth, stream, value)

    # ---- large streaming: 32 GiB in place, CTR stream + 2^20 small messages
    streaming = None if args.no_stream else run_streaming(torch, tdes, synth, stream)
    if streaming is not None:
        streaming["uniform_reading"] = run_streaming_uniform(torch, tdes, synth)

    # ---- serving: Poisson arrivals at fractions of the measured peak
    serving = None if args.no_serve else run_serving(torch, tdes, synth, x)

    # ---- context: the paper's own design on this GPU, at the paper's sizes
    paper_ctx = None if args.no_paper else run_paper_context(torch, tdes, synth, x, y, ks, stream)

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        hbuf = torch.from_numpy(host.copy()).pin_memory()
        dev_buf = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
        tdes.tdes_ecb_crypt_host(ks, False, hbuf, hbuf, dev_buf)  # warm-up
        # Each call timed on its own and the median kept: the host link and
        # host memory are shared with the GPU's neighbour on the same host,
        # and calls sometimes met a slowdown (a mean of 3 calls once read 142
        # against 157-159 GB/s; in another run plain host-to-device copies ran
        # at 22 GB/s for a while).  Every call's rate is reported.
        n_e2e = 9
        if world > 1:
            dist.barrier()
        calls = []
        for _ in range(n_e2e):
            t = time.perf_counter()
            tdes.tdes_ecb_crypt_host(ks, False, hbuf, hbuf, dev_buf)
            calls.append(time.perf_counter() - t)
        el = float(np.median(calls))
        if world > 1:
            el = reduce_max(el, f"cuda:{dev}")
        # the copies alone, for context: the host link bounds the end-to-end number
        dbuf = torch.empty(NBYTES, dtype=torch.uint8, device=f"cuda:{dev}")
        torch.cuda.synchronize()

        def copy_gbs(dst, src):  # median of three timed copies
            r = []
            for _ in range(3):
                t = time.perf_counter()
                dst.copy_(src, non_blocking=True)
                torch.cuda.synchronize()
                r.append(NBYTES / (time.perf_counter() - t) / 1e9)
            return float(np.median(r))

        h2d = copy_gbs(dbuf, hbuf)
        d2h = copy_gbs(hbuf, dbuf)
        del dbuf
        e2e = {"value": world * NBYTES / el / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": NBYTES, "d2h_bytes_per_step": NBYTES,
               "api": "tdes_ecb_crypt_host (pinned host buffer in place, 256 MiB device staging)",
               "statistic": f"median of {n_e2e} calls, each timed on its own",
               "calls_gbs": [round(NBYTES / c / 1e9, 1) for c in calls],
               "copy_only_h2d_gbs": round(h2d, 1), "copy_only_d2h_gbs": round(d2h, 1)}
        del hbuf, dev_buf

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk, pk_kind = peaks()
    ops = alg_ops_per_32_blocks() * (NBYTES // 8 // 32)
    achieved = ops / (per_launch_ms * 1e-3) / 1e12
    # ALU peak from unit counts and clock: SMs x 64 logic lanes per SM per clock
    # (the lane count the live probe measures) x the maximum SM clock
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = sms * 64 * max_mhz * 1e6 / 1e12
    probe_lanes = alu_peak / (sms * max_mhz * 1e6) if alu_peak else None
    hbm_gbs = 16 * (NBYTES // 8) / (per_launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic()
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "ECB encrypt", "bytes_per_gpu": NBYTES,
                   "l2": "input 1 GiB per step > 129 MB L2: no flush needed",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                     "unit": "Tops/s", "frac": round(achieved / peak, 4) if peak else None,
                     "traffic": traffic,
                     "peak_source": (f"{sms} SMs x 64 LOP3 lanes/clk x {max_mhz:.0f} MHz "
                                     "(max SM clock, MEASURED_PEAKS.json)"),
                     "peak_probe": round(alu_peak / 1e12, 3),
                     "probe_lanes_per_sm_clk": round(probe_lanes, 2) if probe_lanes else None,
                     "alg_ops_per_32_blocks": alg_ops_per_32_blocks(),
                     "hbm_achieved_gbs": round(hbm_gbs, 1),
                     "hbm_peak_gbs": pk.get("hbm_gbs"),
                     "hbm_frac": round(hbm_gbs / pk.get("hbm_gbs", HBM_FALLBACK_GBS), 4),
                     "hbm_peak_source": pk_kind},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "paper_design_context": paper_ctx,
        "extra": {"kernel_ms_per_launch": round(per_launch_ms, 4),
                  "ecb_decrypt_gbs": round(NBYTES / (dec_ms * 1e-3) / 1e9, 3),
                  "ctr_gbs": round(NBYTES / (ctr_ms * 1e-3) / 1e9, 3),
                  "cbc_decrypt_gbs": round(NBYTES / (cbc_dec_ms * 1e-3) / 1e9, 3),
                  "ecb_1mib_single_launch_us": round(small_us, 2),
                  "ecb_1mib_python_call_us": round(small_call_us, 2),
                  "cbc_encrypt_chain_ns_per_block": round(chain_ms * 1e6 / n_chain, 1),
                  "key_schedule_ms": round(keysched_ms, 3),
                  "sbox_lop3_per_round": tdes.tdes_sbox_gate_count()},
    }
    des_ops = alg_ops_per_32_blocks(1) * (NBYTES // 8 // 32)
    line["single_des"] = {
        "workload": "DES ECB encrypt of the same 1 GiB under the triple's first key "
                    "(tdes_des_key_schedule; EDE3 triples with K1 = K2 or K2 = K3 take the "
                    "same 16-round path)",
        "gbs": round(NBYTES / (des_ms * 1e-3) / 1e9, 3),
        "ms": round(des_ms, 4),
        "alg_ops_per_32_blocks": alg_ops_per_32_blocks(1),
        "alu_achieved": round(des_ops / (des_ms * 1e-3) / 1e12, 3),
        "alu_frac": round(des_ops / (des_ms * 1e-3) / 1e12 / peak, 4) if peak else None,
        "vs_ede3": round(per_launch_ms / des_ms, 3),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(keys)
        line["cpu_library_reference"] = openssl_reference(keys, host, ecb_out)
    line["batched"] = batched
    line["serving"] = serving
    line["large_streaming"] = streaming
    line["summary"] = summary(line)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def summary(line: dict) -> dict:
    """The headline figures of every workload in a few hundred bytes, printed
    last so that a truncated copy of the line still carries them."""
    out = {"ecb_1gib_gbs": line["value"], "roofline_frac": line["roofline"]["frac"],
           "e2e_gbs": round(line["e2e"]["value"], 1) if line.get("e2e") else None}
    b = line.get("batched")
    if b:
        out["batched"] = {"parallel_gbs": b["parallel_modes_gbs"],
                          "vs_ecb": b["parallel_modes_vs_plain_ecb"],
                          "makespan_ms": b["makespan_ms"],
                          "tuned_gain": b["autotune"]["gain"]}
    sv = line.get("serving")
    if sv:
        out["serving"] = {"peak_gbs": sv["peak_closed_loop_gbs"],
                          "p50_p99_ms": {str(p["load"]): [p["p50_ms"], p["p99_ms"]]
                                         for p in sv["points"]},
                          "gbs_at_0.95": sv["points"][-1]["achieved_gbs"],
                          "max_slots_busy": max(p["max_slots_busy"] for p in sv["points"])}
    st = line.get("large_streaming")
    if st:
        u = st.get("uniform_reading") or {}
        out["streaming"] = {"gbs": st["gbps"], "uniform_msgs_gbs": u.get("messages_gbps"),
                            "uniform_all_gbs": u.get("gbps")}
    return out


# ---------------------------------------------------------------- batched
BATCH_WORKLOAD = ("4096 messages, lengths log-uniform 64 B..4 MiB (multiples of 8), uniform "
                  "random payloads, own seeded key triple each, modes ECB 40% / CTR 30% / "
                  "CBC-decrypt 20% / CBC-encrypt 10%, seeded IVs; one persistent launch "
                  "replayed as a CUDA graph")


def graph_call_ms(torch, fn, calls=20, reps=5):
    """Device time per call of `fn` (one library call on the current stream):
    `calls` calls captured in a CUDA graph and replayed, so that the host's
    per-call overhead (Python, argument checks, launch) does not pace the GPU."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        for _ in range(calls):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * calls)


def time_graph(torch, batch, stream, reps):
    batch.launch_graph(stream)  # capture + warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        batch.launch_graph(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_batched(torch, tdes, synth, stream, ecb_gbs):
    """Config-3 batch: whole-batch makespan, and the parallel modes alone."""
    from paper_2007_10752_gb300.workloads import build_batched
    src, dst, kt, ents, lens, modes = build_batched(torch, tdes)
    total = int(lens.sum())
    par = ents[ents["mode"] != 4]
    par_bytes = int(par["nbytes"].sum())
    # the library's autotuner on the parallel-mode part (the throughput part;
    # out of place, so its repeated runs leave the inputs intact): it times
    # the candidate shapes and stores the winner in the cache, then the whole
    # batch runs in the same shape
    bpar = tdes.Batch(kt, par)
    tune = bpar.autotune(reps=5, flags=tdes.TUNE_FORCE)
    par_ms = time_graph(torch, bpar, stream, 20)
    default_shape = tune["baseline"]
    bdef = tdes.Batch(kt, par)
    bdef.set_shape(default_shape["warps_per_cta"], default_shape["ctas_per_sm"],
                   default_shape["tiles_per_claim"], default_shape["round_form"])
    par_default_ms = time_graph(torch, bdef, stream, 20)
    del bdef
    ball = tdes.Batch(kt, ents)
    best = tune["best"]
    ball.set_shape(best["warps_per_cta"], best["ctas_per_sm"], best["tiles_per_claim"],
                   best["round_form"])
    all_ms = time_graph(torch, ball, stream, 2)
    cbc = ents[ents["mode"] == 4]
    longest = int(cbc["nbytes"].max()) if len(cbc) else 0
    bc = tdes.Batch(kt, cbc[[int(np.argmax(cbc["nbytes"]))]]) if len(cbc) else None
    chain_ms = time_graph(torch, bc, stream, 2) if bc else 0.0
    par_gbs = par_bytes / (par_ms * 1e-3) / 1e9
    info = ball.info()
    return {
        "workload": BATCH_WORKLOAD,
        "messages": len(ents), "bytes": total,
        "makespan_ms": round(all_ms, 3), "makespan_gbs": round(total / (all_ms * 1e-3) / 1e9, 3),
        "parallel_modes_bytes": par_bytes, "parallel_modes_ms": round(par_ms, 3),
        "parallel_modes_gbs": round(par_gbs, 3),
        "parallel_modes_vs_plain_ecb": round(par_gbs / ecb_gbs, 4),
        "cbc_encrypt_longest_bytes": longest,
        "cbc_encrypt_longest_chain_ms": round(chain_ms, 3),
        "cbc_encrypt_ns_per_block": round(chain_ms * 1e6 / max(1, longest // 8), 1),
        "autotune": {"class": tune["key"], "tuned_shape": tune["best"],
                     "default_shape": default_shape, "candidates": tune["candidates"],
                     "tuned_ms": round(par_ms, 3), "default_ms": round(par_default_ms, 3),
                     "gain": round(par_default_ms / par_ms, 4),
                     "cache": tdes.tdes_autotune_cache_path()},
        "tiles": info["n_tiles"], "small_items": info["n_small_items"],
        "cbc_encrypt_messages": info["n_cbc_enc_messages"],
    }


# -------------------------------------------- paper's design, as context
# Table I, GPU-1 (RTX 2060 Super) of the paper: 3DES ECB encryption time in ms
# (three kernel launches) for 2^2 .. 2^17 blocks.
PAPER_TABLE1_GPU1_MS = [0.032, 0.033, 0.033, 0.032, 0.033, 0.032, 0.035, 0.050, 0.089, 0.161,
                        0.305, 0.592, 1.184, 2.324, 4.511, 8.399]


def run_paper_context(torch, tdes, synth, x, y, ks, stream):
    """The paper's kernels (one CTA per block, a thread per bit, three launches)
    rebuilt on this GB300, against this library at Table I's sizes: its default
    dispatch, and each of its two single-key paths forced (bitsliced tiles; one
    block per thread), which also shows where the small-call cutoff belongs."""
    from paper_2007_10752_gb300 import paper_design
    keys = synth.key_triple(SEED)

    def ours(xs, ys, cutoff=None):
        prev = tdes.tdes_set_small_cutoff(cutoff) if cutoff is not None else None
        ms = graph_call_ms(torch, lambda: tdes.tdes_ecb_encrypt(ks, xs, ys))
        if prev is not None:
            tdes.tdes_set_small_cutoff(prev)
        return ms

    rows = []
    for e, paper_ms in zip(range(2, 18), PAPER_TABLE1_GPU1_MS):
        n = 8 << e
        xs, ys = x[:n], y[:n]
        times = sorted(paper_design.paper_ecb(keys, xs, ys) for _ in range(5))
        pd_ms = times[2]
        lib_ms = ours(xs, ys)
        bs_ms = ours(xs, ys, 0)
        sc_ms = ours(xs, ys, 1 << 40)
        rows.append({"blocks": 1 << e, "paper_table1_rtx2060s_ms": paper_ms,
                     "paper_design_gb300_ms": round(pd_ms, 4), "library_gb300_ms": round(lib_ms, 4),
                     "bitsliced_gb300_ms": round(bs_ms, 4),
                     "one_block_per_thread_gb300_ms": round(sc_ms, 4),
                     "speedup_vs_paper_design_gb300": round(pd_ms / lib_ms, 1)})
    cutoff = tdes.tdes_set_small_cutoff(0)
    tdes.tdes_set_small_cutoff(cutoff)
    return {"note": "paper's design rebuilt on GB300 (libtdes_tools.so); device times of its "
                    "three encryption launches vs one call of this library (default dispatch, "
                    "and each path forced), the latter replayed from a CUDA graph so that "
                    "host overhead does not pace it; Table I numbers are the paper's own "
                    "hardware, context only", "small_cutoff_blocks": cutoff, "rows": rows}


# ------------------------------------------------------- large streaming
STREAM_WORKLOAD = ("32 GiB seeded buffer in place: [0, 16 GiB) one single-key CTR stream, then "
                   "2^20 messages of 64 B under 65536 seeded key triples (ECB 40% / CTR 30% / "
                   "CBC-decrypt 20% / CBC-encrypt 10%); one batch plan replayed as one CUDA "
                   "graph (the stream through the single-key CTR kernel, the messages through "
                   "the mixed-key and persistent batch kernels)")


def run_streaming(torch, tdes, synth, stream, reps=5):
    from paper_2007_10752_gb300.workloads import STREAM_BYTES, STREAM_N_SMALL as N_SMALL
    from paper_2007_10752_gb300.workloads import build_streaming
    buf, kt, d, keys, nonce = build_streaming(torch, tdes)
    b = tdes.Batch(kt, d)
    ms = time_graph(torch, b, stream, reps)
    processed = STREAM_BYTES + 64 * N_SMALL
    info = b.info()
    # the CTR stream alone through the single-key entry point, same bytes
    ks = tdes.KeySchedule.from_triple(keys[-1].tobytes())
    x = buf[:STREAM_BYTES]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tdes.tdes_ctr_crypt(ks, nonce, 0, x, x)
    e0.record(stream)
    for _ in range(reps):
        tdes.tdes_ctr_crypt(ks, nonce, 0, x, x)
    e1.record(stream)
    torch.cuda.synchronize()
    ctr_ms = e0.elapsed_time(e1) / reps
    del buf, x
    torch.cuda.empty_cache()
    return {"workload": STREAM_WORKLOAD, "processed_bytes": processed,
            "ms": round(ms, 3), "gbps": round(processed / (ms * 1e-3) / 1e9, 3),
            "ctr_stream_alone_ms": round(ctr_ms, 3),
            "ctr_stream_alone_gbps": round(STREAM_BYTES / (ctr_ms * 1e-3) / 1e9, 3),
            "tiles": info["n_tiles"], "small_items": info["n_small_items"],
            "cbc_encrypt_messages": info["n_cbc_enc_messages"],
            "direct_messages": info["n_direct_messages"]}


UNIFORM_WORKLOAD = ("the same 32 GiB buffer in place: [0, 16 GiB) the single-key CTR stream, "
                    "[16 GiB, 32 GiB) read as 2^28 messages of 64 B under 65536 seeded key "
                    "triples (same mode mix; per-message key, mode and IV arrays drawn on the "
                    "device); tdes_uniform_crypt (plan and run on the device) and the CTR call "
                    "on two streams of one CUDA graph")


def run_streaming_uniform(torch, tdes, synth, reps=3):
    """Config 5, reading every byte of the second 16 GiB as a 64-byte message."""
    from paper_2007_10752_gb300 import workloads as W
    seed, n, n_keys = W.STREAM_SEED, W.STREAM_N_UNIFORM, W.STREAM_N_KEYS
    buf = torch.empty(W.STREAM_TOTAL, dtype=torch.uint8, device="cuda")
    synth.fill_device(buf, seed)
    keys = synth.key_triples(seed, n_keys + 1)  # the last triple keys the CTR stream
    kt = tdes.KeyTable(keys)
    k, md, v = W.uniform_arrays_device(torch, seed, n, n_keys)
    x_ctr, x_msg = buf[:W.STREAM_BYTES], buf[W.STREAM_BYTES:]
    scratch = torch.empty(tdes.tdes_uniform_scratch_bytes(kt, n, 64), dtype=torch.uint8,
                          device="cuda")
    skipped = torch.zeros(1, dtype=torch.int64, device="cuda")
    ks = tdes.KeySchedule.from_triple(keys[-1].tobytes())
    nonce = synth.nonce32(seed)
    torch.cuda.synchronize()

    def uniform():
        tdes.tdes_uniform_crypt(kt, k, md, v, x_msg, x_msg, 64, scratch=scratch, skipped=skipped)

    side = torch.cuda.Stream()

    def both():
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            tdes.tdes_ctr_crypt(ks, nonce, 0, x_ctr, x_ctr)
        uniform()
        torch.cuda.current_stream().wait_stream(side)

    uni_ms = graph_call_ms(torch, uniform, calls=1, reps=reps)
    both_ms = graph_call_ms(torch, both, calls=1, reps=reps)
    info = tdes.tdes_uniform_info(scratch)
    out = {"workload": UNIFORM_WORKLOAD, "messages": n,
           "messages_ms": round(uni_ms, 3),
           "messages_gbps": round(n * 64 / (uni_ms * 1e-3) / 1e9, 3),
           "processed_bytes": W.STREAM_TOTAL, "ms": round(both_ms, 3),
           "gbps": round(W.STREAM_TOTAL / (both_ms * 1e-3) / 1e9, 3),
           "skipped": int(skipped.item()), "plan": info}
    del buf, x_ctr, x_msg, k, md, v, scratch
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- serving
SERVE_WORKLOAD = ("open-loop Poisson arrivals; sizes 80% uniform 64 B..4 KiB, 20% log-uniform "
                  "64 KiB..16 MiB; key drawn per request from 16384 resident triples; modes "
                  "ECB/CTR/CBC-decrypt 1/3 each; 8 GiB admission budget; payloads resident "
                  "in HBM; latency = completion - scheduled arrival")


def run_serving(torch, tdes, synth, in_pool, n_points=100000, n_peak=20000):
    kt = tdes.KeyTable(synth.key_triples(4, 16384))
    out_pool = torch.empty(8 << 30, dtype=torch.uint8, device=in_pool.device)
    # the library's server autotuner on this request mix (closed loop); the
    # server below then starts in the tuned configuration by default
    # 50000 requests a run: with 20000 (about 200 samples above the 99th
    # percentile) the tuner's choice changed between calls
    tune = tdes.tdes_server_autotune(kt, in_pool, out_pool, 50000, flags=tdes.TUNE_FORCE,
                                     seed=11)
    srv = tdes.Server(kt, budget_bytes=8 << 30)
    srv.loadtest(in_pool, out_pool, 2000, 0.0, seed=99)  # warm-up
    # the closed-loop peak, which sets every load point: the median of three
    # runs of 50000 requests (one run of 20000 varied by about 5% between calls)
    peaks = sorted((srv.loadtest(in_pool, out_pool, 50000, 0.0, seed=sd) for sd in (5, 6, 7)),
                   key=lambda r: r["gbps"])
    peak = peaks[1]
    points = []
    for frac in (0.25, 0.5, 0.75, 0.95):
        r = srv.loadtest(in_pool, out_pool, n_points, frac * peak["gbps"], seed=int(frac * 100))
        points.append({"load": frac, "offered_gbs": round(r["offered_gbps"], 2),
                       "achieved_gbs": round(r["gbps"], 2),
                       "p50_ms": round(r["p50_ms"], 4), "p99_ms": round(r["p99_ms"], 4),
                       "p999_ms": round(r["p999_ms"], 4),
                       "small_p50_ms": round(r["small_p50_ms"], 4),
                       "small_p99_ms": round(r["small_p99_ms"], 4),
                       "large_p50_ms": round(r["large_p50_ms"], 4),
                       "large_p99_ms": round(r["large_p99_ms"], 4),
                       "requests": r["requests"], "batches": r["batches"],
                       "max_slots_busy": r["max_slots_busy"],
                       "max_device_overlap": r["max_device_overlap"],
                       "device_overlap_frac": round(r["device_overlap_frac"], 4),
                       "duration_s": round(r["duration_s"], 3)})
    # host payloads: request buffers in pinned host memory, read and written by
    # the kernels over the host link (the server's default; its optional device
    # staging measured lower closed-loop throughput)
    # The tuner's shape is chosen on device payloads; over the host link the
    # built-in shape (4 slots) is measured beside it.
    host_in = in_pool[: 1 << 30].cpu().pin_memory()
    host_out = torch.empty(2 << 30, dtype=torch.uint8).pin_memory()
    # Over the host link single runs now and then met a stall of a few ms (a
    # peak 25% low, or a p99 of 9.6 ms at half load, in 1 of 3 bench runs), so
    # the peak and the half-load point are each the median of three runs.
    def host_point(server):
        pk = sorted((server.loadtest(host_in, host_out, n_peak, 0.0, seed=sd) for sd in (7, 17, 27)),
                    key=lambda r: r["gbps"])[1]
        half = sorted((server.loadtest(host_in, host_out, n_points // 4, 0.5 * pk["gbps"], seed=sd)
                       for sd in (8, 18, 28)), key=lambda r: r["p99_ms"])[1]
        return pk, half

    hpeak, hhalf = host_point(srv)
    srv.close()
    builtin = {k: tune["baseline"][k] for k in ("warps_per_cta", "reserve_ctas_per_sm", "slots",
                                                 "round_form")}
    srv_b = tdes.Server(kt, budget_bytes=8 << 30, **builtin)
    bpeak, bhalf = host_point(srv_b)
    srv_b.close()
    del out_pool, host_in, host_out
    keys = ("warps_per_cta", "reserve_ctas_per_sm", "slots", "round_form")
    tuned = {k: tune["best"][k] for k in keys}
    default = {k: tune["baseline"][k] for k in keys}
    return {"workload": SERVE_WORKLOAD, "peak_closed_loop_gbs": round(peak["gbps"], 2),
            "peak_runs_gbs": [round(r["gbps"], 2) for r in peaks],
            "peak_p50_ms": round(peak["p50_ms"], 3),
            "peak_max_slots_busy": peak["max_slots_busy"],
            "peak_device_overlap_frac": round(peak["device_overlap_frac"], 4),
            "autotune": {"class": tune["key"], "tuned": tuned, "default": default,
                         "objective": "p99 at a common offered load, closed-loop GB/s >= 97% "
                                      "of the default's",
                         "load_gbs": round(tune["load_gbps"], 2),
                         "tuned_p99_ms": round(tune["best_p99_ms"], 4),
                         "default_p99_ms": round(tune["baseline_p99_ms"], 4),
                         "tuned_gbs": round(tune["best_gbps"], 2),
                         "default_gbs": round(tune["baseline_gbps"], 2),
                         "candidates": tune["candidates"]},
            "points": points,
            "host_payloads": {"note": "same request mix, payloads in pinned host memory "
                                      "(kernels access it over NVLink-C2C); tuned server, "
                                      "then the built-in shape; each figure the median of "
                                      "three runs",
                              "peak_closed_loop_gbs": round(hpeak["gbps"], 2),
                              "load_0.5": {"offered_gbs": round(hhalf["offered_gbps"], 2),
                                           "achieved_gbs": round(hhalf["gbps"], 2),
                                           "p50_ms": round(hhalf["p50_ms"], 4),
                                           "p99_ms": round(hhalf["p99_ms"], 4)},
                              "builtin_shape": builtin,
                              "builtin_peak_closed_loop_gbs": round(bpeak["gbps"], 2),
                              "builtin_load_0.5": {"offered_gbs": round(bhalf["offered_gbps"], 2),
                                                   "achieved_gbs": round(bhalf["gbps"], 2),
                                                   "p50_ms": round(bhalf["p50_ms"], 4),
                                                   "p99_ms": round(bhalf["p99_ms"], 4)}},
            "server": srv.config}


# ------------------------------------------------------------- reference
def run_reference(args):
    """The CPU oracle on the host cores: rank 0 only."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    from paper_2007_10752_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    keys = synth.key_triple(SEED)
    probe = synth.random_bytes(SEED, 1 << 16)
    t = time.perf_counter()
    oracle.tdes_parallel(keys, probe, "ecb_enc", threads=cores)
    rate = (1 << 16) / max(time.perf_counter() - t, 1e-6)
    # whole run about 60 s: size each step's sample from the calibration
    per_step = int(min(max(rate * 60.0 / (args.steps + args.warmup), 1 << 16), NBYTES)) // 8 * 8
    data = synth.random_bytes(SEED, per_step)
    for _ in range(args.warmup):
        oracle.tdes_parallel(keys, data, "ecb_enc", threads=cores)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.tdes_parallel(keys, data, "ecb_enc", threads=cores)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms * 1e-3) / 1e9
    sample = (f"ECB encrypt of the first {per_step} bytes of the 1 GiB workload per step, "
              f"{cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GB/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "ECB encrypt", "sample_bytes": per_step},
        "cpu_baseline": {"value": round(value, 6), "unit": "GB/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
