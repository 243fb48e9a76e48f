"""The CUDA path's generated code, checked on the CPU against the oracle.

* Every stored S-box circuit, evaluated over all 64 inputs, equals the
  oracle's table-driven S-box (two independent transcriptions of the
  appendix tables meet here).
* The generated header is up to date with the generator.
* The generated bitsliced code itself (rounds, keyed planes, key-table
  recipe, transposes, IP/FP renames) and the scalar path, compiled for the
  host from the kernels' own headers, reproduce the oracle bit for bit.
"""
import json
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2007_10752_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_2007_10752_gb300", "gen")
sys.path.insert(0, GEN)
import emit_cuda  # noqa: E402
import make_sboxes  # noqa: E402


def test_sbox_circuits_match_oracle_exhaustively():
    store = json.load(open(os.path.join(GEN, "sbox_lop3.json")))
    m = (1 << 64) - 1
    for g, circ in enumerate(store["sboxes"]):
        tts = make_sboxes.circuit_tables(circ)
        for t, (gid, neg) in enumerate(circ["outputs"]):
            v = tts[gid] ^ (m if neg else 0)
            for x in range(64):
                want = (oracle.sbox(g, x) >> (3 - t)) & 1
                assert (v >> x) & 1 == want, (g, t, x)


def test_generated_headers_are_current(tmp_path):
    emit_cuda.emit(str(tmp_path / "tdes_generated.cuh"))
    gen_dir = os.path.join(ROOT, "paper_2007_10752_gb300", "csrc", "generated")
    for name in ("tdes_generated.cuh", "tdes_generated_scalar.cuh"):
        assert open(tmp_path / name).read() == open(os.path.join(gen_dir, name)).read(), name


def test_round_schedule_and_recipe_shape():
    sched = emit_cuda.schedule()
    assert len(sched) == 48
    for r in range(47):
        tgt, src = sched[r]
        # target and source always differ; stage boundaries repeat the target
        assert tgt != src
        if r in (15, 31):
            assert sched[r + 1][0] == tgt
        else:
            assert sched[r + 1][0] == src
    words = emit_cuda.recipe()
    assert len(words) == emit_cuda.TABLE_WORDS
    assert all(len(refs) <= 2 for refs, _ in words)
    # the single-DES schedule is EDE3's first pass; its table has no re-keying
    assert emit_cuda.schedule(1) == sched[:16]
    rekey, epi, nwords = emit_cuda.layout(1)
    assert rekey == () and epi == emit_cuda.ROUND0 + 16 * 64 and nwords == epi + 64
    words1 = emit_cuda.recipe(1)
    assert len(words1) == nwords
    # rounds 0..14 need the same key bits as in EDE3; the last round's
    # updates key for nothing further, and single DES reads only one key
    assert words1[:emit_cuda.ROUND0 + 15 * 64] == words[:emit_cuda.ROUND0 + 15 * 64]
    rows1 = emit_cuda.resolve(words1, 1)
    for d in ("enc", "dec"):
        assert all(b == 255 or b < 64 for _, a, b in rows1[d] for b in (a, b))


@pytest.fixture(scope="module")
def host_check(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("hc") / "tdes_host_check")
    subprocess.check_call([nvcc, "-O1", "-std=c++17", "-o", exe,
                           os.path.join(ROOT, "tests", "host_check", "tdes_host_check.cu")])
    return exe


def _run(exe, mode, keys, data):
    r = subprocess.run([exe, mode, bytes(keys).hex()], input=data.tobytes(), capture_output=True,
                       timeout=120)
    assert r.returncode == 0
    return np.frombuffer(r.stdout, dtype=np.uint8)


KEYSETS = [
    ("seeded", lambda: synth.key_triple(77)),
    ("k1=k2=k3", lambda: synth.key_triple(78)[:8] * 3),
    ("weak", lambda: b"\x01" * 8 + b"\xfe" * 8 + synth.key_triple(79)[:8]),
    ("all-zero", lambda: b"\x00" * 24),
]


@pytest.mark.parametrize("name,mk", KEYSETS, ids=[k[0] for k in KEYSETS])
@pytest.mark.parametrize("mode", ["bs_enc", "bs_dec", "b1_enc", "b1_dec", "sc_enc", "sc_dec",
                                  "sn_enc", "sn_dec", "s1_enc", "s1_dec"])
def test_generated_code_matches_oracle(host_check, name, mk, mode):
    keys = mk()
    data = synth.random_bytes(len(name) * 31 + 5, 8 * 75)  # 2 full groups of 32 + a ragged one
    got = _run(host_check, mode, keys, data)
    if mode[1] == "1":  # one DES pass under K1
        want = oracle.des_ecb(keys[:8], data, decrypt=mode.endswith("dec"))
    else:
        want = oracle.tdes_ecb(keys, data, decrypt=mode.endswith("dec"))
    assert (got == want).all()
