"""Search LOP3 circuits for the eight DES S-boxes and store the smallest found.

Compiles ``sbox_search.c`` and ``resub_sboxes.c`` with gcc, runs one search
process per S-box in parallel, passes each returned circuit through the
resubstitution post-pass, checks every circuit exhaustively (all 64 inputs)
against the S-box table of ``des_tables.py``, and rewrites ``sbox_lop3.json``
for any S-box where the new circuit has fewer gates than the stored one.

Run:  python -m paper_2007_10752_gb300.gen.make_sboxes [iterations] [seed] [extra args]
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import des_tables  # noqa: E402

JSON_PATH = os.path.join(HERE, "sbox_lop3.json")


def eval_lut(lut: int, a: int, b: int, c: int) -> int:
    m = (1 << 64) - 1
    r = 0
    for i in range(8):
        if (lut >> i) & 1:
            r |= (a if i & 4 else ~a & m) & (b if i & 2 else ~b & m) & (c if i & 1 else ~c & m)
    return r


def input_tables():
    out = []
    for v in range(6):
        t = 0
        for x in range(64):
            if (x >> (5 - v)) & 1:
                t |= 1 << x
        out.append(t)
    return out


def circuit_tables(circ):
    """Truth tables of every signal of a circuit (inputs first)."""
    tts = input_tables()
    for a, b, c, lut in circ["gates"]:
        tts.append(eval_lut(lut, tts[a], tts[b], tts[c]))
    return tts


def verify(g: int, circ) -> bool:
    target = des_tables.sbox_truth_tables(g)
    tts = circuit_tables(circ)
    m = (1 << 64) - 1
    for t, (gid, neg) in enumerate(circ["outputs"]):
        v = tts[gid] ^ (m if neg else 0)
        if v != target[t]:
            return False
    return True


def parse(text: str):
    gates, outs = [], [None] * 4
    for line in text.splitlines():
        f = line.split()
        if not f:
            continue
        if f[0] == "g":
            gid, a, b, c, lut = map(int, f[1:])
            assert gid == 6 + len(gates)
            gates.append([a, b, c, lut])
        elif f[0] == "out":
            t, gid, neg = map(int, f[1:])
            outs[t] = [gid, neg]
    return {"gates": gates, "outputs": outs}


def to_text(circ) -> str:
    """A circuit in the text format of sbox_search.c (input of resub_sboxes.c)."""
    lines = [f"g {6 + i} {a} {b} {c} {lut}" for i, (a, b, c, lut) in enumerate(circ["gates"])]
    lines += [f"out {t} {gid} {neg}" for t, (gid, neg) in enumerate(circ["outputs"])]
    return "\n".join(lines) + "\n"


def resub(exe: str, circ):
    """The circuit after the resubstitution post-pass (or unchanged if it fails)."""
    r = subprocess.run([exe], input=to_text(circ), capture_output=True, text=True)
    return parse(r.stdout) if r.returncode == 0 else circ


def load():
    if os.path.exists(JSON_PATH):
        with open(JSON_PATH) as f:
            return json.load(f)
    return {"sboxes": [None] * 8}


def main(argv):
    iters = argv[0] if argv else "30"
    seed = argv[1] if len(argv) > 1 else "1"
    extra = argv[2:] if len(argv) > 2 else ["0", "1", "99"]
    tmp = tempfile.mkdtemp(prefix="sbox_search_")
    exe = os.path.join(tmp, "sbox_search")
    rexe = os.path.join(tmp, "resub_sboxes")
    subprocess.check_call(["gcc", "-O3", "-o", exe, os.path.join(HERE, "sbox_search.c")])
    subprocess.check_call(["gcc", "-O3", "-o", rexe, os.path.join(HERE, "resub_sboxes.c")])
    procs = []
    for g in range(8):
        tts = des_tables.sbox_truth_tables(g)
        procs.append(subprocess.Popen([exe] + [f"{t:016x}" for t in tts] + [iters, seed] + extra,
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True))
    store = load()
    changed = False
    for g, p in enumerate(procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            print(f"S{g + 1}: search failed")
            continue
        circ = parse(out)
        if not verify(g, circ):
            raise SystemExit(f"S{g + 1}: search returned a wrong circuit")
        small = resub(rexe, circ)
        if verify(g, small) and len(small["gates"]) < len(circ["gates"]):
            circ = small
        old = store["sboxes"][g]
        n_new, n_old = len(circ["gates"]), (len(old["gates"]) if old else None)
        print(f"S{g + 1}: {n_new} gates (stored: {n_old})")
        if old is None or n_new < n_old:
            store["sboxes"][g] = circ
            changed = True
    if changed:
        store["total_gates"] = sum(len(s["gates"]) for s in store["sboxes"] if s)
        with open(JSON_PATH, "w") as f:
            json.dump(store, f, indent=None, separators=(",", ":"))
            f.write("\n")
        print(f"wrote {JSON_PATH}: {store['total_gates']} gates in total")


if __name__ == "__main__":
    main(sys.argv[1:])
