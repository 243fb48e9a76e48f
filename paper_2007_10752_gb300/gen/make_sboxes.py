"""Search LOP3 circuits for the eight DES S-boxes and store the smallest found.

Compiles ``sbox_search.c`` and ``resub_sboxes.c`` with gcc, runs one search
process per S-box in parallel, passes each returned circuit through the
resubstitution post-pass, checks every circuit exhaustively (all 64 inputs)
against the S-box table of ``des_tables.py``, and rewrites ``sbox_lop3.json``
for any S-box where the new circuit has fewer gates than the stored one.
Every circuit it writes carries its provenance: the iteration count, seed
and extra arguments of the search and a hash of the two C sources, so that
``--reproduce`` can derive it again, gate for gate (the search is
deterministic for given arguments).  ``prune_sboxes`` marks the circuits it
shrinks, and reproduction applies the same pruning.

Run:  python -m paper_2007_10752_gb300.gen.make_sboxes [iterations] [seed] [extra args]
      python -m paper_2007_10752_gb300.gen.make_sboxes --reproduce
"""
from __future__ import annotations

import hashlib
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


def sources_hash() -> str:
    """Hash of the search and post-pass sources that a provenance refers to."""
    h = hashlib.sha256()
    for name in ("sbox_search.c", "resub_sboxes.c"):
        with open(os.path.join(HERE, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def tools():
    """Compiles the search and the post-pass; returns their paths."""
    tmp = tempfile.mkdtemp(prefix="sbox_search_")
    exe = os.path.join(tmp, "sbox_search")
    rexe = os.path.join(tmp, "resub_sboxes")
    subprocess.check_call(["gcc", "-O3", "-o", exe, os.path.join(HERE, "sbox_search.c")])
    subprocess.check_call(["gcc", "-O3", "-o", rexe, os.path.join(HERE, "resub_sboxes.c")])
    return exe, rexe


def derive(g: int, iters: str, seed: str, extra, exe: str, rexe: str, pruned: bool = False):
    """S-box g's circuit as the recorded search derives it: search, the
    resubstitution post-pass when it removes gates, and gate elimination when
    the provenance says the stored circuit was pruned."""
    tts = des_tables.sbox_truth_tables(g)
    out = subprocess.run([exe] + [f"{t:016x}" for t in tts] + [str(iters), str(seed)] +
                         [str(x) for x in extra], capture_output=True, text=True, check=True).stdout
    circ = parse(out)
    small = resub(rexe, circ)
    if verify(g, small) and len(small["gates"]) < len(circ["gates"]):
        circ = small
    if pruned:
        import prune_sboxes  # noqa: E402 (sibling module)
        circ = prune_sboxes.prune(g, circ)
    return circ


def reproduce() -> int:
    """Derives every stored circuit that has a recorded provenance again and
    compares it gate for gate; returns the number of mismatches."""
    store = load()
    exe, rexe = tools()
    bad = 0
    for g, c in enumerate(store["sboxes"]):
        prov = c.get("provenance", {})
        if not prov.get("recorded"):
            print(f"S{g + 1}: provenance not recorded ({prov.get('note', '')[:60]}...)")
            continue
        if prov.get("sources") != sources_hash():
            print(f"S{g + 1}: recorded with other search sources ({prov.get('sources')})")
            bad += 1
            continue
        d = derive(g, prov["iterations"], prov["seed"], prov["extra"], exe, rexe,
                   prov.get("pruned", False))
        same = d["gates"] == c["gates"] and d["outputs"] == c["outputs"]
        print(f"S{g + 1}: {'reproduced' if same else 'DIFFERS'} ({len(c['gates'])} gates)")
        bad += 0 if same else 1
    return bad


def main(argv):
    if argv and argv[0] == "--reproduce":
        raise SystemExit(1 if reproduce() else 0)
    iters = argv[0] if argv else "30"
    seed = argv[1] if len(argv) > 1 else "1"
    extra = argv[2:] if len(argv) > 2 else ["0", "1", "99"]
    exe, rexe = tools()
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
            circ["provenance"] = {"recorded": True, "iterations": int(iters), "seed": int(seed),
                                  "extra": [int(x) for x in extra], "sources": sources_hash(),
                                  "pruned": False}
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
