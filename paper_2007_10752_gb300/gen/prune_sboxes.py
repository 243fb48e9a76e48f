"""Shrink stored S-box circuits by gate elimination.

For each gate g: if every gate that reads g can be rewritten as one LUT over
three other signals created before it (so the circuit stays acyclic) with
its truth table unchanged, and g is not an output, then g is deleted.  The
pass repeats until no gate can be removed.  Every rewritten circuit is
checked exhaustively before ``sbox_lop3.json`` is updated.

Run:  python -m paper_2007_10752_gb300.gen.prune_sboxes [path.json ...]
"""
from __future__ import annotations

import itertools
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import make_sboxes as M  # noqa: E402

MASK = (1 << 64) - 1


def fit3(a, b, c, t):
    lut = 0
    for i in range(8):
        cls = (a if i & 4 else ~a & MASK) & (b if i & 2 else ~b & MASK) & (c if i & 1 else ~c & MASK)
        on = cls & t
        if on:
            if on != cls:
                return None
            lut |= 1 << i
    return lut


def try_remove(circ, gidx):
    """Circuit without gate gidx (signal id 6 + gidx), or None."""
    gates = circ["gates"]
    sig = 6 + gidx
    if any(gid == sig for gid, _ in circ["outputs"]):
        return None
    tts = M.circuit_tables(circ)
    new_gates = [list(g) for g in gates]
    for ci, (a, b, c, lut) in enumerate(gates):
        if sig not in (a, b, c):
            continue
        cons = 6 + ci
        cands = [s for s in range(cons) if s != sig]
        found = None
        for x, y, z in itertools.combinations(cands, 3):
            l = fit3(tts[x], tts[y], tts[z], tts[cons])
            if l is not None:
                found = [x, y, z, l]
                break
        if found is None:
            return None
        new_gates[ci] = found
    # drop the gate and renumber signals above it
    def rn(s):
        return s - 1 if s > sig else s
    out = {"gates": [], "outputs": []}
    for i, (a, b, c, l) in enumerate(new_gates):
        if i == gidx:
            continue
        out["gates"].append([rn(a), rn(b), rn(c), l])
    out["outputs"] = [[rn(gid), neg] for gid, neg in circ["outputs"]]
    return out


def prune(g, circ):
    changed = True
    while changed:
        changed = False
        for gi in range(len(circ["gates"]) - 1, -1, -1):
            cand = try_remove(circ, gi)
            if cand is not None and M.verify(g, cand):
                circ = cand
                changed = True
                break
    return circ


def main(paths):
    store = M.load()
    changed = False
    sources = paths or [None]
    for g in range(8):
        best = store["sboxes"][g]
        for p in sources:
            c = best if p is None else json.load(open(p.format(g=g)))
            if not M.verify(g, c):
                continue
            prov = dict(c.get("provenance", {"recorded": False}))
            c = prune(g, c)
            if len(c["gates"]) < len(best["gates"]):
                print(f"S{g + 1}: {len(best['gates'])} -> {len(c['gates'])}")
                prov["pruned"] = True
                c["provenance"] = prov
                best = c
                changed = True
        store["sboxes"][g] = best
    if changed:
        store["total_gates"] = sum(len(s["gates"]) for s in store["sboxes"])
        with open(M.JSON_PATH, "w") as f:
            json.dump(store, f, indent=None, separators=(",", ":"))
            f.write("\n")
        print("total", store["total_gates"])
    else:
        print("no gate removed")


if __name__ == "__main__":
    main(sys.argv[1:])
