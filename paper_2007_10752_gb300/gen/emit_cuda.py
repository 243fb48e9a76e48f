"""Emit the generated CUDA headers of the bitsliced 3DES kernels.

Writes ``paper_2007_10752_gb300/csrc/generated/tdes_generated.cuh`` (the
bitsliced path) and ``tdes_generated_scalar.cuh`` (tables of the scalar
one-block-per-thread path) from ``des_tables.py`` and ``sbox_lop3.json``:

* ``tdes_round``: one Feistel round over 32 blocks held as bit-planes
  (Sec. III-B: expansion, round-key XOR, the eight S-boxes, the
  permutation, XOR into the other half).  The expansion and the permutation
  are register renames; each S-box is its LOP3 circuit; the round-key XOR is
  folded into the XOR into the other half (see "keyed planes" below).
* ``tdes_ip`` / ``tdes_fp``: the initial and final permutations as renames
  between the transposed words and the two halves.
* ``kTdesRecipe``: for every word of the per-key round-constant table, the
  one or two key bits whose XOR it holds, for encryption and decryption; the
  key-schedule kernel gathers them (PC-1, the rotations and PC-2 of
  Sec. III-A are composed here into one bit selection per round-key bit).

Keyed planes.  Each of the 32 bits of a half is stored XORed with the
round-key bit that its first use as an S-box input needs, so that input costs
nothing.  The 16 half bits that the expansion uses twice get their second
copy with one XOR of a uniform mask (done as an integer multiply-add, which
runs outside the logic pipe).  When a half is updated, the stored key bit is
swapped for the one its next use needs inside the same 3-input XOR that adds
the S-box output, so the round key costs no extra logic operation.

Run:  python -m paper_2007_10752_gb300.gen.emit_cuda   (or emit() from build)
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import des_tables as T  # noqa: E402

OUT_DIR = os.path.join(os.path.dirname(HERE), "csrc", "generated")
OUT = os.path.join(OUT_DIR, "tdes_generated.cuh")

# ---- table layout (32-bit words) ----
# A table serves `stages` DES passes (3: EDE3; 1: single DES, which EDE3
# reduces to when two adjacent keys are equal, Sec. III-B).
PRO = 0                 # 64 words: prologue XOR of L (0..31) and R (32..63), by half bit
ROUND0 = 64             # 16*stages rounds x 64 words; S-box g: 8g + [c0 c1 c2 c3 d1 d2 m1 m2]


def layout(stages=3):
    """Word offsets of the passes of a table for `stages` DES passes:
    (rekey offsets at the stage boundaries, epilogue offset, table words)."""
    nr = 16 * stages
    rekey = tuple(ROUND0 + nr * 64 + 64 * i for i in range(stages - 1))
    epi = ROUND0 + nr * 64 + 64 * (stages - 1)
    return rekey, epi, epi + 64


REKEY, EPI, TABLE_WORDS = layout(3)  # re-keying of the source half at rounds 16, 32

# secondary expansion positions: inputs b1, b2 of every S-box (their half bits
# are also inputs b5, b6 of the previous S-box, which take the stored copy)
SECONDARY = [j for j in range(48) if j % 6 in (0, 1)]
PRIMARY_POS = {}
for j in range(48):
    if j % 6 not in (0, 1):
        PRIMARY_POS[T.E[j] - 1] = j
assert sorted(PRIMARY_POS) == list(range(32))

# f-bit i receives S-output bit P[i]-1; invert to route S-outputs to half bits
P_INV = [0] * 32
for i, q in enumerate(T.P):
    P_INV[q - 1] = i


def schedule(stages=3):
    """(target, source) half of each of the 16*stages rounds (48 for EDE3).

    Rounds XOR into the target half in place.  Inside a DES stage the halves
    alternate; between stages the final swap of one stage and the first of
    the next cancel (FP then IP is the identity and the halves enter the next
    stage as R16 || L16), so the target repeats.
    """
    out = []
    for stage in range(stages):
        for k in range(16):
            even = (k % 2 == 0)
            if stage == 1:
                out.append(("R", "L") if even else ("L", "R"))
            else:
                out.append(("L", "R") if even else ("R", "L"))
    return out


def recipe(stages=3):
    """For each table word: (set of subkey-bit refs (round, position), kind).

    kind 0: word = mask of the XOR of the refs; kind 1: the same mask | 1
    (the multiplier of the multiply-add form of a masked XOR).
    """
    sched = schedule(stages)
    nr = len(sched)
    rekey, epi, nwords = layout(stages)
    kappa = {"L": [frozenset()] * 32, "R": [frozenset()] * 32}
    words = [(frozenset(), 0)] * nwords

    def need(r, i):
        return frozenset({(r, PRIMARY_POS[i])})

    def next_source(half, r):
        for r2 in range(r + 1, nr):
            if sched[r2][1] == half:
                return r2
        return None

    # prologue: key the first source half for round 0
    s0 = sched[0][1]
    for i in range(32):
        base = PRO + (0 if s0 == "L" else 32) + i
        words[base] = (kappa[s0][i] ^ need(0, i), 0)
        kappa[s0] = kappa[s0][:i] + [need(0, i)] + kappa[s0][i + 1:]
    for r, (tgt, src) in enumerate(sched):
        if r and r % 16 == 0:
            base = rekey[r // 16 - 1] + (0 if src == "L" else 32)
            kap = list(kappa[src])
            for i in range(32):
                words[base + i] = (kap[i] ^ need(r, i), 0)
                kap[i] = need(r, i)
            kappa[src] = kap
        for i in range(32):
            assert kappa[src][i] == need(r, i), (r, i)
        r2 = next_source(tgt, r)
        kt = list(kappa[tgt])
        for g in range(8):
            base = ROUND0 + 64 * r + 8 * g
            for t in range(4):
                i = P_INV[4 * g + t]
                new = need(r2, i) if r2 is not None else frozenset()
                words[base + t] = (kt[i] ^ new, 0)
                kt[i] = new
            for u in range(2):
                j = 6 * g + u
                i = T.E[j] - 1
                d = kappa[src][i] ^ frozenset({(r, j)})
                words[base + 4 + u] = (d, 0)
                words[base + 6 + u] = (d, 1)
        kappa[tgt] = kt
    for h, off in (("L", 0), ("R", 32)):
        for i in range(32):
            words[epi + off + i] = (kappa[h][i], 0)
    return words


# S-box whose six-bit round-key group sits in byte p of a scalar round-key word
# pair: rotr(R, 27) puts the expansion windows of S-boxes 1, 7, 5, 3 (0-based
# 0, 6, 4, 2) at bits 0, 8, 16, 24, and rotr(R, 23) those of S-boxes 2, 8, 6, 4.
SCALAR_GROUP_ORDER = (0, 6, 4, 2, 1, 7, 5, 3)


def subkey_source(direction, r, stages=3):
    """(key index 0..2, DES round-key index 0..15) of round r: EDE3 for three
    stages, a single DES pass under the first key for one."""
    stage, k = divmod(r, 16)
    if stages == 1:
        return (0, k) if direction == "enc" else (0, 15 - k)
    if direction == "enc":   # E_K1, D_K2, E_K3
        return [(0, k), (1, 15 - k), (2, k)][stage]
    return [(2, 15 - k), (1, k), (0, 15 - k)][stage]   # D_K3, E_K2, D_K1


def resolve(words, stages=3):
    """Refs -> key bits: entries (kind, a, b) with a, b = 64*key + (bit-1) or 255."""
    rkb = T.round_key_bits()
    out = {}
    for direction in ("enc", "dec"):
        rows = []
        for refs, kind in words:
            bits = []
            for (r, j) in sorted(refs):
                key, sub = subkey_source(direction, r, stages)
                bits.append(64 * key + rkb[sub][j] - 1)
            assert len(bits) <= 2
            bits += [255] * (2 - len(bits))
            rows.append((kind, bits[0], bits[1]))
        out[direction] = rows
    return out


def plane_index(k):
    """Transposed word holding block bit k (1..64): (word 0/1, bit position in word).

    A block is loaded as two little-endian 32-bit words of its big-endian
    bytes, so bit k sits in word (k-1)//32, byte ((k-1)//8)%4, bit 7-(k-1)%8.
    """
    w = (k - 1) // 32
    byte = ((k - 1) // 8) % 4
    return w, 8 * byte + 7 - (k - 1) % 8


def emit_sbox(lines, g, circ, targets):
    """The S-box's gates in order; each output's update (the XOR into the
    other half, with the key swap) follows right after the output's gate, so
    the output need not stay live to the end of the S-box."""
    xs = [f"x{u}" for u in range(6)]
    names = list(xs)
    comps = ["x", "y", "z", "w"]
    by_gate = {}
    for t, (gid, neg) in enumerate(circ["outputs"]):
        by_gate.setdefault(gid, []).append((t, neg))
    lines.append(f"    const uint4 kc = *reinterpret_cast<const uint4*>(k + {8 * g});")

    def updates(gid):
        for t, neg in by_gate.get(gid, []):
            i = targets[t]
            lut = 0x69 if neg else 0x96
            lines.append(f"    T[{i}] = lop3<0x{lut:02x}>(T[{i}], {names[gid]}, kc.{comps[t]});")

    for gid in range(6):
        updates(gid)
    for n, (a, b, c, lut) in enumerate(circ["gates"]):
        nm = f"s{g}_{n}"
        lines.append(f"    const uint32_t {nm} = lop3<0x{lut:02x}>({names[a]}, {names[b]}, {names[c]});")
        names.append(nm)
        updates(6 + n)
    return None


def emit(path: str = OUT) -> str:
    with open(os.path.join(HERE, "sbox_lop3.json")) as f:
        sboxes = json.load(f)["sboxes"]
    words = recipe()
    rows = resolve(words)
    words1 = recipe(1)
    rows1 = resolve(words1, 1)
    _, epi1, nwords1 = layout(1)
    L = []
    L.append("// GENERATED by paper_2007_10752_gb300/gen/emit_cuda.py -- do not edit.")
    L.append("// Bitsliced 3DES-EDE3 round, permutations and key-table recipe derived from the")
    L.append("// tables of Appendix A and the S-box circuits in gen/sbox_lop3.json.")
    L.append("#pragma once")
    L.append("#include <cstdint>")
    L.append("")
    L.append(f"#define TDES_TABLE_WORDS {TABLE_WORDS}")
    L.append(f"#define TDES_TABLE_PRO {PRO}")
    L.append(f"#define TDES_TABLE_ROUND0 {ROUND0}")
    L.append(f"#define TDES_TABLE_REKEY16 {REKEY[0]}")
    L.append(f"#define TDES_TABLE_REKEY32 {REKEY[1]}")
    L.append(f"#define TDES_TABLE_EPI {EPI}")
    gates = sum(len(c["gates"]) for c in sboxes)
    L.append(f"#define TDES_SBOX_GATES {gates}  // LOP3 per round for the eight S-boxes")
    # Which half each key-mask pass touches: the other half's words are all
    # zero by construction of the keyed-plane schedule (checked here).
    def half_defs(prefix, ws, passes):
        zero = lambda base: all(not ws[base + i][0] for i in range(32))  # noqa: E731
        for name, base in passes.items():
            l_zero, r_zero = zero(base), zero(base + 32)
            assert l_zero != r_zero, f"{name}: expected exactly one half to need key masks"
            L.append(f"#define {prefix}_{name}_HALF_R {0 if r_zero else 1}  // 1: the R half, 0: the L half")

    half_defs("TDES", words, {"PRO": PRO, "REKEY16": REKEY[0], "REKEY32": REKEY[1], "EPI": EPI})
    L.append("")
    L.append("// Single-DES tables (one pass of 16 rounds under the first key): the same")
    L.append("// rounds and prologue layout, no re-keying, its own epilogue.")
    L.append(f"#define TDES1_TABLE_WORDS {nwords1}")
    L.append(f"#define TDES1_TABLE_EPI {epi1}")
    half_defs("TDES1", words1, {"PRO": PRO, "EPI": epi1})
    L.append("")
    L.append("// Needs TDES_HD and lop3<LUT>(a, b, c) from tdes_bitslice.cuh.")
    L.append("")
    mixed_lines = []
    for mixed in (False, True):
        if mixed:  # into its own header: only the batch kernel's mixed-key tiles use it
            main_lines, L = L, mixed_lines
        if not mixed:
            L.append("// One round: T ^= f(S, round key).  S and T hold keyed planes; k points at")
            L.append("// this round's 64 constants (per S-box: 4 update masks, 2 masks of the")
            L.append("// doubled expansion inputs, 2 multipliers = mask | 1), in shared memory.")
            L.append("TDES_HD void tdes_round(uint32_t (&T)[32], const uint32_t (&S)[32],")
            L.append("                        const uint32_t* __restrict__ k) {")
        else:
            L.append("// The same round for tables whose masks differ from bit to bit (one key")
            L.append("// per bit position: tiles of small messages under many keys).  The")
            L.append("// multiply-add form of a masked XOR holds only for all-0 or all-1 masks,")
            L.append("// so the doubled expansion inputs take a plain XOR; the multipliers are")
            L.append("// not read.")
            L.append("TDES_HD void tdes_round_mixed(uint32_t (&T)[32], const uint32_t (&S)[32],")
            L.append("                              const uint32_t* __restrict__ k) {")
        for g in range(8):
            circ = sboxes[g]
            L.append(f"    {{  // S-box {g + 1}")
            L.append(f"    const uint4 kd = *reinterpret_cast<const uint4*>(k + {8 * g + 4});")
            for u in range(6):
                j = 6 * g + u
                i = T.E[j] - 1
                if u == 0 and not mixed:
                    L.append(f"    const uint32_t x0 = S[{i}] * kd.z + kd.x;  // second copy: XOR by multiply-add")
                elif u == 1 and not mixed:
                    L.append(f"    const uint32_t x1 = S[{i}] * kd.w + kd.y;")
                elif u == 0:
                    L.append(f"    const uint32_t x0 = S[{i}] ^ kd.x;  // second copy")
                elif u == 1:
                    L.append(f"    const uint32_t x1 = S[{i}] ^ kd.y;")
                else:
                    L.append(f"    const uint32_t x{u} = S[{i}];")
            emit_sbox(L, g, circ, P_INV[4 * g:4 * g + 4])
            L.append("    }")
        L.append("}")
        L.append("")
    L = main_lines
    L.append("// Initial permutation: transposed words A0/A1 (bit position -> plane) to halves.")
    L.append("TDES_HD void tdes_ip(const uint32_t (&A0)[32], const uint32_t (&A1)[32],")
    L.append("                     uint32_t (&Lh)[32], uint32_t (&Rh)[32]) {")
    for j in range(64):
        w, c = plane_index(T.IP[j])
        dst = f"Lh[{j}]" if j < 32 else f"Rh[{j - 32}]"
        L.append(f"    {dst} = A{w}[{c}];")
    L.append("}")
    L.append("")
    L.append("// Final permutation of R16 || L16 back to transposed words A0/A1.")
    L.append("TDES_HD void tdes_fp(const uint32_t (&Lh)[32], const uint32_t (&Rh)[32],")
    L.append("                     uint32_t (&A0)[32], uint32_t (&A1)[32]) {")
    for k in range(1, 65):
        src = T.FP[k - 1]  # preoutput bit: 1..32 from R16, 33..64 from L16
        s = f"Rh[{src - 1}]" if src <= 32 else f"Lh[{src - 33}]"
        w, c = plane_index(k)
        L.append(f"    A{w}[{c}] = {s};")
    L.append("}")
    L.append("")
    L.append("// Key-table recipe: per word {kind, bit a, bit b}; bit = 64*key + (key bit - 1),")
    L.append("// 255 = none.  Word = -(bit a ^ bit b), OR 1 when kind is 1.  [0] encrypt, [1] decrypt.")
    for name, rws, nw in (("TDES_RECIPE_INIT", rows, TABLE_WORDS),
                          ("TDES1_RECIPE_INIT", rows1, nwords1)):
        L.append(f"#define {name} {{ \\")
        for direction in ("enc", "dec"):
            L.append("  { \\")
            rr = rws[direction]
            for s0 in range(0, nw, 8):
                chunk = ", ".join("{%d,%d,%d}" % r for r in rr[s0:s0 + 8])
                L.append(f"    {chunk}, \\")
            L.append("  }, \\")
        L.append("}")
    text = "\n".join(L) + "\n"
    _write(path, text)
    hdr = ["// GENERATED by paper_2007_10752_gb300/gen/emit_cuda.py -- do not edit.",
           "// Round of the bitsliced path for tables with a different key per bit",
           "// position (from the S-box circuits in gen/sbox_lop3.json).",
           "#pragma once",
           "#include <cstdint>",
           "",
           "// Needs TDES_HD and lop3<LUT>(a, b, c) from tdes_bitslice.cuh.",
           ""]
    _write(os.path.join(os.path.dirname(path), "tdes_generated_mixed.cuh"),
           "\n".join(hdr + mixed_lines) + "\n")
    L = []
    L.append("// GENERATED by paper_2007_10752_gb300/gen/emit_cuda.py -- do not edit.")
    L.append("// Tables of the scalar (one block per thread) 3DES path, from Appendix A.")
    L.append("#pragma once")
    L.append("#include <cstdint>")
    L.append("")
    L.append("// Scalar path.  Per EDE3 round r: 8 six-bit round-key groups, byte p holding")
    L.append("// the group of S-box SCALAR_GROUP_ORDER[p] (so the 8 bytes read as two")
    L.append("// little-endian words line up with the expansion windows of rotr(R, 27) and")
    L.append("// rotr(R, 23)); entry [dir][r][6p + u] = key bit of bit u of byte p:")
    L.append("// 64*key + (key bit - 1), [0] encrypt, [1] decrypt.")
    L.append("#define TDES_SCALAR_GROUP_ORDER {" + ",".join(map(str, SCALAR_GROUP_ORDER)) + "}")
    L.append("#define TDES_SUBKEY_INIT { \\")
    rkb = T.round_key_bits()
    for direction in ("enc", "dec"):
        L.append("  { \\")
        for r in range(48):
            key, sub = subkey_source(direction, r)
            bits = []
            for pos in range(8):
                g = SCALAR_GROUP_ORDER[pos]
                bits += [64 * key + rkb[sub][6 * g + u] - 1 for u in range(6)]
            L.append("    {" + ",".join(map(str, bits)) + "}, \\")
        L.append("  }, \\")
    L.append("}")
    L.append("")
    L.append("// S-box g combined with the permutation: the f-output word (half bit i at")
    L.append("// position 32-i) of 6-bit input x (b1 most significant).")
    L.append("#define TDES_SP_INIT { \\")
    for g in range(8):
        vals = []
        for x in range(64):
            b1, b6 = (x >> 5) & 1, x & 1
            v = T.SBOX[g][2 * b1 + b6][(x >> 1) & 0xF]
            w = 0
            for i in range(1, 33):
                q = T.P[i - 1]
                if 4 * g + 1 <= q <= 4 * g + 4 and (v >> (3 - (q - 4 * g - 1))) & 1:
                    w |= 1 << (32 - i)
            vals.append(f"0x{w:08x}u")
        L.append("  {" + ",".join(vals) + "}, \\")
    L.append("}")
    L.append("")
    L.append("// Warp-cooperative round (one chain per warp): lane l computes half bit")
    L.append("// i = 32 - l of the round function, S-box output bit P[i].  Per lane:")
    L.append("// {mask of that output bit over the 64 S-box inputs (low, high word),")
    L.append("//  right-rotation of R that puts the S-box's expansion window at bits 5..0,")
    L.append("//  byte of the round-key word pair holding the S-box's key group}.")
    L.append("#define TDES_LANE_SBOX_INIT { \\")
    for lane in range(32):
        i = 32 - lane
        q = T.P[i - 1] - 1
        g, t = q // 4, q % 4
        mask = 0
        for x in range(64):
            b1, b6 = (x >> 5) & 1, x & 1
            v = T.SBOX[g][2 * b1 + b6][(x >> 1) & 0xF]
            if (v >> (3 - t)) & 1:
                mask |= 1 << x
        rot = (27 - 4 * g) % 32
        pos = SCALAR_GROUP_ORDER.index(g)
        L.append(f"  {{0x{mask & 0xFFFFFFFF:08x}u, 0x{mask >> 32:08x}u, {rot}u, {pos}u}}, \\")
    L.append("}")
    L.append("// Per lane l: 0-based source bit of output bits 32 - l and 64 - l of IP and FP.")
    for name, perm in (("IP", T.IP), ("FP", T.FP)):
        L.append(f"#define TDES_LANE_{name}_INIT {{ \\")
        L.append("  " + ", ".join("{%du, %du}" % (perm[32 - l - 1] - 1, perm[64 - l - 1] - 1)
                               for l in range(32)) + " \\")
        L.append("}")
    L.append("")
    L.append("// Initial / final permutation by nibbles: entry [n][v] is the output word")
    L.append("// contribution of value v in input nibble n (input bits 4n+1..4n+4).")
    for name, perm in (("IPN", T.IP), ("FPN", T.FP)):
        dest = {src: j for j, src in enumerate(perm, start=1)}  # input bit -> output bit
        L.append(f"#define TDES_{name}_INIT {{ \\")
        for n in range(16):
            vals = []
            for v in range(16):
                w = 0
                for t in range(4):
                    if (v >> (3 - t)) & 1:
                        w |= 1 << (64 - dest[4 * n + t + 1])
                vals.append(f"0x{w:016x}ull")
            L.append("  {" + ",".join(vals) + "}, \\")
        L.append("}")
    L.append("")
    L.append("// Initial and final permutation as 0-based source bit (bit 1 = index 0).")
    L.append("#define TDES_IP_INIT {" + ",".join(str(x - 1) for x in T.IP) + "}")
    L.append("#define TDES_FP_INIT {" + ",".join(str(x - 1) for x in T.FP) + "}")
    text = "\n".join(L) + "\n"
    _write(os.path.join(os.path.dirname(path), "tdes_generated_scalar.cuh"), text)
    return path


def _write(path, text):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)


if __name__ == "__main__":
    print(emit())
