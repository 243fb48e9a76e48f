"""Write tests/golden/tdes_vectors.txt from the CPU oracle (and nothing else).

Every input comes from the seeded generator; every expected value from
``oracle/``.  The vectors are cross-checked against an independent 3DES
implementation by tests/test_oracle_pins.py, and the GPU tests compare the
CUDA library against them.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2007_10752_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "tdes_vectors.txt")

# (mode, seed, nblocks, ctr0)
CASES = [
    ("ecb_enc", 11, 1, 0), ("ecb_enc", 12, 3, 0), ("ecb_enc", 13, 33, 0),
    ("ecb_dec", 21, 1, 0), ("ecb_dec", 22, 5, 0), ("ecb_dec", 23, 33, 0),
    ("ctr", 31, 1, 0), ("ctr", 32, 7, 0), ("ctr", 33, 33, 0xFFFFFFDF),
    ("cbc_enc", 41, 1, 0), ("cbc_enc", 42, 9, 0), ("cbc_enc", 43, 33, 0),
    ("cbc_dec", 51, 1, 0), ("cbc_dec", 52, 9, 0), ("cbc_dec", 53, 33, 0),
]


def main():
    lines = [
        "# 3DES-EDE3 vectors written by tests/golden/make_golden.py from the CPU oracle.",
        "# Inputs: paper_2007_10752_gb300.synth (SplitMix64) with the seed in column 2.",
        "# mode seed keys(K1||K2||K3 hex) iv_or_nonce(hex) ctr0 input(hex) output(hex)",
    ]
    for mode, seed, nblocks, ctr0 in CASES:
        keys = synth.key_triple(seed)
        data = synth.random_bytes(seed, 8 * nblocks)
        if mode == "ctr":
            ivn = synth.nonce32(seed)
            out = oracle.tdes_ctr(keys, ivn, ctr0, data)
        elif mode.startswith("cbc"):
            ivn = synth.iv64(seed)
            f = oracle.tdes_cbc_encrypt if mode == "cbc_enc" else oracle.tdes_cbc_decrypt
            out = f(keys, ivn, data)
        else:
            ivn = 0
            out = oracle.tdes_ecb(keys, data, decrypt=(mode == "ecb_dec"))
        lines.append(f"{mode} {seed} {keys.hex()} {ivn:x} {ctr0} {data.tobytes().hex()} "
                     f"{out.tobytes().hex()}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: {len(CASES)} vectors")


if __name__ == "__main__":
    main()
