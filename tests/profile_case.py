"""A small, self-contained launch sequence for profiler captures (test and
measurement infrastructure, not part of the library).

Runs `--launches` back-to-back launches of one kernel of the library on a
seeded buffer of `--mib` MiB (default 256 MiB: larger than the 129 MB L2, a
few hundred MB on the device) and exits.  Used as the target of ncu
captures, whose commands are recorded beside their summaries in profiles/.

  python tests/profile_case.py --kernel ecb --mib 256 --launches 3
  python tests/profile_case.py --kernel batch --launches 3
  python tests/profile_case.py --kernel batch_ctr --mib 256   (one CTR message as a batch)
  python tests/profile_case.py --kernel ecb --des   (single-DES schedule)
  python tests/profile_case.py --kernel uniform --msgs 268435456 --keys 65536
      (tdes_uniform_crypt: 64-byte messages in place, the second half of the
       large streaming workload; every kernel of the call, --launches calls)
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))  # the repository
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=["ecb", "ecb_dec", "ctr", "cbc_dec", "cbc_enc", "batch",
                                         "batch_ctr", "batch_cbc_enc", "uniform"],
                    default="ecb")
    ap.add_argument("--mib", type=int, default=256)
    ap.add_argument("--kib", type=int, default=0, help="size in KiB (overrides --mib)")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--des", action="store_true", help="a single-DES schedule (one pass)")
    ap.add_argument("--msgs", type=int, default=1 << 24, help="uniform: 64-byte messages")
    ap.add_argument("--keys", type=int, default=4096, help="uniform: key triples (a power of two)")
    args = ap.parse_args()

    import torch

    from paper_2007_10752_gb300 import build, synth, tdes
    build.build()
    torch.cuda.set_device(0)
    if args.kernel == "batch":
        # the parallel-mode messages of the 4096-message batched workload
        import numpy as np

        from paper_2007_10752_gb300.workloads import build_batched
        src, dst, kt, d, lens, modes = build_batched(torch, tdes)
        b = tdes.Batch(kt, d[d["mode"] != 4])
        for _ in range(args.launches):
            b.launch()
        torch.cuda.synchronize()
        print(f"batch: {args.launches} launches of {int(np.sum(d['mode'] != 4))} messages done")
        return
    if args.kernel == "uniform":
        from paper_2007_10752_gb300 import workloads as W
        seed, n_msg = W.STREAM_SEED, args.msgs
        buf = torch.empty(n_msg * 64, dtype=torch.uint8, device="cuda")
        synth.fill_device(buf, seed, start_byte=W.STREAM_BYTES)
        kt = tdes.KeyTable(synth.key_triples(seed, args.keys))
        k, md, v = W.uniform_arrays_device(torch, seed, n_msg, args.keys)
        scratch = torch.empty(tdes.tdes_uniform_scratch_bytes(kt, n_msg, 64), dtype=torch.uint8,
                              device="cuda")
        for _ in range(args.launches):
            tdes.tdes_uniform_crypt(kt, k, md, v, buf, buf, 64, scratch=scratch)
        torch.cuda.synchronize()
        print(f"uniform: {args.launches} calls on {n_msg} messages done:",
              tdes.tdes_uniform_info(scratch))
        return
    n = (args.kib << 10) if args.kib else (args.mib << 20)
    keys = synth.key_triple(2)
    if args.kernel == "batch_cbc_enc":
        # one CBC-encryption chain as a batch (walked by one warp)
        import numpy as np
        x = torch.from_numpy(synth.random_bytes(2, n)).cuda()
        y = torch.empty_like(x)
        kt = tdes.KeyTable(np.frombuffer(keys, dtype=np.uint8).reshape(1, 24))
        b = tdes.Batch(kt, [(tdes.MODE_CBC_ENCRYPT, 0, 5, x.data_ptr(), y.data_ptr(), n)])
        for _ in range(args.launches):
            b.launch()
        torch.cuda.synchronize()
        print(f"batch_cbc_enc: {args.launches} launches on {n >> 10} KiB done")
        return
    if args.kernel == "batch_ctr":
        # the single-key CTR stream of the large streaming workload, at this size
        import numpy as np
        x = torch.from_numpy(synth.random_bytes(2, n)).cuda()
        kt = tdes.KeyTable(np.frombuffer(keys, dtype=np.uint8).reshape(1, 24))
        b = tdes.Batch(kt, [(tdes.MODE_CTR, 0, 1 << 32, x.data_ptr(), x.data_ptr(), n)])
        for _ in range(args.launches):
            b.launch()
        torch.cuda.synchronize()
        print(f"batch_ctr: {args.launches} launches on {n >> 20} MiB done")
        return
    x = torch.from_numpy(synth.random_bytes(2, n)).cuda()
    y = torch.empty_like(x)
    ks = tdes.KeySchedule.des(keys[:8]) if args.des else tdes.KeySchedule.from_triple(keys)
    for _ in range(args.launches):
        if args.kernel == "ecb":
            tdes.tdes_ecb_encrypt(ks, x, y)
        elif args.kernel == "ecb_dec":
            tdes.tdes_ecb_decrypt(ks, x, y)
        elif args.kernel == "ctr":
            tdes.tdes_ctr_crypt(ks, 1, 0, x, y)
        elif args.kernel == "cbc_enc":
            tdes.tdes_cbc_encrypt(ks, 1, x, y)
        else:
            tdes.tdes_cbc_decrypt(ks, 1, x, y)
    torch.cuda.synchronize()
    print(f"{args.kernel}: {args.launches} launches on {args.mib} MiB done")


if __name__ == "__main__":
    main()
