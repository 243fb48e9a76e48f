"""Build libtdes_gb300.so in-tree for sm_103a.

Steps: regenerate csrc/generated/tdes_generated.cuh from the generator
(tables + stored S-box circuits), compile the two translation units with
nvcc in parallel (-gencode arch=compute_103a,code=sm_103a -lineinfo), link a
shared library next to this file.  ptxas resource usage (registers, spills,
shared memory) is kept in _build/ptxas.txt.

Run:  python -m paper_2007_10752_gb300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libtdes_gb300.so")
TOOLS_LIB = os.path.join(HERE, "libtdes_tools.so")  # benchmark/test tools, not the cipher
SOURCES = ["tdes_api.cu", "tdes_kernels.cu", "tdes_small.cu", "tdes_noalloc.cu", "tdes_batch.cu",
           "tdes_tune.cu", "tdes_ctx.cu",
           "tdes_serve.cu", "tdes_uniform.cu"]
TOOLS_SOURCES = ["tdes_tools.cu", "tdes_paper_design.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr"]
_lock = threading.Lock()


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(CSRC, "generated", "tdes_generated.cuh"),
              os.path.join(CSRC, "generated", "tdes_generated_scalar.cuh"),
              os.path.join(CSRC, "generated", "tdes_generated_mixed.cuh"),
              os.path.join(ROOT, "include", "tdes.h")]
    gen = os.path.join(HERE, "gen")
    files += [os.path.join(gen, f) for f in ("des_tables.py", "emit_cuda.py", "sbox_lop3.json")]
    return [f for f in files if os.path.exists(f)]


def build(force: bool = False, verbose: bool = False) -> str:
    with _lock:
        sys.path.insert(0, os.path.join(HERE, "gen"))
        try:
            import emit_cuda  # noqa: WPS433 (build-time generator)
            emit_cuda.emit()
        finally:
            sys.path.pop(0)
        newest = max(os.path.getmtime(f) for f in _inputs())
        if (not force and all(os.path.exists(x) and os.path.getmtime(x) >= newest
                                  for x in (LIB, TOOLS_LIB))):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        objs, procs = [], []
        for src in SOURCES + TOOLS_SOURCES:
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
        logs = []
        for src, p in procs:
            out, _ = p.communicate()
            logs.append(f"== {src}\n{out}")
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{out}")
        with open(os.path.join(BUILD, "ptxas.txt"), "w") as f:
            f.write("\n".join(logs))
        for lib, srcs in ((LIB, SOURCES), (TOOLS_LIB, TOOLS_SOURCES)):
            tmp = lib + f".tmp{os.getpid()}"
            lib_objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in srcs]
            subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *lib_objs])
            os.replace(tmp, lib)
        if verbose:
            print("\n".join(logs))
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
