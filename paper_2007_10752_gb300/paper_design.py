"""ctypes front end of the paper's own kernel design (libtdes_tools.so),
rebuilt on GB300 as a benchmark context point; not part of the cipher API."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.path.join(HERE, "libtdes_tools.so"))
        lib.tdes_tools_paper_ecb.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_float)]
        _lib = lib
    return _lib


def paper_ecb(keys24: bytes, x, out, decrypt: bool = False) -> float:
    """ECB 3DES of CUDA tensor x into out with the paper's design; returns the
    milliseconds of its three encryption launches (synchronous)."""
    import torch
    n = x.numel()
    work = torch.empty(16 * n + 8192, dtype=torch.uint8, device=x.device)
    ms = ctypes.c_float()
    rc = _load().tdes_tools_paper_ecb(bytes(keys24), int(decrypt), x.data_ptr(), out.data_ptr(),
                                      n, work.data_ptr(), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"paper-design kernels failed: CUDA error {rc}")
    return ms.value
