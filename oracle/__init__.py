"""CPU oracle for 3DES-EDE3 -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C transcription of the method of
"Bit-level Parallelization of 3DES Encryption on GPU", Sec. III (key
generation, DES rounds, the 3DES EDE equations), one byte per bit, with the
appendix tables as printed.  CTR and CBC wrap it by their usual definitions
(the paper itself only runs ECB, Sec. V).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does.
"""
from .oracle import (  # noqa: F401
    HEADER,
    SOURCE,
    Oracle,
    build,
    compile_oracle,
    default,
    des_block,
    des_cbc_decrypt,
    des_cbc_encrypt,
    des_ctr,
    des_ecb,
    des_round_keys,
    sbox,
    tdes_block,
    tdes_cbc_decrypt,
    tdes_cbc_encrypt,
    tdes_ctr,
    tdes_ecb,
    tdes_messages,
    tdes_parallel,
)
