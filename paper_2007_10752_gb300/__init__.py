"""GB300-native (sm_103a) 3DES-EDE3: bitsliced CUDA kernels behind a small C ABI.

``paper_2007_10752_gb300.tdes`` is the thin ctypes binding of the C ABI
declared in ``include/tdes.h`` (it loads ``libtdes_gb300.so``, built by
``paper_2007_10752_gb300.build``).  ``paper_2007_10752_gb300.synth`` draws
the seeded synthetic inputs.  Importing the package itself loads nothing.
"""
__all__ = ["tdes", "synth", "build"]
