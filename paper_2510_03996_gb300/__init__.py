"""GB300-native RNS-CKKS rotation path of FHEON (arxiv 2510.03996).

The compute path is the CUDA library ``libfheon`` (csrc/, sm_103a) behind the
C ABI of include/fheon.h; ``paper_2510_03996_gb300.fheon`` is its thin ctypes
binding and fails loudly when the library is missing.
"""
