"""CPU oracle of the FHEON rotation path: plain C RNS-CKKS plus FHEON's layer packing.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in
this package.  It shares no code with the CUDA library, and the CUDA library
never calls it.
"""
from ._lib import build  # noqa: F401
from . import ckks  # noqa: F401
