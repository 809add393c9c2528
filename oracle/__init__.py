"""CKKS oracle (test infrastructure only).

Plain, slow CPU statement of the CryptoTL server-side evaluation (Sec. 3.1 of the
paper): schoolbook negacyclic products, big-integer CRT, O(N^2) slot encoding.  Only
tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library in ``paper_2205_11935_gb300``.
"""
from .ckks_oracle import Oracle, build_oracle  # noqa: F401
