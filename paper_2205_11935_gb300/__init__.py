"""GB300-native CKKS server path of CryptoTL (arXiv 2205.11935).

The compute lives in the CUDA library ``_build/libctl.so`` behind the C-ABI of
``include/ctl.h``; ``ctl`` is its ctypes binding.
"""
from . import ctl  # noqa: F401
from .ctl import Context, Keys, Ciphertext, Model, CtlError, plan_primes, lib  # noqa: F401
