"""GB300-native server answer path of constant-weight PIR (arXiv 2202.07569).

The compute path lives in the CUDA library built from ``csrc/`` and is
reached through its C ABI (``include/cwpir.h``); ``binding`` marshals
arguments to it.  Importing this package loads nothing: the library is
loaded on first use and a missing library is an error, never a fallback.
"""
__all__ = ["binding", "synthetic"]
