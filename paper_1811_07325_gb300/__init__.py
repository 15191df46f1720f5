"""GB300-native Strassen multiplication (Stark, arXiv 1811.07325).

The compute path is ``libstark.so`` (CUDA for sm_103a behind a C ABI, see
``include/stark.h``); :mod:`paper_1811_07325_gb300.stark` is its thin ctypes
binding.  Importing this package loads nothing: the library is opened on
first use and an import of the binding fails loudly if it has not been built.
"""
__all__ = ["stark", "synth"]
