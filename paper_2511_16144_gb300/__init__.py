"""GB300-native language-feature Gaussian splatting (LEGO-SLAM mapping hot path).

The compute lives in ``liblgs.so`` (hand-written CUDA for sm_103a behind the
C ABI declared in ``include/lgs.h``); ``lgs`` is its thin ctypes binding.
Importing this package loads nothing: the library is opened on first use and
a missing library raises instead of falling back to anything else.
"""
__all__ = ["synth", "lgs"]
