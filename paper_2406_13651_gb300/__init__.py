"""GB300-native CLAMP hot path: majorized forward-model agents inside the MACE iteration.

The compute path lives in a CUDA shared library (``csrc/``) behind a C ABI
(``include/clamp.h``); ``clamp`` is the thin Python binding over it.  Importing
this package loads nothing; ``paper_2406_13651_gb300.clamp`` loads the library
and fails loudly when it has not been built.
"""
__all__ = ["inputs", "clamp"]
