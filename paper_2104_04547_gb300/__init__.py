"""GB300-native Coherent Fusion pose scoring.

The scoring path is the CUDA library behind ``include/fusion.h``; ``fusion``
is its ctypes binding and ``build`` compiles it for sm_103a.
"""

__all__ = ["build", "fusion"]
