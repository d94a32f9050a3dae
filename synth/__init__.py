"""Seeded synthetic inputs (poses, weights, model presets) for Coherent Fusion scoring.

This package only makes inputs; it holds none of the method's arithmetic.
Both the CUDA path and the CPU oracle consume what it produces.
"""

from . import configs, poses, weights  # noqa: F401
