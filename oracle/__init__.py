"""FP64 CPU oracle for Coherent Fusion scoring (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package; the product path never does.
"""

from . import fusion_oracle  # noqa: F401
