"""Packing poses by atom count (host logic)."""

import numpy as np

from paper_2104_04547_gb300.batching import pack_by_atoms


def test_pack_by_atoms_covers_all_and_respects_limits():
    rng = np.random.default_rng(0)
    sizes = rng.integers(150, 1090, size=500)
    batches = pack_by_atoms(sizes, 64, 64 * 700)
    flat = sorted(i for b in batches for i in b)
    assert flat == list(range(500))
    for b in batches:
        assert len(b) <= 64
        assert sum(int(sizes[i]) for i in b) <= 64 * 700 or len(b) == 1
    # sorted by size: batch maxima are non-decreasing
    mx = [max(int(sizes[i]) for i in b) for b in batches]
    assert mx == sorted(mx)


def test_oversized_pose_gets_its_own_batch():
    batches = pack_by_atoms([10, 5000, 20], 8, 100)
    assert [sorted(b) for b in batches] == [[0, 2], [1]]
