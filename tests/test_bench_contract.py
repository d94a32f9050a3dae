"""bench.py's stored conv traffic (CPU).

The DRAM bytes per conv launch that bench.py reports as `roofline.traffic` come from an ncu capture and
are valid only for the kernel source they were taken on.  These tests fail when the conv kernel's code
changes without a new capture (the stored source hash no longer matches), and check that the stored
figures are plausible: one per conv layer of the benchmarked model, each at or below the layer's
algorithmic bytes (input + output + weights: a larger figure would mean re-reads from DRAM).
"""

import pytest

import bench
from synth import configs


def test_traffic_was_taken_on_the_current_conv_source():
    assert bench.conv_source_hash() == bench.CONV_TRAFFIC["src"], \
        "conv kernel changed since the ncu traffic capture: re-capture and update CONV_TRAFFIC"


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_traffic_at_or_below_algorithmic_bytes(dtype):
    desc = configs.model(bench.MODEL)
    per_layer = bench.CONV_TRAFFIC[dtype]
    assert len(per_layer) == len(desc["conv"])
    mean = bench.conv_traffic(dtype, bench.CONV_TRAFFIC["poses"])
    assert mean == pytest.approx(sum(per_layer) / len(per_layer))
    assert mean <= bench.conv_algorithmic_bytes(desc, dtype, bench.CONV_TRAFFIC["poses"])
    assert bench.conv_traffic(dtype, bench.CONV_TRAFFIC["poses"] + 1) is None   # other batch sizes: no figure
