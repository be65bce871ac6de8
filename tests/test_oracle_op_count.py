"""The FP64 oracle's operation count per track-layer, measured by compiling
its own source with a counting scalar type: the reference figure beside the
fit's structured numerator (768 flops per track-layer, counted on the
Cartesian formulation with the Jacobian's structural zeros)."""
import shutil

import pytest

from paper_1705_02876_gb300 import synth


@pytest.mark.skipif(shutil.which("g++") is None, reason="no g++")
def test_oracle_flops_per_track_layer(oracle):
    b = synth.make_fit_batch(1, [100])  # the fit workload's tracks: every one reaches all 10 layers
    c = oracle.op_count_fit(b)
    assert c["layers"] == 100 * b.geom.n_layers
    per = c["total"] / c["layers"]
    # the dense 6x6 products make the oracle's count more than twice the
    # structured one; every track-layer takes the same operations
    assert 768 < per < 2500
    assert c["total"] % c["layers"] == 0
    one = oracle.op_count_fit(synth.make_fit_batch(2, [1]))
    assert one["total"] / one["layers"] == per
