"""The benchmark's DVH report (host post-processing of the GPU's doses) on a
hand-worked example: cumulative DVH, its band over scenarios and the dose
metrics."""
import numpy as np
import pytest

import bench


def test_dvh_report_hand_worked():
    # structure 1 has 4 voxels; voxel 4 belongs to no structure
    doses = np.array([[10.0, 20.0, 30.0, 40.0, 99.0],
                      [0.0, 20.0, 20.0, 60.0, 99.0]])
    labels = np.array([1, 1, 1, 1, -1])
    r = bench.dvh_report(doses, labels, levels=[0.0, 15.0, 25.0, 50.0])
    assert list(r) == ["target"]
    t = r["target"]
    assert t["voxels"] == 4
    # V(d): s0 -> 1, 3/4, 2/4, 0 ; s1 -> 1, 3/4, 1/4, 1/4
    assert t["dvh_nominal"] == [1.0, 0.75, 0.5, 0.0]
    assert t["dvh_band_min"] == [1.0, 0.75, 0.25, 0.0]
    assert t["dvh_band_max"] == [1.0, 0.75, 0.5, 0.25]
    m = t["metrics_gy"]
    assert m["mean"] == [25.0, 25.0, 25.0]
    assert m["max"] == [40.0, 50.0, 60.0]
    # D98: 0.02 quantile; s0: 10 + 0.06 * 10 = 10.6, s1: 0 + 0.06 * 20 = 1.2
    assert m["d98"] == pytest.approx([1.2, 5.9, 10.6])
    # D2: 0.98 quantile; s0: 30 + 0.94 * 10 = 39.4, s1: 20 + 0.94 * 40 = 57.6
    assert m["d2"] == pytest.approx([39.4, 48.5, 57.6])
