"""The anomaly threshold of §4.5 (moving mean + moving standard deviation
over a window of 5) on hand sequences."""
import math

import pytest

from paper_2305_18376_gb300.anomaly import AnomalyThreshold, threshold


def test_threshold_by_hand():
    # mean 3, sample variance ((−2)² + (−1)² + 0 + 1² + 2²)/4 = 2.5
    assert threshold([1.0, 2.0, 3.0, 4.0, 5.0]) == pytest.approx(3.0 + math.sqrt(2.5), abs=1e-15)
    assert threshold([2.0, 2.0, 2.0, 2.0, 2.0]) == 2.0
    assert threshold([7.0]) is None


def test_tensor_flags_use_the_previous_five_updates_only():
    det = AnomalyThreshold(5)
    seq = [1.0, 2.0, 3.0, 4.0, 5.0,      # no threshold yet
           5.0,                           # thr = 3 + sqrt(2.5) = 4.58 → flag
           4.0,                           # window 2,3,4,5,5: mean 3.8, sd sqrt(1.7) → thr 5.10 → no
           9.0]                           # window 3,4,5,5,4: mean 4.2, sd sqrt(0.7) → thr 5.04 → flag
    flags = [det.observe(v, {})[0] for v in seq]
    assert flags == [False] * 5 + [True, False, True]


def test_slice_series_advance_only_when_the_slice_has_rows():
    det = AnomalyThreshold(5)
    nan = float("nan")
    # slice 0 gets rows every update; slice 1 every other update
    for t in range(5):
        _, fl, _, thr = det.observe(0.0, [1.0 + 0.1 * t, 2.0 if t % 2 == 0 else nan])
        assert fl == [] and thr == {}
    # slice 0: window 1.0..1.4 (mean 1.2, sd 0.158) → 1.5 is flagged;
    # slice 1 has only 3 past values → no threshold
    _, fl, _, thr = det.observe(0.0, [1.5, 50.0])
    assert fl == [0] and set(thr) == {0}
    assert thr[0] == pytest.approx(1.2 + math.sqrt(0.025), abs=1e-12)


def test_mapping_and_sequence_inputs_agree():
    a, b = AnomalyThreshold(5), AnomalyThreshold(5)
    vals = [[0.5, 0.7], [0.6, 0.2], [0.4, 0.9], [0.5, 0.3], [0.55, 0.6], [3.0, 0.61]]
    for v in vals:
        ra = a.observe(1.0, v)
        rb = b.observe(1.0, {0: v[0], 1: v[1]})
        assert ra[1] == rb[1]
    assert ra[1] == [0]
