"""The bench's reference arm times the FP64 oracle on a bounded sample of the
c4 stream.  Algorithm 1 fixes no scale between S_k and V, so from an unfitted
start W grows without bound within a few updates; the sample starts from the
fitted state the GPU arm also uses.  Here: twenty updates of a 20-slice sample
stay finite with W of order one (the planted weights are U(0,1)).  (With 10
slices the fitted start is too ill-conditioned: the stream drifts until an SVD
fails; the bench samples 50 slices by default.)"""
import numpy as np

import bench


def test_oracle_sample_stays_fitted_over_twenty_updates():
    r = bench.oracle_sample("c4", 20, 20)
    assert len(r["times"]) == 20 and all(np.isfinite(r["times"]))
    assert all(n > 0 for n in r["rows"])
    assert np.isfinite(r["max_abs_W"]) and r["max_abs_W"] < 10.0, r["max_abs_W"]
