"""Anomaly flags of the dual-way stream (§3.4, §4.5): host logic over the
reconstruction errors that dash_local_errors() returns after each update.

The paper flags an update whose tensor-level error te (Definition 2), and a
slice whose slice-level error se_k (Definition 1), exceeds a threshold equal
to the moving average plus the moving standard deviation of that error over
a window of 5.  It does not say which 5 values form the window nor which
standard deviation.  Reading taken here: the window holds the previous 5
values of the same series (te over the previous updates; se_k over the
previous updates in which slice k received rows), so that the flag of an
update depends only on the past; the standard deviation is the sample one
(divisor n − 1, as MATLAB's std, the paper's platform); a series with fewer
than `window` past values has no threshold yet and is never flagged.
"""
from __future__ import annotations

import math
from collections import deque
from typing import Dict, List, Optional


def threshold(past) -> Optional[float]:
    """Moving mean + moving sample standard deviation of the values in
    `past` (None when there are fewer than two)."""
    n = len(past)
    if n < 2:
        return None
    mean = sum(past) / n
    var = sum((x - mean) ** 2 for x in past) / (n - 1)
    return mean + math.sqrt(var)


class AnomalyThreshold:
    """Feed the errors of each update in order; get the flags of that update.

    observe(te, se) takes te (float) and se (per-slice errors: a mapping
    slice id → se_k, or a sequence indexed by slice id with NaN for slices
    without new rows, as dash_local_errors fills it) and returns
    (tensor_flag, flagged_slice_ids, tensor_threshold, slice_thresholds)."""

    def __init__(self, window: int = 5):
        if window < 2:
            raise ValueError("window must be at least 2")
        self.window = window
        self._te = deque(maxlen=window)
        self._se: Dict[int, deque] = {}

    def _thr(self, past) -> Optional[float]:
        return threshold(list(past)) if len(past) == self.window else None

    def observe(self, te: float, se):
        if isinstance(se, dict):
            items = se.items()
        else:
            items = ((k, v) for k, v in enumerate(se) if not math.isnan(v))
        t_thr = self._thr(self._te)
        t_flag = t_thr is not None and te > t_thr
        self._te.append(float(te))
        flagged: List[int] = []
        s_thr: Dict[int, float] = {}
        for k, v in items:
            k = int(k)
            past = self._se.setdefault(k, deque(maxlen=self.window))
            thr = self._thr(past)
            if thr is not None:
                s_thr[k] = thr
                if v > thr:
                    flagged.append(k)
            past.append(float(v))
        return t_flag, sorted(flagged), t_thr, s_thr
