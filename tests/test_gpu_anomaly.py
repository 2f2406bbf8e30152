"""Anomaly flags (§3.4 Definitions 1-2, the threshold rule of §4.5) from the
library's reconstruction errors against the same rule applied to the
oracle's slice_error / tensor_error, on a planted stream with one injected
anomalous batch."""
import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from paper_2305_18376_gb300.anomaly import AnomalyThreshold
from synth.planted import PlantedStream, tiny
from tests._parity import oracle_fit_p, segs_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_flags_from_gpu_errors_equal_the_oracles(prec):
    from paper_2305_18376_gb300 import DashModel
    T_BAD, BAD = 7, (3, 11)
    w = tiny(K0=20, J=32, R=4, steps=10, sigma=0.05, lam=0.9, new=1, rows=("uniform", 4, 12),
             init_rows=("uniform", 30, 60))
    tdt = torch.float64 if prec == "fp64" else torch.float32
    s = PlantedStream(w)
    V0 = np.random.default_rng(4).random((w.J, w.R))
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, tdt), V0, 3)
    m = DashModel(w.J, w.R, w.lam, precision=prec, input_dtype="f64" if prec == "fp64" else "f32",
                  max_slices=64, max_rows=4096, max_segments=512)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    det_g, det_o = AnomalyThreshold(5), AnomalyThreshold(5)
    rng = np.random.default_rng(9)
    flagged_bad = None
    for t in range(1, 11):
        b = s.batch(t)
        Xb = b.X.clone().to(tdt)
        if t == T_BAD:                 # the anomaly: the rows of two slices replaced by noise
            rp = b.row_ptr.tolist()
            for q, k in enumerate(b.slice_ids.tolist()):
                if k in BAD:
                    n = rp[q + 1] - rp[q]
                    Xb[rp[q]:rp[q + 1]] = torch.from_numpy(3.0 * rng.standard_normal((n, w.J))).to(tdt)
        segs = [(k, Xb[b.row_ptr[q]:b.row_ptr[q + 1]].to(torch.float64).numpy())
                for q, k in enumerate(b.slice_ids.tolist())]
        X = O._group(segs, st.K, b.n_new, w.J)
        st, Uo = O.dash_update_p(st, list(X.items()), b.n_new, w.lam)
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), Xb.cuda())
        te, _, se = m.local_errors()
        ks = sorted(k for k in X if X[k].shape[0] > 0)
        Xh = {k: O.reconstruct_p(Uo[k], st.W[k], st.V) for k in ks}
        se_o = {k: O.slice_error(X[k], Xh[k]) for k in ks}
        te_o = O.tensor_error([X[k] for k in ks], [Xh[k] for k in ks])
        fg = det_g.observe(te, se)
        fo = det_o.observe(te_o, se_o)
        # thresholds are continuous in the errors: compare flags away from ties
        margin = 1e-3 * max(te_o, 1e-30)
        if fo[2] is not None and abs(te_o - fo[2]) > margin:
            assert fg[0] == fo[0], (t, te, te_o, fg[2], fo[2])
        for k in ks:
            thr = fo[3].get(k)
            if thr is not None and abs(se_o[k] - thr) > 1e-3 * thr:
                assert (k in fg[1]) == (k in fo[1]), (t, k, se[k], se_o[k], thr)
        if t == T_BAD:
            flagged_bad = (fg[0], fg[1])
    m.close()
    tflag, sflags = flagged_bad
    assert tflag, "the anomalous update was not flagged at the tensor level"
    assert set(BAD) <= set(sflags), ("anomalous slices not flagged", sflags)
