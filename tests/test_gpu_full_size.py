"""Mode P at the benchmark's full size (the c4 stream: K0 = 50,000 slices,
J = 512, R = 32, ~1.7 M new rows per update), in the launch configuration the
benchmark times (FP32 input, tensor-core products, the default row
pipeline), checked on sampled outputs the FP64 oracle computes one by one
and on properties that hold at any size:

* sampled slices (old and new): U_k,new (Eq. 11), c_k, D_k (Eqs. 15-16) and
  W(k,:) (Eq. 12) against the oracle's per-slice functions, from the state
  before the update;
* F and G increments (Eqs. 20-21), every entry, against FP64 sums over every
  touched slice of the oracle's U_k,new and W(k,:) (Lemmas 1-2);
* V = F G⁺ (Eq. 17) from the GPU's F and G.
"""
import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream, workload
from tests._parity import rel

pytestmark = pytest.mark.gpu

TOL = 1e-4          # mixed-precision bar of the bulk products


def test_c4_full_size_sampled_outputs():
    from paper_2305_18376_gb300 import DashModel
    w = workload("c4")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = PlantedStream(w, device="cuda", dtype=torch.float32, seed=w.seed + 1000)
    b0, b1 = s.batch(0), s.batch(1)
    b2 = s.batch(2)
    del s
    m = DashModel(w.J, w.R, w.lam, precision="f16x3", input_dtype="f32",
                  max_slices=w.K0 + 3 * w.new_slices_per_step,
                  max_rows=max(b0.n_rows, b1.n_rows, b2.n_rows),
                  max_segments=max(b.slice_ids.numel() for b in (b0, b1, b2)) + 8,
                  stream=stream.cuda_stream, max_staged_rows=1)
    m.set_factors(np.random.default_rng(7).random((w.J, w.R)))
    m.fit_initial_device(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X, 2)
    del b0
    m.update_device(b1.slice_ids.numpy(), b1.row_ptr.numpy(), b1.X)
    st0 = m.get_state_p()
    del b1
    torch.cuda.empty_cache()
    m.update_device(b2.slice_ids.numpy(), b2.row_ptr.numpy(), b2.X)
    assert m.last_plan()["chunk_rows"] == b2.n_rows        # the split row pipeline took every row
    st1 = m.get_state_p()
    U = m.new_rows()
    lam, R = w.lam, w.R
    ids, rp = b2.slice_ids.numpy(), b2.row_ptr.numpy()
    V0 = st0["V"]

    # ---- sampled slices, one by one ----------------------------------------
    rng = np.random.default_rng(0)
    old = [q for q, k in enumerate(ids) if k < b2.K_before and rp[q + 1] > rp[q]]
    new = [q for q, k in enumerate(ids) if k >= b2.K_before]
    pick = rng.choice(old, 40, replace=False).tolist() + rng.choice(new, 10, replace=False).tolist()
    worst = {"U": 0.0, "c": 0.0, "D": 0.0, "W": 0.0}
    for q in pick:
        k = int(ids[q])
        Xk = b2.X[rp[q]:rp[q + 1]].double().cpu().numpy()
        is_new = k >= b2.K_before
        wk = np.ones(R) if is_new else st0["W"][k]
        Uo = O.update_u_new(Xk, V0, wk)
        c0 = np.zeros(R) if is_new else st0["c"][k]
        D0 = np.zeros((R, R)) if is_new else st0["D"][k]
        co = lam * c0 + O.c_term(Xk, V0, Uo)
        Do = lam * D0 + Uo.T @ Uo
        Wo = O.solve_w_row(co, Do, V0)
        errs = {"U": rel(U[rp[q]:rp[q + 1]], Uo), "c": rel(st1["c"][k], co),
                "D": rel(st1["D"][k], Do), "W": rel(st1["W"][k], Wo)}
        for name, e in errs.items():
            worst[name] = max(worst[name], e)
            assert e <= TOL, (k, name, e)
    print("full-size sampled slices, worst relative errors:", worst)

    # ---- F and G increments against the oracle, every touched slice ---------
    # U_k,new (Lemma 1) and W(k,:) (Lemma 2) from the oracle's per-slice
    # functions and the state before the update; c_k's data term through the
    # Khatri-Rao identity vec(X)ᵀ(V ⊙ U) = Σ_i ((X V) ∗ U)(i, :) (Appendix
    # A.2), which the oracle pins check against its literal c_term.
    J = w.J
    segs_of = {}
    for q, k in enumerate(ids):
        segs_of.setdefault(int(k), []).append(q)
    F_inc = np.zeros((J, R))
    G_inc = np.zeros((R, R))
    chunk = 1 << 17
    order = sorted(segs_of, key=lambda k: rp[segs_of[k][0]])
    r0 = 0
    Xh = None
    for k in order:
        qs = segs_of[k]
        lo, hi = int(rp[qs[0]]), int(rp[qs[-1] + 1])
        if Xh is None or hi > r0 + Xh.shape[0] or lo < r0:
            r0 = lo
            Xh = b2.X[lo:max(hi, min(lo + chunk, b2.n_rows))].double().cpu().numpy()
        Xk = np.concatenate([Xh[int(rp[q]) - r0:int(rp[q + 1]) - r0] for q in qs])
        if Xk.shape[0] == 0:
            continue
        is_new = k >= b2.K_before
        wk = np.ones(R) if is_new else st0["W"][k]
        Uo = O.update_u_new(Xk, V0, wk)
        c0 = np.zeros(R) if is_new else st0["c"][k]
        D0 = np.zeros((R, R)) if is_new else st0["D"][k]
        co = lam * c0 + np.sum((Xk @ V0) * Uo, axis=0)
        Wo = O.solve_w_row(co, lam * D0 + Uo.T @ Uo, V0)
        Ut = Uo * Wo                                  # U_k,new S_k,new (Eqs. 20-21)
        F_inc += Xk.T @ Ut
        G_inc += Ut.T @ Ut
    assert rel(st1["G"] - lam * st0["G"], G_inc) <= TOL
    assert rel(st1["F"] - lam * st0["F"], F_inc) <= TOL
    # ---- V = F G⁺ -------------------------------------------------------------
    assert rel(st1["V"], st1["F"] @ O.pinv(st1["G"])) <= 1e-6
    m.close()
