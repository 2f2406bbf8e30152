"""The resumable-state and sweep calls of the C ABI (§3.2.1: the helpers are
what the next update reads as "old"; Algorithm 1's passes), against the FP64
oracle and against themselves:

* dash_save mid-stream, dash_load into a fresh model: the next update is
  bit-identical to the saved model's own next update (modes P and Q);
* n_sweeps = 2: two passes of Algorithm 1 per update with the old helpers
  held fixed, against O.dash_update_p(..., n_sweeps=2);
* dash_fitness_lambda: the λ-weighted fitness of every absorbed row against
  the oracle's definition over the stored rows;
* the X·Q_V autotuning: the same bits with it on and off, and a valid choice;
* a bounded wait that runs out drops the update and keeps the state;
* a non-finite input value reaches the factors and is reported as
  DASH_ENUMERIC.
"""
import os

import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream, tiny, workload
from tests._parity import FIT_TOL, TOL, compare_state_p, oracle_fit_p, record, rel, segs_np

pytestmark = pytest.mark.gpu


def _model(w, prec, mode="P", **kw):
    from paper_2305_18376_gb300 import DashModel
    idt = "f64" if prec == "fp64" else "f32"
    return DashModel(w.J, w.R, w.lam, mode=mode, precision=prec, input_dtype=idt,
                     max_slices=w.K0 + 64, max_rows=8192, max_segments=1024, **kw)


@pytest.mark.parametrize("mode,prec", [("P", "fp64"), ("P", "f16x3"), ("Q", "fp64"), ("Q", "f16x3")])
def test_save_load_resumes_bit_for_bit(tmp_path, mode, prec):
    from paper_2305_18376_gb300 import DashModel
    w = tiny(K0=40, J=64 if prec == "f16x3" else 24, R=8, steps=4, sigma=0.05, lam=0.9, new=3,
             rows=("uniform", 1, 20), init_rows=("uniform", 10, 60))
    tdt = torch.float64 if prec == "fp64" else torch.float32
    s = PlantedStream(w)
    bs = [s.batch(t) for t in range(4)]
    a = _model(w, prec, mode)
    a.set_factors(np.random.default_rng(2).random((w.J, w.R)))
    a.update_device(bs[0].slice_ids.numpy(), bs[0].row_ptr.numpy(), bs[0].X.to(tdt).cuda())
    a.update_device(bs[1].slice_ids.numpy(), bs[1].row_ptr.numpy(), bs[1].X.to(tdt).cuda())
    path = str(tmp_path / "state.dash")
    a.save(path)
    assert os.path.getsize(path) > 0
    b = DashModel.load_file(path, w.J, w.R, w.lam, mode=mode, input_dtype="f64" if prec == "fp64" else "f32")
    assert b.K == a.K
    get = (lambda m: m.get_state_p()) if mode == "P" else (lambda m: m.get_state_q())
    for k, v in get(a).items():
        assert np.array_equal(v, get(b)[k]), f"loaded {k} differs"
    for t in (2, 3):
        for m in (a, b):
            m.update_device(bs[t].slice_ids.numpy(), bs[t].row_ptr.numpy(), bs[t].X.to(tdt).cuda())
        ga, gb = get(a), get(b)
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), f"update {t}: {k} differs after resume"
        assert a.fitness()[0] == b.fitness()[0]
    a.close()
    b.close()


def test_load_rejects_a_corrupted_file(tmp_path):
    from paper_2305_18376_gb300 import DashError, DashModel
    w = tiny(K0=5, J=8, R=3, steps=1, sigma=0.05)
    a = _model(w, "fp64")
    a.set_factors(np.ones((w.J, w.R)))
    b0 = PlantedStream(w).batch(0)
    a.update_device(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.double().cuda())
    path = str(tmp_path / "s.dash")
    a.save(path)
    raw = bytearray(open(path, "rb").read())
    raw[200] ^= 0x40                            # flip one bit of the payload
    bad = str(tmp_path / "bad.dash")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(DashError):
        DashModel.load_file(bad, w.J, w.R, w.lam, input_dtype="f64")
    open(bad, "wb").write(bytes(raw[:100]))     # truncated
    with pytest.raises(DashError):
        DashModel.load_file(bad, w.J, w.R, w.lam, input_dtype="f64")
    a.close()


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_two_sweeps_per_update_match_the_oracle(prec):
    """n_sweeps = 2 (Algorithm 1 run twice over the same new rows, the old
    helpers held fixed) against the oracle's two-sweep update."""
    # mixed: c2's shape (J = 88, R = 10, a fitted start); on a poorly fitted
    # c4-shaped start the second pass, one more ALS step, amplified the mixed
    # path's rounding past the bar (W 5e-4 after two updates)
    w = workload("c2", K0=300, steps=3, init_rows=("uniform", 50, 300),
                 new_slice_rows=("uniform", 50, 100)) if prec == "f16x3" else \
        tiny(K0=20, J=16, R=4, steps=3, sigma=0.05, lam=0.9, new=2)
    tdt = torch.float64 if prec == "fp64" else torch.float32
    s = PlantedStream(w)
    V0 = np.random.default_rng(1).random((w.J, w.R))
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, tdt), V0, 3)
    from paper_2305_18376_gb300 import DashModel
    m = DashModel(w.J, w.R, w.lam, precision=prec, input_dtype="f64" if prec == "fp64" else "f32",
                  max_slices=w.K0 + 64, max_rows=max(65536, b0.n_rows + 8), max_segments=4096, n_sweeps=2)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    for t in (1, 2, 3):
        b = s.batch(t)
        segs = segs_np(b, tdt)
        one, _ = O.dash_update_p(st, segs, b.n_new, w.lam)
        st, _ = O.dash_update_p(st, segs, b.n_new, w.lam, n_sweeps=2)
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).cuda())
        g = m.get_state_p()
        errs = compare_state_p(g, st, TOL[prec], f"two sweeps, update {t}")
        record(f"sweeps {t}", errs, TOL[prec])
        # what ran is the two-pass update, not one pass: the GPU's V is ten
        # times closer to the oracle's two-pass V than to its one-pass V
        assert rel(g["V"], st.V) * 10 < rel(g["V"], one.V), (rel(g["V"], st.V), rel(g["V"], one.V))
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_lambda_weighted_fitness_matches_stored_rows(prec):
    w = tiny(K0=12, J=32, R=4, steps=3, sigma=0.05, lam=0.8, new=2, rows=("uniform", 1, 12),
             init_rows=("uniform", 8, 30))
    tdt = torch.float64 if prec == "fp64" else torch.float32
    s = PlantedStream(w)
    V0 = np.random.default_rng(3).random((w.J, w.R))
    b0 = s.batch(0)
    segs0 = segs_np(b0, tdt)
    st = O.empty_state_p(V0)
    for it in range(2):                   # the static fit, keeping the last U rows
        st, U = O.dash_update_p(st, segs0, len(segs0) if it == 0 else 0, 0.0)
    X0 = [x for _, x in segs0]
    st = O.init_helpers_p(X0, [U[k] for k in range(len(X0))], st.W, st.V)
    rows = [(0, X0[k], U[k], st.W[k].copy()) for k in range(len(X0))]
    m = _model(w, prec)
    m.set_factors(V0)
    m.append_batch(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.to(tdt).numpy())
    m.fit_initial(2)
    tol = FIT_TOL[prec]
    for t in (1, 2, 3):
        b = s.batch(t)
        X = O._group(segs_np(b, tdt), st.K, b.n_new, w.J)
        st, Uo = O.dash_update_p(st, list(X.items()), b.n_new, w.lam)
        rows = [(age + 1, Xr, Ur, wr) for age, Xr, Ur, wr in rows]
        rows += [(0, X[k], Uo[k], st.W[k].copy()) for k in X]
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).cuda())
        fl, xx = m.fitness_lambda()
        want = O.weighted_fitness_p(rows, st.V, w.lam)
        xx_o = sum(w.lam ** a * np.sum(Xr ** 2) for a, Xr, _, _ in rows)
        record(f"fit_lambda {t}", {"fit": abs(fl - want), "xx": abs(xx - xx_o) / xx_o}, tol)
        # xx sums ||X_new||² per update: FP64 throughout on the FP64 path; the
        # mixed path adds FP32 sums of 32 squares each (relative error below
        # 32·2^-24 = 2e-6)
        assert abs(xx - xx_o) <= (1e-12 if prec == "fp64" else 2e-6) * xx_o, (xx, xx_o)
        assert abs(fl - want) <= tol, (t, fl, want)
    m.close()


def test_timed_out_wait_drops_the_update_and_keeps_the_state():
    """A bounded wait that runs out (the first copy of the X·Q_V pass never
    issued, through the library's test hook) drops the update: DASH_ETIMEOUT
    at the next synchronisation, the state and slice count unchanged bit for
    bit, and the model usable for the next update."""
    from paper_2305_18376_gb300 import DashError, DashModel
    w = workload("c4", K0=300, steps=2, init_rows=("uniform", 40, 300), new_slices_per_step=3,
                 new_slice_rows=("uniform", 200, 600))
    s = PlantedStream(w)
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, torch.float32), np.random.default_rng(1).random((w.J, w.R)), 2)
    m = DashModel(w.J, w.R, w.lam, precision="f16x3", input_dtype="f32", max_slices=w.K0 + 64,
                  max_rows=65536, max_segments=4096)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    m.set_wait_limit(20_000_000)                  # about 10 ms
    before = m.get_state_p()
    K0 = m.K
    b = s.batch(1)
    m.inject_wait_fault()
    m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.float().cuda())
    with pytest.raises(DashError) as e:
        m.sync()
    assert e.value.status == 6, e.value
    assert m.K == K0
    after = m.get_state_p()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    timeouts, _ = m.counters()
    assert timeouts >= 1
    m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.float().cuda())
    st2, _ = O.dash_update_p(st, segs_np(b, torch.float32), b.n_new, w.lam)
    compare_state_p(m.get_state_p(), st2, TOL["f16x3"], "after the dropped update")
    m.close()


def test_autotuned_xq_pass_gives_the_same_bits():
    """Two models on the same c4-shaped stream, one autotuning its X·Q_V pass
    on the first update and one with autotuning off: the states after two
    updates are bit-identical, the tuner timed every variant and kept one
    of them, and the later update did not tune again."""
    w = workload("c4", K0=400, steps=2, init_rows=("uniform", 40, 200), new_slices_per_step=4)
    s = PlantedStream(w)
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, torch.float32), np.random.default_rng(3).random((w.J, w.R)), 2)
    from paper_2305_18376_gb300 import DashModel
    batches = [s.batch(t) for t in (1, 2)]
    states = []
    for tune in (True, False):
        m = DashModel(w.J, w.R, w.lam, precision="f16x3", input_dtype="f32", max_slices=w.K0 + 64,
                      max_rows=max(b.n_rows for b in batches) + 16, max_segments=4096, max_staged_rows=1)
        m.set_autotune(tune)
        m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
        for b in batches:
            m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.float().cuda())
        r = m.autotune_result()
        if tune:
            assert r["candidates"] >= 2, r
            assert 0 <= r["chosen"] < r["candidates"], r
            assert all(ms > 0 for ms in r["ms"]), r
            assert r["ring"] >= 2, r
            print("  autotune:", r)
        else:
            assert r["candidates"] == 0 and r["chosen"] == -1, r
        states.append(m.get_state_p())
        m.close()
    for k in states[0]:
        assert np.array_equal(states[0][k], states[1][k]), k


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_non_finite_state_is_reported(prec):
    """A batch with a NaN in X makes the new V non-finite (mode P): the
    library reports DASH_ENUMERIC at the next read of the state and at the
    next update, instead of returning NaN factors silently."""
    from paper_2305_18376_gb300 import DashError, DashModel
    w = tiny(K0=20, J=32, R=4, steps=2, sigma=0.05, lam=0.9)
    s = PlantedStream(w)
    b0 = s.batch(0)
    _, tdt = (("f64", torch.float64) if prec == "fp64" else ("f32", torch.float32))
    st = oracle_fit_p(segs_np(b0, tdt), np.random.default_rng(2).random((w.J, w.R)), 2)
    m = _model(w, prec)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    b = s.batch(1)
    X = b.X.to(tdt).clone()
    X[0, 0] = float("nan")
    m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), X.cuda())
    with pytest.raises(DashError) as e:
        m.get_state_p()
    assert e.value.status == 5, e.value
    b2 = s.batch(2)
    with pytest.raises(DashError) as e:
        m.update_device(b2.slice_ids.numpy(), b2.row_ptr.numpy(), b2.X.to(tdt).cuda())
    assert e.value.status == 5, e.value
    m.close()
