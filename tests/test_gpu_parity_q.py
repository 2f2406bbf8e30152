"""Mode Q (U_k = Q_k H S_k) on the GPU against the FP64 oracle, element by
element, through the C ABI.

Tolerances (tests/_parity.shadow_tol): the stated ones (FP64 1e-10, mixed
1e-4, fitness 1e-3), widened only where the problem's conditioning puts them
out of reach.  A shadow oracle run perturbs every bulk product A_new at the
path's rounding level (FP64: 2^-53·sqrt(J+R); mixed: one FP32 rounding);
the limit is 16 times the spread between shadow and oracle when that is
larger than the stated tolerance — for every quantity on the FP64 path, and
for the new Q rows and Y_k on the mixed path (V, H, W, L keep 1e-4 there).
The polar factor Q_k moves by about u·cond(A_k) under a rounding of size u
of A_k, and cond(A_k) reaches 1e4-1e6 on the J=512, R=32 planted shape.
The new Q rows and Y_k are also checked slice by slice, each against the
stated tolerance widened only by that slice's own shadow spread; the records
count the slices whose limit was widened.  Every comparison prints its
errors and limits.
"""
import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream, ragged_batch, tiny, workload
from tests._parity import (FIT_TOL, SHADOW_FACTOR, SHADOW_U, TOL, a_noise, compare_state_q, gpu_rows_by_slice,
                           oracle_y, perturb, record, rel, segs_np, shadow_scale, shadow_tol)

pytestmark = pytest.mark.gpu

PREC_DTYPE = {"fp64": ("f64", torch.float64), "fp32": ("f32", torch.float32),
              "f16x3": ("f32", torch.float32)}


def _model(J, R, lam, prec, **kw):
    from paper_2305_18376_gb300 import DashModel
    idt, _ = PREC_DTYPE[prec]
    return DashModel(J, R, lam, mode="Q", precision=prec, input_dtype=idt, **kw)


def _oracle_fit(X0, V0, R, iters, noise=None):
    """The static fit as the library runs it: iters single-batch updates with
    λ = 0 from H = I, W = 1 (each equals one PARAFAC2-ALS iteration, a pinned
    identity), then the helpers of the final factors."""
    J = V0.shape[0]
    st = O.StateQ(V=np.array(V0, dtype=np.float64), H=np.eye(R), W=np.ones((len(X0), R)),
                  L=np.zeros((len(X0), R, R)), Z=np.zeros((len(X0), R, J)))
    segs = list(enumerate(X0))
    for _ in range(iters):
        st, _, _ = O.dash_update_q(st, segs, 0, 0.0, a_noise=noise)
    return O.init_helpers_q(X0, st.H, st.V, st.W, a_noise=noise)


def _q_spread(st_a, Qa, st_b, Qb) -> dict:
    sp = {"V": rel(st_b.V, st_a.V), "H": rel(st_b.H, st_a.H), "W": rel(st_b.W, st_a.W),
          "L": rel(st_b.L, st_a.L), "Y": rel(oracle_y(st_b), oracle_y(st_a))}
    if Qa is not None:
        sp["Q"] = max((rel(Qb[k], Qa[k]) for k in Qa), default=0.0)
    return sp


def _max_spread(spreads):
    return {k: max(sp[k] for sp in spreads) for k in spreads[0]}


def _run_stream(w, prec, n_steps, init_iters=2, via="batch", seed_v=1, start="fit"):
    """Initialise both sides (the same static fit, or the oracle's state
    loaded with set_state_q), then stream n_steps updates.  A shadow oracle
    run on inputs perturbed by SHADOW_U[prec] sets the tolerances."""
    _, tdt = PREC_DTYPE[prec]
    u = SHADOW_U[prec]
    prng = np.random.default_rng(99)
    s = PlantedStream(w)
    rng = np.random.default_rng(seed_v)
    V0 = rng.random((w.J, w.R))
    b0 = s.batch(0)
    X0 = [x for _, x in segs_np(b0, tdt)]
    noise = a_noise(shadow_scale(prec, w.J, w.R), prng)
    st = _oracle_fit(X0, V0, w.R, init_iters)
    # two independent shadows; the limit takes the larger spread
    shs = [_oracle_fit([perturb(x, u, prng) for x in X0], V0, w.R, init_iters, noise)
           for _ in range(2)]
    m = _model(w.J, w.R, w.lam, prec, max_slices=w.K0 + w.new_slices_per_step * n_steps + 8,
               max_rows=max(4096, b0.n_rows * 2), max_segments=4096)
    if start == "fit":
        m.set_factors(V0)
        m.append_batch(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.to(tdt).numpy())
        m.fit_initial(init_iters)
        tol0 = shadow_tol(prec, _max_spread([_q_spread(st, None, sh, None) for sh in shs]))
        e0 = compare_state_q(m.get_state_q(), st, tol0, "init")
        print("  init errors:", e0, "limits:", tol0)
        record("init", e0, tol0)
    else:
        m.set_state_q(st.V, st.H, st.W, st.L, oracle_y(st))
    worst = {}
    for t in range(1, n_steps + 1):
        b = s.batch(t)
        segs = segs_np(b, tdt)
        X = O._group(segs, st.K, b.n_new, w.J)
        st, Qo, _ = O.dash_update_q(st, list(X.items()), b.n_new, w.lam)
        spreads, Qsh = [], []
        for i, sh in enumerate(shs):
            Xs = {k: perturb(x, u, prng) for k, x in X.items()}
            shs[i], Qs, _ = O.dash_update_q(sh, list(Xs.items()), b.n_new, w.lam, a_noise=noise)
            spreads.append(_q_spread(st, Qo, shs[i], Qs))
            Qsh.append(Qs)
        tol = shadow_tol(prec, _max_spread(spreads))
        Xg = b.X.to(tdt)
        if via == "batch":
            m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), Xg.numpy())
            m.update()
        else:
            m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), Xg.cuda())
        g = m.get_state_q()
        errs = compare_state_q(g, st, tol, f"update {t}")
        # slice by slice: the new Q rows and Y_k of each slice against the
        # stated bar, widened only by that slice's own shadow spread
        rows = gpu_rows_by_slice(m.new_rows(), b)
        q_err = {k: rel(rows[k], Qo[k]) for k in rows}
        q_tol = {k: max(TOL[prec], SHADOW_FACTOR * max(rel(Qs[k], Qo[k]) for Qs in Qsh)) for k in rows}
        Yo = oracle_y(st)
        Ysh = [oracle_y(sh) for sh in shs]
        y_err = {k: rel(g["Y"][k], Yo[k]) for k in range(st.K)}
        y_tol = {k: max(TOL[prec], SHADOW_FACTOR * max(rel(Y[k], Yo[k]) for Y in Ysh)) for k in range(st.K)}
        bad = [k for k in q_err if not q_err[k] <= q_tol[k]] + [k for k in y_err if not y_err[k] <= y_tol[k]]
        assert not bad, ("per-slice Q/Y mismatch", bad[:5], q_err, q_tol)
        errs["Q"] = max(q_err.values(), default=0.0)
        errs["Q_slices_widened"] = sum(1 for k in q_tol if q_tol[k] > TOL[prec])
        errs["Q_slices"] = len(q_tol)
        errs["Y_slice"] = max(y_err.values(), default=0.0)
        errs["Y_slices_widened"] = sum(1 for k in y_tol if y_tol[k] > TOL[prec])
        errs["Y_slices"] = len(y_tol)
        tol = dict(tol, Q=max(q_tol.values(), default=TOL[prec]),
                   Y_slice=max(y_tol.values(), default=TOL[prec]))
        fit_g, _ = m.fitness()
        fit_o = O.fitness([X[k] for k in sorted(X)],
                          [O.reconstruct_q(Qo[k], st.H, st.W[k], st.V) for k in sorted(X)])
        errs["fit"] = abs(fit_g - fit_o)
        print(f"  update {t}:", errs, "limits:", tol)
        record(f"update {t}", errs, tol)
        assert errs["fit"] <= FIT_TOL[prec], (fit_g, fit_o)
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    m.close()
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_stream_parity_q(prec):
    w = tiny(K0=6, J=9, R=3, steps=4, sigma=0.05, lam=0.9)
    _run_stream(w, prec, 4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_stream_from_loaded_state_q(prec):
    w = tiny(K0=7, J=8, R=3, steps=3, sigma=0.05, lam=0.8, init_rows=("uniform", 4, 9))
    _run_stream(w, prec, 3, start="state", via="device")


def test_c1_workload_q_fp64():
    """K0=50, J=100, R=10, λ=1, updates of +10 rows / +5 slices, FP64."""
    w = workload("c1")
    worst = _run_stream(w, "fp64", 4, init_iters=3)
    print("c1 mode-Q fp64 worst relative errors:", worst)


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_c2_shaped_q(prec):
    w = workload("c2", K0=120, init_rows=("uniform", 50, 300), new_slice_rows=("uniform", 50, 100),
                 steps=3)
    worst = _run_stream(w, prec, 3, init_iters=2)
    print(f"c2-shaped mode-Q {prec} worst relative errors:", worst)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_c4_shaped_q(prec):
    """J=512, R=32, lognormal slice lengths, +1..64 rows per slice: the shape
    of the mixed-precision workload at K0=60."""
    w = workload("c4", K0=60, steps=2)
    worst = _run_stream(w, prec, 2, init_iters=2)
    print(f"c4-shaped mode-Q {prec} worst relative errors:", worst)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ragged_edges_q(prec):
    """Empty segments, a slice with fewer rows than R (rank-deficient L_k),
    several segments for one slice, untouched slices, new slices."""
    _, tdt = PREC_DTYPE[prec]
    J, R, lam = 7, 4, 0.7
    rng = np.random.default_rng(11)
    V0 = rng.random((J, R))
    X0 = [rng.standard_normal((n, J)) for n in (9, 6, 2, 12)]
    X0 = [torch.from_numpy(x).to(tdt).to(torch.float64).numpy() for x in X0]
    st = _oracle_fit(X0, V0, R, 2)
    m = _model(J, R, lam, prec, max_slices=16, max_rows=256, max_segments=64)
    m.set_state_q(st.V, st.H, st.W, st.L, oracle_y(st))
    b = ragged_batch(4, 2, J, rows=[3, 0, 1, 2, 5, 0], seed=4, dtype=tdt,
                     slice_ids=[0, 2, 4, 0, 5, 5])
    segs = segs_np(b, tdt)
    X = O._group(segs, st.K, b.n_new, J)
    st, Qo, _ = O.dash_update_q(st, list(X.items()), b.n_new, lam)
    m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).numpy())
    m.update()
    tol = TOL[prec]
    errs = compare_state_q(m.get_state_q(), st, tol, "ragged")
    rows = gpu_rows_by_slice(m.new_rows(), b)
    for k in rows:
        assert rel(rows[k], Qo[k]) <= tol, (k, rel(rows[k], Qo[k]))
    print("ragged mode-Q errors:", errs)
    record("ragged", errs, tol)
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_short_slices_at_rank_32_q(prec):
    """R = 32 with slices of 1-15 rows (rank-deficient L_k, whose QR leaves
    only rounding residues in the columns past the rank): every result stays
    finite and matches the oracle."""
    _, tdt = PREC_DTYPE[prec]
    J, R, lam = 40, 32, 0.9
    rng = np.random.default_rng(21)
    sizes = [60, 9, 15, 3, 1, 45, 12, 33]
    X0 = [torch.from_numpy(rng.random((n, J)) + 0.1 * rng.standard_normal((n, J))).to(tdt)
          .to(torch.float64).numpy() for n in sizes]
    V0 = rng.random((J, R))
    st = _oracle_fit(X0, V0, R, 2)
    m = _model(J, R, lam, prec, max_slices=32, max_rows=1024, max_segments=64)
    m.set_factors(V0)
    rp = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    m.append_batch(np.arange(len(sizes), dtype=np.int64), rp,
                   np.concatenate(X0).astype(np.float64 if prec == "fp64" else np.float32))
    m.fit_initial(2)
    b = ragged_batch(len(sizes), 1, J, rows=[2, 0, 4, 1, 7, 3], seed=8, dtype=tdt,
                     slice_ids=[1, 2, 3, 4, 8, 0])
    segs = segs_np(b, tdt)
    X = O._group(segs, st.K, b.n_new, J)
    st, Qo, _ = O.dash_update_q(st, list(X.items()), b.n_new, lam)
    m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).numpy())
    m.update()
    g = m.get_state_q()                    # DASH_ENUMERIC would raise here
    for k, v in g.items():
        assert np.all(np.isfinite(v)), k
    errs = {k: rel(g[k], v) for k, v in (("V", st.V), ("H", st.H), ("W", st.W))}
    print(f"short slices R=32 {prec}:", errs)
    record("short slices", errs, 1e-8 if prec == "fp64" else 1e-4)
    assert max(errs.values()) <= (1e-8 if prec == "fp64" else 1e-4), errs
    m.close()


def test_q_orthonormal_and_deterministic():
    """The first update on an empty model sees every row of a slice at once,
    so its Q rows are the polar factor: QᵀQ = I when the slice has at least
    R rows.  Two identical runs give identical bits."""
    w = tiny(K0=4, J=6, R=3, steps=3, sigma=0.05, lam=1.0, init_rows=("uniform", 5, 8),
             rows=("uniform", 2, 4))
    outs = []
    for _ in range(2):
        s = PlantedStream(w)
        m = _model(w.J, w.R, 1.0, "fp64", max_slices=32, max_rows=1024, max_segments=256)
        m.set_factors(np.random.default_rng(1).random((w.J, w.R)))
        # one static iteration, then stream; keep the Q rows of slice 0
        b0 = s.batch(0)
        m.append_batch(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.numpy())
        m.update()
        q0 = [gpu_rows_by_slice(m.new_rows(), b0)[0]]
        for t in range(1, 4):
            b = s.batch(t)
            m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.numpy())
            m.update()
            q0.append(gpu_rows_by_slice(m.new_rows(), b).get(0, np.zeros((0, w.R))))
        g = m.get_state_q()
        outs.append((g, q0))
        m.close()
    for k in "VHWLY":
        assert np.array_equal(outs[0][0][k], outs[1][0][k]), k
    q = outs[0][1][0]
    assert q.shape[0] >= w.R
    assert rel(q.T @ q, np.eye(w.R)) < 1e-12


def test_set_state_q_rejects_lower_entries():
    from paper_2305_18376_gb300 import DashError
    m = _model(5, 2, 1.0, "fp64", max_slices=4, max_rows=64, max_segments=16)
    L = np.array([[[1.0, 0.0], [0.5, 1.0]]])
    with pytest.raises(DashError):
        m.set_state_q(np.ones((5, 2)), np.eye(2), np.ones((1, 2)), L, np.zeros((1, 2, 5)))
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_local_errors_q(prec):
    """Definitions 1-2 in mode Q (X̂ = Q_new H S_k Vᵀ with the updated
    factors), and the direct fitness equals dash_fitness()."""
    _, tdt = PREC_DTYPE[prec]
    w = tiny(K0=6, J=9, R=3, steps=1, sigma=0.05, lam=0.9)
    s = PlantedStream(w)
    rng = np.random.default_rng(1)
    V0 = rng.random((w.J, w.R))
    b0 = s.batch(0)
    X0 = [x for _, x in segs_np(b0, tdt)]
    st = _oracle_fit(X0, V0, w.R, 2)
    m = _model(w.J, w.R, w.lam, prec, max_slices=64, max_rows=1024, max_segments=256)
    m.set_state_q(st.V, st.H, st.W, st.L, oracle_y(st))
    b = s.batch(1)
    X = O._group(segs_np(b, tdt), st.K, b.n_new, w.J)
    st, Qo, _ = O.dash_update_q(st, list(X.items()), b.n_new, w.lam)
    m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).cuda())
    te, fd, se = m.local_errors()
    ks = sorted(X)
    Xh = {k: O.reconstruct_q(Qo[k], st.H, st.W[k], st.V) for k in ks}
    se_o = {k: O.slice_error(X[k], Xh[k]) for k in ks if X[k].shape[0] > 0}
    te_o = O.tensor_error([X[k] for k in se_o], [Xh[k] for k in se_o])
    # se and te are means of |x - x̂| with x̂ ≈ x: a relative error TOL of the
    # factors moves each x̂ by about TOL·max|X|, so the bar applies at the
    # scale of the data, not of the residual
    xmax = max(float(np.max(np.abs(X[k]))) for k in se_o)
    tol = TOL[prec] * xmax
    record("local errors", {"te": abs(te - te_o) / xmax,
                            "se": max(abs(se[k] - v) for k, v in se_o.items()) / xmax}, TOL[prec])
    assert abs(te - te_o) <= tol, (te, te_o)
    for k, v in se_o.items():
        assert abs(se[k] - v) <= tol, (k, se[k], v)
    assert abs(m.fitness()[0] - fd) <= 1e-12
    m.close()
