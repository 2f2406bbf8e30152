"""Mode P (Algorithm 1) on the GPU against the FP64 oracle, element by
element, through the C ABI.

FP64 products: every factor and helper within 1e-10 (relative, normwise
max); FP32 products: within 1e-4 and batch fitness within 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream, ragged_batch, tiny, workload
from tests._parity import (FIT_TOL, TOL, compare_state_p, gpu_rows_by_slice, oracle_batch_fitness_p,
                           oracle_fit_p, perturb, record, rel, segs_np)

pytestmark = pytest.mark.gpu

PREC_DTYPE = {"fp64": ("f64", torch.float64), "fp32": ("f32", torch.float32),
              "f16x3": ("f32", torch.float32), "f16x3-fused": ("f32", torch.float32),
              "f16x3-split": ("f32", torch.float32), "f16x3-split-warp": ("f32", torch.float32)}


def _model(J, R, lam, prec, **kw):
    """prec: a precision, or "f16x3-fused" / "f16x3-split" / "f16x3-split-warp"
    for the tensor-core products with that row pipeline."""
    from paper_2305_18376_gb300 import DashModel
    idt, _ = PREC_DTYPE[prec]
    base, _, path = prec.partition("-")
    m = DashModel(J, R, lam, precision=base, input_dtype=idt, **kw)
    if path:
        m.set_row_path(path)
    return m


def _run_stream(w, prec, n_steps, init_iters=3, via="batch", seed_v=1):
    """Initialise both sides with the same static fit, then stream."""
    _, tdt = PREC_DTYPE[prec]
    s = PlantedStream(w)
    rng = np.random.default_rng(seed_v)
    V0 = rng.random((w.J, w.R))
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, tdt), V0, init_iters)
    m = _model(w.J, w.R, w.lam, prec, max_slices=w.K0 + w.new_slices_per_step * n_steps + 8,
               max_rows=max(4096, b0.n_rows * 2), max_segments=4096)
    m.set_factors(V0)
    m.append_batch(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.to(tdt).numpy())
    m.fit_initial(init_iters)
    record("init", compare_state_p(m.get_state_p(), st, TOL[prec], "init"), TOL[prec])
    worst = {}
    for t in range(1, n_steps + 1):
        b = s.batch(t)
        segs = segs_np(b, tdt)
        X = O._group(segs, st.K, b.n_new, w.J)
        st, Uo = O.dash_update_p(st, list(X.items()), b.n_new, w.lam)
        Xg = b.X.to(tdt)
        if via == "batch":
            m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), Xg.numpy())
            m.update()
        elif via == "device":
            m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), Xg.cuda())
        else:   # append_rows / append_slices
            ids = b.slice_ids.tolist()
            rp = b.row_ptr.tolist()
            old = [(q, k) for q, k in enumerate(ids) if k < b.K_before]
            for q, k in old:
                m.append_rows(k, Xg[rp[q]:rp[q + 1]].numpy())
            new = [Xg[rp[q]:rp[q + 1]].numpy() for q, k in enumerate(ids) if k >= b.K_before]
            first = m.append_slices(new)
            assert first == b.K_before
            m.update()
        g = m.get_state_p()
        print(f"  update {t} errors:", {k: rel(g[k], getattr(st, k)) for k in "VWcDFG"})
        errs = compare_state_p(g, st, TOL[prec], f"update {t}")
        rows = gpu_rows_by_slice(m.new_rows(), b)
        errs["U"] = max(rel(rows[k], Uo[k]) for k in rows)
        assert errs["U"] <= TOL[prec], errs
        fit_g, xn = m.fitness()
        fit_o = oracle_batch_fitness_p(st, Uo, X)
        errs["fit"] = abs(fit_g - fit_o)
        record(f"update {t}", errs, TOL[prec])
        assert abs(fit_g - fit_o) <= FIT_TOL[prec], (fit_g, fit_o)
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
    m.close()
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3-fused", "f16x3-split", "f16x3-split-warp"])
def test_small_stream_parity(prec):
    w = tiny(K0=6, J=9, R=3, steps=4, sigma=0.05, lam=0.9)
    _run_stream(w, prec, 4)


@pytest.mark.parametrize("via", ["rows", "device"])
def test_staging_paths_agree(via):
    w = tiny(K0=5, J=7, R=2, steps=3, sigma=0.05, lam=0.8)
    _run_stream(w, "fp64", 3, via=via)


def test_c1_workload_fp64():
    """K0=50, J=100, R=10, λ=1, 10 updates of +10 rows / +5 slices, FP64."""
    w = workload("c1")
    worst = _run_stream(w, "fp64", 10, init_iters=5)
    print("c1 fp64 worst relative errors:", worst)


@pytest.mark.parametrize("prec", ["fp32", "f16x3-fused", "f16x3-split"])
def test_c2_shaped(prec):
    """c2's shape (J=88, R=10, +1 row per slice, +10 slices) at K0=300."""
    w = workload("c2", K0=300, init_rows=("uniform", 50, 300), new_slice_rows=("uniform", 50, 100),
                 steps=5)
    worst = _run_stream(w, prec, 5, init_iters=3)
    print(f"c2-shaped {prec} worst relative errors:", worst)


def _state_from_oracle(w, prec, lam):
    """A fitted oracle state for a small planted tensor."""
    _, tdt = PREC_DTYPE[prec]
    s = PlantedStream(w)
    b0 = s.batch(0)
    X0 = [x for _, x in segs_np(b0, tdt)]
    rng = np.random.default_rng(3)
    U, W, V = O.static_als_p(X0, rng.random((w.J, w.R)), np.ones((len(X0), w.R)), 2)
    return O.init_helpers_p(X0, U, W, V)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3-fused", "f16x3-split"])
def test_ragged_edge_batch_from_oracle_state(prec):
    """One update from an oracle state with: a slice split in two segments,
    untouched slices (λ decay only), a 1-row segment, a segment longer than
    one tile (ragged tail), and new slices of 0 and 70 rows."""
    _, tdt = PREC_DTYPE[prec]
    w = tiny(K0=8, J=37, R=5, steps=0, sigma=0.05, init_rows=("uniform", 10, 20))
    st = _state_from_oracle(w, prec, 0.7)
    ids = [0, 2, 2, 5, 7, 8, 9]
    rows = [3, 2, 1, 133, 1, 0, 70]
    b = ragged_batch(8, 2, 37, rows, seed=9, slice_ids=ids, dtype=tdt)
    segs = segs_np(b, tdt)
    st2, Uo = O.dash_update_p(st, segs, 2, 0.7)
    m = _model(37, 5, 0.7, prec, max_slices=16, max_rows=512, max_segments=64)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    m.append_batch(ids, b.row_ptr.numpy(), b.X.numpy())
    m.update()
    g = m.get_state_p()
    compare_state_p(g, st2, TOL[prec], "ragged")
    got = gpu_rows_by_slice(m.new_rows(), b)
    for k in Uo:
        assert rel(got[k], Uo[k]) <= TOL[prec]
    assert np.all(g["W"][8] == 0.0)          # new slice without rows: w = 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rank_deficient_gram_uses_the_pseudo_inverse(prec):
    """J < R: VᵀV is singular, Lemma 1 needs the pseudo-inverse (eigen path)."""
    J, R = 4, 5
    _, tdt = PREC_DTYPE[prec]
    rng = np.random.default_rng(4)
    V0 = rng.random((J, R))
    b = ragged_batch(0, 4, J, [6, 2, 9, 4], seed=5, dtype=tdt)
    segs = segs_np(b, tdt)
    st, Uo = O.dash_update_p(O.empty_state_p(V0), segs, 4, 1.0)
    m = _model(J, R, 1.0, prec, max_slices=8, max_rows=64, max_segments=8)
    m.set_factors(V0)
    m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.numpy())
    m.update()
    tol = TOL[prec]
    record("J<R", compare_state_p(m.get_state_p(), st, tol, "J<R"), tol)
    got = gpu_rows_by_slice(m.new_rows(), b)
    for k in Uo:
        assert rel(got[k], Uo[k]) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3-fused", "f16x3-split"])
def test_zero_weight_entries_take_the_general_lemma1_path(prec):
    """A slice whose S_k has zero entries: S (S Γ S)⁺ ≠ Γ⁻¹ S⁻¹ (in the
    fused kernel this is its in-kernel FP64 fallback)."""
    _, tdt = PREC_DTYPE[prec]
    w = tiny(K0=4, J=8, R=3, steps=0, sigma=0.05)
    st = _state_from_oracle(w, prec, 1.0)
    st.W[1, 0] = 0.0
    st.W[2, :] = 0.0
    b = ragged_batch(4, 0, 8, [5, 4, 3], seed=6, slice_ids=[0, 1, 2], dtype=tdt)
    segs = segs_np(b, tdt)
    st2, Uo = O.dash_update_p(st, segs, 0, 0.9)
    m = _model(8, 3, 0.9, prec, max_slices=8, max_rows=64, max_segments=8)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.numpy())
    m.update()
    tol = TOL[prec]
    record("zero w", compare_state_p(m.get_state_p(), st2, tol, "zero w"), tol)
    got = gpu_rows_by_slice(m.new_rows(), b)
    for k in Uo:
        assert rel(got[k], Uo[k]) <= tol


@pytest.mark.parametrize("prec", ["fp32", "f16x3-fused", "f16x3-split", "f16x3-split-warp"])
def test_fused_tiles_span_many_slices_and_ctas(prec):
    """A few thousand small slices of 1-64 rows (c4's update shape at small J
    and R): many tiles per CTA, big and split slices on the chunked path in
    the same update."""
    w = tiny(K0=3000, J=48, R=8, steps=2, sigma=0.1, lam=0.95, rows=("uniform", 1, 64),
             new=5, new_rows=("uniform", 100, 700), init_rows=("uniform", 8, 40))
    worst = _run_stream(w, prec, 2, init_iters=2)
    print(f"many-slice {prec} worst relative errors:", worst)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3-fused", "f16x3-split", "f16x3-split-warp"])
def test_c4_shape_small_k(prec):
    """c4's J = 512 and R = 32 (full register tiles of the MMA path) at
    K0 = 300 slices."""
    w = workload("c4", K0=300, steps=2, init_rows=("uniform", 40, 300),
                 new_slices_per_step=3, new_slice_rows=("uniform", 200, 600))
    worst = _run_stream(w, prec, 2, init_iters=2)
    print(f"c4-shaped {prec} worst relative errors:", worst)


def test_empty_update_is_pure_decay():
    w = tiny(K0=4, J=8, R=3, steps=0, sigma=0.05)
    st = _state_from_oracle(w, "fp64", 0.5)
    st2, _ = O.dash_update_p(st, [], 0, 0.5)
    m = _model(8, 3, 0.5, "fp64", max_slices=8, max_rows=64, max_segments=8)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    m.update()
    compare_state_p(m.get_state_p(), st2, 1e-10, "empty")


def test_update_is_deterministic():
    w = tiny(K0=30, J=40, R=6, steps=1, sigma=0.05)
    st = _state_from_oracle(w, "fp32", 0.9)
    s = PlantedStream(w)
    s.batch(0)
    b = s.batch(1)
    outs = []
    for _ in range(2):
        m = _model(40, 6, 0.9, "fp32", max_slices=64, max_rows=4096, max_segments=128)
        m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
        m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.float().numpy())
        m.update()
        outs.append(m.get_state_p())
        m.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_capacity_and_argument_errors_leave_state_unchanged():
    from paper_2305_18376_gb300 import DashError
    m = _model(6, 2, 0.9, "fp32", max_slices=4, max_rows=8, max_segments=4)
    m.set_factors(np.ones((6, 2)))
    with pytest.raises(DashError):
        m.append_rows(0, np.zeros((2, 6), np.float32))        # slice 0 does not exist
    with pytest.raises(DashError):
        m.append_slices([np.zeros((9, 6), np.float32)])       # > max_rows
    with pytest.raises(DashError):
        m.append_batch([0, 2], [0, 1, 2], np.zeros((2, 6), np.float32))   # id gap
    assert m.K == 0
    m.append_slices([np.ones((3, 6), np.float32)])
    m.update()
    assert m.K == 1


@pytest.mark.parametrize("prec", ["fp64", "f16x3-fused", "f16x3-split"])
def test_local_errors_match_definitions(prec):
    """Definitions 1-2 on the last update's rows: se per slice, te, and the
    direct batch fitness, against the oracle's slice_error / tensor_error /
    fitness with the same updated factors."""
    _, tdt = PREC_DTYPE[prec]
    w = tiny(K0=7, J=10, R=3, steps=2, sigma=0.05, lam=0.9, new=2)
    s = PlantedStream(w)
    rng = np.random.default_rng(4)
    b0 = s.batch(0)
    X0 = [x for _, x in segs_np(b0, tdt)]
    U, W, V = O.static_als_p(X0, rng.random((w.J, w.R)), np.ones((len(X0), w.R)), 2)
    st = O.init_helpers_p(X0, U, W, V)
    m = _model(w.J, w.R, w.lam, prec, max_slices=64, max_rows=1024, max_segments=256)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    for t in (1, 2):
        b = s.batch(t)
        X = O._group(segs_np(b, tdt), st.K, b.n_new, w.J)
        st, Uo = O.dash_update_p(st, list(X.items()), b.n_new, w.lam)
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).cuda())
        te, fd, se = m.local_errors()
        ks = sorted(X)
        Xh = {k: O.reconstruct_p(Uo[k], st.W[k], st.V) for k in ks}
        se_o = {k: O.slice_error(X[k], Xh[k]) for k in ks if X[k].shape[0] > 0}
        te_o = O.tensor_error([X[k] for k in se_o], [Xh[k] for k in se_o])
        fit_o = O.fitness([X[k] for k in ks], [Xh[k] for k in ks])
        # se and te are means of |x - x̂| with x̂ ≈ x: the factors' relative
        # error TOL moves each x̂ by at most about TOL·|x̂| ≤ TOL·max|X|, so
        # the stated bar applies to se and te at the scale of the data, not
        # of the (much smaller) residual
        xmax = max(float(np.max(np.abs(X[k]))) for k in se_o)
        tol = TOL[prec] * xmax
        record(f"local errors {t}", {"te": abs(te - te_o) / xmax,
                                     "se": max(abs(se[k] - v) for k, v in se_o.items()) / xmax,
                                     "fit": abs(fd - fit_o)}, TOL[prec])
        assert abs(te - te_o) <= tol, (te, te_o)
        assert abs(fd - fit_o) <= FIT_TOL[prec], (fd, fit_o)
        for k, v in se_o.items():
            assert abs(se[k] - v) <= tol, (k, se[k], v)
        untouched = [k for k in range(st.K) if k not in se_o]
        assert all(np.isnan(se[k]) for k in untouched)
        # the direct fitness agrees with the Gram-form fitness of the update
        # (GPU against GPU: the Gram form ||X||² − 2·cross + ||X̂||² cancels
        # to about 1e-8 relative of ||X||² at σ = 0.05, hence 1e-9 there)
        assert abs(m.fitness()[0] - fd) <= (1e-9 if prec == "fp64" else 1e-3)
    m.close()


def test_large_host_appends_overlap_and_match_device_updates():
    """Host batches of >= 64 MB are split over several copy streams into a
    double-buffered staging area; the next batch is appended while the
    previous update runs.  The result is bit-identical to device-resident
    updates of the same batches."""
    w = tiny(K0=600, J=512, R=8, steps=3, sigma=0.05, lam=0.9, rows=("uniform", 40, 80),
             new=4, new_rows=("uniform", 100, 300), init_rows=("uniform", 40, 80))
    s = PlantedStream(w)
    bs = [s.batch(t) for t in range(4)]
    assert min(b.n_rows for b in bs[1:]) * w.J * 4 >= 64 << 20    # the split-copy path
    kw = dict(max_slices=w.K0 + 64, max_rows=max(b.n_rows for b in bs) + 8, max_segments=4096)
    ma = _model(w.J, w.R, w.lam, "f16x3", **kw)
    mb = _model(w.J, w.R, w.lam, "f16x3", **kw)
    V0 = np.random.default_rng(2).random((w.J, w.R))
    for m in (ma, mb):
        m.set_factors(V0)
        m.update_device(bs[0].slice_ids.numpy(), bs[0].row_ptr.numpy(), bs[0].X.float().cuda())
    pinned = [torch.empty(b.X.shape, dtype=torch.float32, pin_memory=True).copy_(b.X.float())
              for b in bs]
    ma.append_batch(bs[1].slice_ids.numpy(), bs[1].row_ptr.numpy(), pinned[1])
    for t in (1, 2, 3):
        ma.update()
        if t < 3:                       # next batch's copy overlaps this update
            ma.append_batch(bs[t + 1].slice_ids.numpy(), bs[t + 1].row_ptr.numpy(), pinned[t + 1])
        fa = ma.fitness()[0]
        mb.update_device(bs[t].slice_ids.numpy(), bs[t].row_ptr.numpy(), bs[t].X.float().cuda())
        assert fa == mb.fitness()[0]
    ga, gb = ma.get_state_p(), mb.get_state_p()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    ma.close()
    mb.close()


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_rows_error_is_the_global_error_of_accumulated_rows(prec):
    """dash_rows_error over every row of several updates (each with the U rows
    its update produced) against the oracle's Σ ||X_k − U_k S_k Vᵀ||² with the
    current S_k and V: the global error of §4.1."""
    _, tdt = PREC_DTYPE[prec]
    w = tiny(K0=7, J=10, R=3, steps=3, sigma=0.05, lam=0.9, new=2)
    s = PlantedStream(w)
    rng = np.random.default_rng(4)
    b0 = s.batch(0)
    X0 = [x for _, x in segs_np(b0, tdt)]
    U, W, V = O.static_als_p(X0, rng.random((w.J, w.R)), np.ones((len(X0), w.R)), 2)
    st = O.init_helpers_p(X0, U, W, V)
    m = _model(w.J, w.R, w.lam, prec, max_slices=64, max_rows=1024, max_segments=256)
    m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
    ids_all, rows_all, X_all, U_gpu, U_orc = [], [0], [], [], []
    for t in (1, 2, 3):
        b = s.batch(t)
        X = O._group(segs_np(b, tdt), st.K, b.n_new, w.J)
        st, Uo = O.dash_update_p(st, list(X.items()), b.n_new, w.lam)
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).cuda())
        U_gpu.append(m.new_rows())
        rp = b.row_ptr.tolist()
        for q, k in enumerate(b.slice_ids.tolist()):
            ids_all.append(k)
            rows_all.append(rows_all[-1] + rp[q + 1] - rp[q])
            U_orc.append(Uo[k][: rp[q + 1] - rp[q]] if k in Uo else np.zeros((0, w.R)))
        X_all.append(b.X.to(tdt))
        # the oracle side: every accumulated segment with the current factors
        e2_o = x2_o = 0.0
        Xc = torch.cat(X_all).numpy().astype(np.float64)
        for q, k in enumerate(ids_all):
            xs = Xc[rows_all[q]:rows_all[q + 1]]
            xh = O.reconstruct_p(U_orc[q], st.W[k], st.V)
            e2_o += float(np.sum((xs - xh) ** 2))
            x2_o += float(np.sum(xs ** 2))
        e2, x2, ea = m.rows_error(ids_all, rows_all, torch.cat(X_all).cuda(),
                                  torch.from_numpy(np.concatenate(U_gpu)).cuda())
        # the mixed path's X̂ is within ~1e-5 of |X|; the residual is ~σ, so
        # its sum of squares carries that error amplified by |X|/σ
        tol = 1e-8 if prec == "fp64" else 5e-3
        assert abs(x2 - x2_o) <= 1e-12 * x2_o
        assert abs(e2 - e2_o) <= tol * e2_o, (t, e2, e2_o)
        assert ea > 0
    m.close()


def test_long_stream_from_an_unfitted_start_tracks_the_oracle():
    """Algorithm 1 fixes no scale between S_k and V (Eqs. 11-17 are invariant
    under S_k → αS_k, V → V/α).  From an unfitted start (one static iteration
    on slices of R..2R rows, c4's update recipe at K0 = 200) the W rows grow
    and V shrinks update after update, until G overflows.  The FP64 path
    follows the oracle update by update:
      * while the state is well scaled (max |W| < 2): within 1e-10;
      * while the systems it inverts stay well posed (cond of G and of VᵀV
        below 1e10, far inside the pseudo-inverse cut-off 1/(R·ε)): within
        1e-10 or 16× the spread of a shadow oracle stream started one FP64
        rounding per entry away, whichever is larger — the drifting update
        map amplifies rounding-sized differences in the oracle itself;
      * after that the pseudo-inverses' rank decisions are themselves
        ill-posed, and the GPU state must have drifted the same way (max |W|
        above 1e3) or been reported non-finite."""
    w = workload("c4", K0=200, steps=14, init_rows=("uniform", 32, 64), new_slices_per_step=1)
    s = PlantedStream(w)
    V0 = np.random.default_rng(0).random((w.J, w.R))
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, torch.float64), V0, 1)
    prng = np.random.default_rng(5)
    sh = O.StateP(*(perturb(getattr(st, f), 2.0 ** -53, prng) for f in ("V", "W", "c", "D", "F", "G")))
    m = _model(w.J, w.R, w.lam, "fp64", max_slices=w.K0 + 64, max_rows=b0.n_rows + 8192,
               max_segments=4096)
    m.set_factors(V0)
    m.append_batch(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.double().numpy())
    m.fit_initial(1)
    compare_state_p(m.get_state_p(), st, TOL["fp64"], "init")
    drifted = compared = False
    for t in range(1, 15):
        b = s.batch(t)
        segs = segs_np(b, torch.float64)
        try:
            with np.errstate(all="ignore"):
                st, _ = O.dash_update_p(st, segs, b.n_new, w.lam)
                sh, _ = O.dash_update_p(sh, segs, b.n_new, w.lam)
            o_ok = all(np.all(np.isfinite(getattr(x, f))) for x in (st, sh) for f in ("V", "W", "G"))
        except np.linalg.LinAlgError:
            o_ok = False
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.double().cuda())
        try:
            g = m.get_state_p()
            g_ok = bool(np.all(np.isfinite(g["W"])) and np.all(np.isfinite(g["V"])))
        except Exception:          # DASH_ENUMERIC: the library saw the overflow
            g, g_ok = None, False
        if not o_ok:
            print(f"  update {t}: oracle state no longer finite; GPU finite: {g_ok}")
            if g_ok:
                assert float(np.max(np.abs(g["W"]))) > 1e3, "GPU state did not drift with the oracle"
            drifted = True
            break
        wmax = float(np.max(np.abs(st.W)))
        cond = max(np.linalg.cond(st.G), np.linalg.cond(st.V.T @ st.V))
        if cond >= 1e10:
            gw = float(np.max(np.abs(g["W"]))) if g_ok else float("inf")
            print(f"  update {t}: max|W| {wmax:.3g}, cond {cond:.3g}: ill-posed; GPU max|W| {gw:.3g}")
            record(f"drift {t}", {"wmax": wmax, "cond": cond, "gpu_wmax": gw}, None)
            assert gw > 1e3, "GPU state did not drift with the oracle"
            drifted = True
            continue
        assert g_ok, f"update {t}: GPU state non-finite while the oracle's is finite and well posed"
        errs = {k: rel(g[k], getattr(st, k)) for k in "VWcDFG"}
        spread = max(rel(getattr(sh, k), getattr(st, k)) for k in "VWcDFG")
        limit = TOL["fp64"] if wmax < 2.0 else max(TOL["fp64"], 16.0 * spread)
        print(f"  update {t}: max|W| {wmax:.3g} cond {cond:.3g} errors {errs} shadow spread {spread:.3g} "
              f"limit {limit:.3g}")
        record(f"drift {t}", {**errs, "shadow_spread": spread, "wmax": wmax, "cond": cond}, limit)
        assert max(errs.values()) <= limit, (t, errs, limit)
        compared = True
        drifted = drifted or wmax > 1e3
    m.close()
    assert compared and drifted, "the stream did not drift: the test no longer covers the unnormalised regime"


@pytest.mark.parametrize("prec", ["fp64", "f16x3"])
def test_graph_launched_updates_are_bit_identical(prec):
    """Updates submitted as one captured CUDA graph (re-used across batches of
    the same launch topology) give the same bits as plain launches."""
    _, tdt = PREC_DTYPE[prec]
    w = workload("c2", K0=300, steps=4, init_rows=("uniform", 50, 300),
                 new_slice_rows=("uniform", 50, 100))
    s = PlantedStream(w)
    b0 = s.batch(0)
    st = oracle_fit_p(segs_np(b0, tdt), np.random.default_rng(1).random((w.J, w.R)), 2)
    ms = []
    for graph in (False, True):
        m = _model(w.J, w.R, w.lam, prec, max_slices=w.K0 + 64, max_rows=8192, max_segments=4096)
        m.set_state_p(st.V, st.W, st.c, st.D, st.F, st.G)
        m.set_graph(graph)
        ms.append(m)
    for t in range(1, 5):
        b = s.batch(t)
        for m in ms:
            m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(tdt).cuda())
        ga, gb = ms[0].get_state_p(), ms[1].get_state_p()
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), (t, k)
        assert ms[0].fitness()[0] == ms[1].fitness()[0]
    inst, upd = ms[1].graph_stats()
    assert inst >= 1 and upd >= 1 and inst + upd == 4, (inst, upd)
    for m in ms:
        m.close()
