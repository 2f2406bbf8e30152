"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: direct
least squares (numpy lstsq), closed forms derived by hand, exact identities,
explicit loops, or library routines (SVD, eigh).  A dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream, ragged_batch, tiny

RNG = np.random.default_rng(20230518)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _segs(batch):
    return [(k, x.numpy()) for k, x in batch.segments()]


# ---------------------------------------------------------------------------
# Linear-algebra building blocks
# ---------------------------------------------------------------------------

def test_khatri_rao_matches_elementwise_definition():
    A = RNG.standard_normal((4, 3))
    B = RNG.standard_normal((5, 3))
    KR = O.khatri_rao(A, B)
    for j in range(4):
        for i in range(5):
            for r in range(3):
                assert KR[j * 5 + i, r] == A[j, r] * B[i, r]


def test_khatri_rao_gram_identity():
    """Appendix A.2: (A ⊙ B)ᵀ(A ⊙ B) = AᵀA ∗ BᵀB."""
    A = RNG.standard_normal((6, 4))
    B = RNG.standard_normal((7, 4))
    KR = O.khatri_rao(A, B)
    assert _rel(KR.T @ KR, (A.T @ A) * (B.T @ B)) < 1e-13


def test_c_term_equals_explicit_triple_sum():
    """vec(X)ᵀ(V ⊙ U) (Eq. 15) = Σ_ij X(i,j) V(j,r) U(i,r) by loops."""
    X = RNG.standard_normal((5, 4))
    V = RNG.standard_normal((4, 3))
    U = RNG.standard_normal((5, 3))
    got = O.c_term(X, V, U)
    want = np.zeros(3)
    for r in range(3):
        for i in range(5):
            for j in range(4):
                want[r] += X[i, j] * V[j, r] * U[i, r]
    assert _rel(got, want) < 1e-13


def test_pinv_penrose_conditions_rank_deficient():
    M = RNG.standard_normal((6, 3)) @ RNG.standard_normal((3, 6))    # rank 3
    P = O.pinv(M)
    assert _rel(M @ P @ M, M) < 1e-10
    assert _rel(P @ M @ P, P) < 1e-10
    assert _rel((M @ P).T, M @ P) < 1e-10
    assert _rel((P @ M).T, P @ M) < 1e-10
    N = RNG.standard_normal((5, 5)) + 5 * np.eye(5)
    assert _rel(O.pinv(N), np.linalg.inv(N)) < 1e-12
    assert np.all(O.pinv(np.zeros((3, 3))) == 0)


def test_inv_sqrt_gives_polar_factor():
    A = RNG.standard_normal((9, 4))
    T = O.inv_sqrt_psd(A.T @ A)
    P, _, Zt = np.linalg.svd(A, full_matrices=False)
    assert _rel(A @ T, P @ Zt) < 1e-12
    assert _rel(T @ (A.T @ A) @ T, np.eye(4)) < 1e-12
    # rank-deficient: Q = A T has orthonormal columns on the range only
    A2 = A[:, :2] @ RNG.standard_normal((2, 4))
    T2 = O.inv_sqrt_psd(A2.T @ A2)
    Q2 = A2 @ T2
    ev = np.linalg.eigvalsh(Q2.T @ Q2)
    assert np.allclose(np.sort(ev), [0, 0, 1, 1], atol=1e-8)


def test_r_factor_is_the_triangular_square_root():
    M = RNG.standard_normal((9, 4))
    L = O.r_factor(M)
    assert np.all(np.tril(L, -1) == 0) and np.all(np.diag(L) > 0)
    assert _rel(L.T @ L, M.T @ M) < 1e-13
    assert _rel(L, np.linalg.cholesky(M.T @ M).T) < 1e-12
    # fewer rows than columns: zero rows below, still LᵀL = MᵀM
    M2 = RNG.standard_normal((2, 4))
    L2 = O.r_factor(M2)
    assert L2.shape == (4, 4) and np.all(L2[2:] == 0)
    assert _rel(L2.T @ L2, M2.T @ M2) < 1e-13
    assert np.all(O.r_factor(np.zeros((0, 3))) == 0)
    # updating by stacking equals factoring all rows at once
    M3 = RNG.standard_normal((5, 4))
    up = O.r_factor(np.vstack([np.sqrt(0.7) * L, M3]))
    assert _rel(up.T @ up, 0.7 * M.T @ M + M3.T @ M3) < 1e-13


def test_inv_sqrt_from_factor_is_accurate_where_the_gram_is_not():
    """T = (LᵀL)^{-1/2} from the factor gives the polar factor A·T to about
    eps·cond(A); through B = AᵀA only to eps·cond(A)²."""
    A = RNG.standard_normal((9, 4))
    T = O.inv_sqrt_from_factor(O.r_factor(A))
    P, _, Zt = np.linalg.svd(A, full_matrices=False)
    assert _rel(A @ T, P @ Zt) < 1e-13
    assert _rel(T, O.inv_sqrt_psd(A.T @ A)) < 1e-12
    # cond(A) = 1e6: the Gram route has cond 1e12
    U, _ = np.linalg.qr(RNG.standard_normal((40, 4)))
    Vq, _ = np.linalg.qr(RNG.standard_normal((4, 4)))
    A = (U * np.array([1.0, 1e-2, 1e-4, 1e-6])) @ Vq.T
    polar = U @ Vq.T
    err_f = _rel(A @ O.inv_sqrt_from_factor(O.r_factor(A)), polar)
    assert err_f < 1e-8
    # rank-deficient: same cut as inv_sqrt_psd on the Gram matrix
    A2 = A[:, :2] @ RNG.standard_normal((2, 4))
    T2 = O.inv_sqrt_from_factor(O.r_factor(A2))
    Q2 = A2 @ T2
    ev = np.linalg.eigvalsh(Q2.T @ Q2)
    assert np.allclose(np.sort(ev), [0, 0, 1, 1], atol=1e-8)
    assert np.all(O.inv_sqrt_from_factor(np.zeros((3, 3))) == 0)


# ---------------------------------------------------------------------------
# Lemma 1-3 as least-squares minimisers
# ---------------------------------------------------------------------------

def test_lemma1_u_new_is_the_least_squares_solution():
    """Lemma 1 (Eq. 11) minimises Eq. 10: compare with lstsq directly."""
    X = RNG.standard_normal((7, 6))
    V = RNG.standard_normal((6, 3))
    w = RNG.random(3) + 0.5
    U = O.update_u_new(X, V, w)
    want = np.linalg.lstsq(V * w, X.T, rcond=None)[0].T
    assert _rel(U, want) < 1e-11
    # the gradient of Appendix A.1 vanishes
    S = np.diag(w)
    g = X @ V @ S - U @ S @ V.T @ V @ S
    assert np.max(np.abs(g)) < 1e-11 * np.max(np.abs(X @ V @ S))


def test_lemma1_rank_deficient_v_gives_minimum_norm_solution():
    """J < R: VᵀV is singular; the pseudo-inverse reading returns lstsq's
    minimum-norm solution."""
    X = RNG.standard_normal((4, 2))
    V = RNG.standard_normal((2, 3))
    w = np.array([1.0, 2.0, 0.5])
    U = O.update_u_new(X, V, w)
    want = np.linalg.lstsq(V * w, X.T, rcond=None)[0].T
    assert _rel(U, want) < 1e-10


def _weighted_lstsq(A, b, wts):
    s = np.sqrt(wts)
    return np.linalg.lstsq(A * s[:, None], b * s[:, None] if b.ndim == 2 else b * s,
                           rcond=None)[0]


@pytest.mark.parametrize("lam", [1.0, 0.6])
def test_lemma2_w_minimises_weighted_loss_with_v_frozen(lam):
    """With V frozen, Eq. 12 (through the streamed c_k, D_k of Eqs. 15-16)
    minimises Eq. 5, i.e. Σ_rows λ^age ||x - (u ∘ w_k) Vᵀ||², over W(k,:)."""
    s = PlantedStream(tiny(K0=4, J=6, R=3, steps=3, sigma=0.05, lam=lam))
    V0 = RNG.random((6, 3))
    ost = O.OracleStream("P", V0, lam)
    for t in range(4):
        b = s.batch(t)
        ost.update(_segs(b), b.n_new, freeze_V=True)
    V = ost.state.V
    assert np.array_equal(V, V0)
    for k in range(ost.state.K):
        Xk, Uk, wts = ost.slice_rows(k)
        # vec over rows: x(i,:) ≈ Σ_r w_r U(i,r) V(:,r)ᵀ
        A = np.stack([np.kron(V[:, r], Uk[:, r]) for r in range(3)], axis=1)
        wrow = np.repeat(wts, 1)
        rw = np.tile(wrow, V.shape[0])              # vec is column-major: rows vary fastest
        want = _weighted_lstsq(A, O.vec(Xk), rw)
        assert _rel(ost.state.W[k], want) < 1e-9


@pytest.mark.parametrize("lam", [1.0, 0.6])
def test_lemma3_v_minimises_weighted_loss_with_w_frozen(lam):
    """With S_k frozen, Eq. 17 through the streamed F, G (Eqs. 20-21)
    minimises Σ_k Σ_rows λ^age ||x - u S_k Vᵀ||² over V."""
    s = PlantedStream(tiny(K0=4, J=6, R=3, steps=3, sigma=0.05, lam=lam))
    V0 = RNG.random((6, 3))
    ost = O.OracleStream("P", V0, lam)
    for t in range(4):
        b = s.batch(t)
        ost.update(_segs(b), b.n_new, freeze_W=True)
    W = ost.state.W
    assert np.all(W == 1.0)
    Ms, Xs, ws = [], [], []
    for k in range(ost.state.K):
        Xk, Uk, wts = ost.slice_rows(k)
        Ms.append(Uk * W[k]); Xs.append(Xk); ws.append(wts)
    want = _weighted_lstsq(np.vstack(Ms), np.vstack(Xs), np.concatenate(ws)).T
    assert _rel(ost.state.V, want) < 1e-9


# ---------------------------------------------------------------------------
# Streamed summaries: λ = 1 exactness and the replay identity
# ---------------------------------------------------------------------------

def test_d_k_streamed_equals_from_scratch_at_lambda_one():
    """Eq. 16 with λ = 1: D_k = U_kᵀU_k over every stored row (Eq. 14)."""
    s = PlantedStream(tiny(K0=5, J=7, R=3, steps=4, sigma=0.05, lam=1.0))
    ost = O.OracleStream("P", RNG.random((7, 3)), 1.0)
    for t in range(5):
        b = s.batch(t)
        ost.update(_segs(b), b.n_new)
    for k in range(ost.state.K):
        _, Uk, _ = ost.slice_rows(k)
        assert _rel(ost.state.D[k], Uk.T @ Uk) < 1e-12


def test_replay_identity_for_c_f_g():
    """Eqs. 15, 20, 21 unrolled: c_k = Σ_t λ^(T-t) vec(X_t)ᵀ(V^(t) ⊙ U_t),
    F = Σ_t λ^(T-t) X_tᵀU_t S^(t), G = Σ_t λ^(T-t) S^(t)U_tᵀU_t S^(t), where
    V^(t) is V at the start of update t and S^(t) the S_k of update t's W step."""
    lam = 0.7
    s = PlantedStream(tiny(K0=3, J=5, R=2, steps=3, sigma=0.05, lam=lam))
    ost = O.OracleStream("P", RNG.random((5, 2)), lam)
    hist = []
    for t in range(4):
        b = s.batch(t)
        V_before = ost.state.V.copy()
        U = ost.update(_segs(b), b.n_new)
        hist.append((V_before, ost.state.W.copy(), dict(ost.last_X), dict(U)))
    T = len(hist)
    K = ost.state.K
    c = np.zeros((K, 2)); F = np.zeros((5, 2)); G = np.zeros((2, 2))
    for t, (Vb, Wt, Xt, Ut) in enumerate(hist):
        a = lam ** (T - 1 - t)
        for k, Xk in Xt.items():
            c[k] += a * O.c_term(Xk, Vb, Ut[k])
            S = np.diag(Wt[k])
            F += a * Xk.T @ Ut[k] @ S
            G += a * S @ Ut[k].T @ Ut[k] @ S
    assert _rel(ost.state.c, c) < 1e-12
    assert _rel(ost.state.F, F) < 1e-12
    assert _rel(ost.state.G, G) < 1e-12


# ---------------------------------------------------------------------------
# Single batch ≡ static ALS, noiseless recovery, closed forms
# ---------------------------------------------------------------------------

def test_single_batch_equals_static_als_iteration():
    s = PlantedStream(tiny(K0=6, J=7, R=3, steps=0, sigma=0.02))
    b = s.batch(0)
    X = [x.numpy() for _, x in b.segments()]
    V0 = RNG.random((7, 3))
    st, U = O.dash_update_p(O.empty_state_p(V0), _segs(b), b.n_new, 1.0)
    U1, W1, V1 = O.static_als_p(X, V0, np.ones((6, 3)), 1)
    assert _rel(st.V, V1) < 1e-10
    assert _rel(st.W, W1) < 1e-10
    for k in range(6):
        assert _rel(U[k], U1[k]) < 1e-10
    # two sweeps on an empty model = two static iterations
    st2, _ = O.dash_update_p(O.empty_state_p(V0), _segs(b), b.n_new, 1.0, n_sweeps=2)
    _, W2, V2 = O.static_als_p(X, V0, np.ones((6, 3)), 2)
    assert _rel(st2.V, V2) < 1e-9 and _rel(st2.W, W2) < 1e-9


def test_noiseless_planted_recovery_mode_p():
    """σ = 0: static ALS reaches fitness 1 within 1e-9, and a Dash stream
    started from it keeps every batch's fitness within 1e-9 of 1."""
    s = PlantedStream(tiny(K0=6, J=8, R=3, steps=3, sigma=0.0))
    b = s.batch(0)
    X = [x.numpy() for _, x in b.segments()]
    V0 = RNG.random((8, 3))
    U, W, V = O.static_als_p(X, V0, np.ones((6, 3)), 6)
    fit = O.fitness(X, [O.reconstruct_p(U[k], W[k], V) for k in range(6)])
    assert fit > 1 - 1e-9
    st = O.init_helpers_p(X, U, W, V)
    for t in range(1, 4):
        bt = s.batch(t)
        st, Un = O.dash_update_p(st, _segs(bt), bt.n_new, 1.0)
        Xn = [x.numpy() for _, x in bt.segments()]
        ks = bt.slice_ids.tolist()
        fit = O.fitness(Xn, [O.reconstruct_p(Un[k], st.W[k], st.V) for k in ks])
        assert fit > 1 - 1e-9


def test_rank_one_update_is_a_power_iteration_step():
    """R = 1 closed form of Lemmas 1-3 on an empty model (derived by hand):
    U_k = X_k v / (w_k ||v||²); c_k = ||X_k v||² / (w_k ||v||²);
    D_k = ||X_k v||² / (w_k² ||v||⁴); hence w_k,new = w_k;
    F = C v / ||v||², G = vᵀ C v / ||v||⁴ with C = Σ X_kᵀX_k; so
    v_new = ||v||² C v / (vᵀ C v): a power-iteration step on C."""
    X = [RNG.standard_normal((n, 5)) for n in (3, 6, 4)]
    C = sum(x.T @ x for x in X)
    v = RNG.random((5, 1))
    st = O.empty_state_p(v)
    st, U = O.dash_update_p(st, list(enumerate(X)), 3, 1.0)
    nv = float((v.T @ v).item())
    want = nv * (C @ v) / float((v.T @ C @ v).item())
    assert _rel(st.V, want) < 1e-12
    assert _rel(st.W, np.ones((3, 1))) < 1e-12
    for k in range(3):
        assert _rel(U[k], X[k] @ v / nv) < 1e-12
    # iterating converges to the dominant eigenvector of C (eigh)
    for _ in range(300):
        st, _ = O.dash_update_p(O.empty_state_p(st.V), list(enumerate(X)), 3, 1.0)
    e = np.linalg.eigh(C)[1][:, -1:]
    u = st.V / np.linalg.norm(st.V)
    assert min(_rel(u, e), _rel(u, -e)) < 1e-8


def test_worked_example_rank_one_exact_fractions():
    """A two-update worked example carried out by hand in exact rationals
    with the R = 1 closed forms (Lemmas 1-3, Eqs. 15-16, 20-21).

    Update 1 (empty model, λ = 1): X = [[1,2],[3,4]], v = (1,1), w = 1:
      Xv = (3,7), U = (3/2, 7/2), c = 29, D = 29/2, w = 29/(2·29/2) = 1,
      F = XᵀU = (12, 17), G = 29/2, v = (24/29, 34/29).
    Update 2 (λ = 1/2): one new row x = (1, 0) for the same slice:
      ||v||² = 1732/841, xv = 24/29, U = (24/29)/(1732/841) = 174/433,
      c = 29/2 + (174/433)(24/29) = 29/2 + 144/433,
      D = 29/4 + (174/433)², w = c / (||v||² D),
      F = (1/2)(12,17) + x·U·w, G = (1/2)(29/2) + w² U², v = F/G.
    """
    Fr = Fraction
    X1 = np.array([[1.0, 2.0], [3.0, 4.0]])
    st = O.empty_state_p(np.array([[1.0], [1.0]]))
    st, U = O.dash_update_p(st, [(0, X1)], 1, 1.0)
    assert _rel(U[0].ravel(), [1.5, 3.5]) < 1e-15
    assert _rel(st.c, [[29.0]]) < 1e-15 and _rel(st.D, [[[14.5]]]) < 1e-15
    assert _rel(st.W, [[1.0]]) < 1e-15
    assert _rel(st.F.ravel(), [12.0, 17.0]) < 1e-15 and _rel(st.G, [[14.5]]) < 1e-15
    assert _rel(st.V.ravel(), [24 / 29, 34 / 29]) < 1e-15
    # update 2, exact rationals
    v = [Fr(24, 29), Fr(34, 29)]
    nv = v[0] ** 2 + v[1] ** 2
    assert nv == Fr(1732, 841)
    xv = v[0]
    u = xv / nv
    assert u == Fr(174, 433)
    c = Fr(29, 2) + u * xv
    D = Fr(29, 4) + u * u
    w = c / (nv * D)
    F = [Fr(6) + 1 * u * w, Fr(17, 2) + 0]
    G = Fr(29, 4) + w * w * u * u
    vnew = [f / G for f in F]
    st, U = O.dash_update_p(st, [(0, np.array([[1.0, 0.0]]))], 0, 0.5)
    assert _rel(U[0], [[float(u)]]) < 1e-14
    assert _rel(st.c, [[float(c)]]) < 1e-14
    assert _rel(st.D, [[[float(D)]]]) < 1e-14
    assert _rel(st.W, [[float(w)]]) < 1e-14
    assert _rel(st.V.ravel(), [float(x) for x in vnew]) < 1e-13


# ---------------------------------------------------------------------------
# Edge cases of the update
# ---------------------------------------------------------------------------

def test_untouched_slice_decays_and_keeps_w_direction():
    """A slice with no new rows: c, D scale by λ (Eqs. 15-16 over all k);
    λ cancels in Eq. 12, so its W row is re-solved with the new VᵀV only."""
    lam = 0.5
    s = PlantedStream(tiny(K0=3, J=5, R=2, steps=0, sigma=0.05))
    b = s.batch(0)
    st, _ = O.dash_update_p(O.empty_state_p(RNG.random((5, 2))), _segs(b), 3, 1.0)
    nb = ragged_batch(3, 0, 5, [4], seed=3, slice_ids=[1])
    st2, _ = O.dash_update_p(st, _segs(nb), 0, lam)
    for k in (0, 2):
        assert _rel(st2.c[k], lam * st.c[k]) < 1e-15
        assert _rel(st2.D[k], lam * st.D[k]) < 1e-15
        assert _rel(st2.W[k], O.solve_w_row(st.c[k], st.D[k], st.V)) < 1e-12


def test_new_empty_slice_gets_zero_weights():
    s = PlantedStream(tiny(K0=3, J=5, R=2, steps=0, sigma=0.05))
    b = s.batch(0)
    st, _ = O.dash_update_p(O.empty_state_p(RNG.random((5, 2))), _segs(b), 3, 1.0)
    nb = ragged_batch(3, 2, 5, [0, 3], seed=4, slice_ids=[3, 4])
    st2, U = O.dash_update_p(st, _segs(nb), 2, 1.0)
    assert st2.K == 5
    assert np.all(st2.W[3] == 0) and np.all(st2.c[3] == 0) and np.all(st2.D[3] == 0)
    assert U[3].shape == (0, 2)
    assert np.all(np.isfinite(st2.V))


def test_split_segments_equal_one_segment():
    """Two segments of the same slice in one batch are its rows in order."""
    s = PlantedStream(tiny(K0=3, J=5, R=2, steps=0, sigma=0.05))
    b = s.batch(0)
    st, _ = O.dash_update_p(O.empty_state_p(RNG.random((5, 2))), _segs(b), 3, 1.0)
    X = RNG.standard_normal((5, 5))
    a, _ = O.dash_update_p(st, [(1, X[:2]), (1, X[2:])], 0, 0.9)
    c, _ = O.dash_update_p(st, [(1, X)], 0, 0.9)
    assert _rel(a.V, c.V) < 1e-14 and _rel(a.W, c.W) < 1e-14


# ---------------------------------------------------------------------------
# Mode Q (constrained U_k = Q_k H S_k)
# ---------------------------------------------------------------------------

def test_mode_q_single_batch_equals_parafac2_als_iteration():
    s = PlantedStream(tiny(K0=6, J=7, R=3, steps=0, sigma=0.02,
                           init_rows=("uniform", 6, 12)))
    b = s.batch(0)
    X = [x.numpy() for _, x in b.segments()]
    V0 = RNG.random((7, 3))
    st, Qn, _ = O.dash_update_q(O.empty_state_q(V0), _segs(b), b.n_new, 1.0)
    Q1, H1, V1, W1 = O.parafac2_als(X, np.eye(3), V0, np.ones((6, 3)), 1)
    assert _rel(st.H, H1) < 1e-9 and _rel(st.V, V1) < 1e-9 and _rel(st.W, W1) < 1e-9
    for k in range(6):
        assert _rel(Qn[k], Q1[k]) < 1e-7


@pytest.mark.parametrize("lam", [1.0, 0.8])
def test_mode_q_summaries_exact_and_q_orthonormal(lam):
    """L_kᵀL_k = B_k and Z_k equal the λ-weighted sums over stored A rows
    (exact at any λ: A rows are frozen), L_k is the Cholesky factor of that
    sum, and Q_k = Ã_k T_k satisfies Q_kᵀΛQ_k = I when B_k has full rank
    (QᵀQ = I at λ = 1)."""
    s = PlantedStream(tiny(K0=4, J=6, R=3, steps=3, sigma=0.05, lam=lam,
                           init_rows=("uniform", 5, 9)))
    ost = O.OracleStream("Q", RNG.random((6, 3)), lam)
    for t in range(4):
        b = s.batch(t)
        ost.update(_segs(b), b.n_new)
    for k in range(ost.state.K):
        Xk, Ak, wts = ost.slice_rows(k)
        B = (Ak * wts[:, None]).T @ Ak
        Z = (Ak * wts[:, None]).T @ Xk
        L = ost.state.L[k]
        assert np.all(np.tril(L, -1) == 0) and np.all(np.diag(L) >= 0)
        assert _rel(L.T @ L, B) < 1e-12
        assert _rel(ost.state.Z[k], Z) < 1e-12
        if Ak.shape[0] >= 3:
            # the unique triangular square root: Cholesky of the from-scratch B
            assert _rel(L, np.linalg.cholesky(B).T) < 1e-9
            T = O.inv_sqrt_from_factor(L)
            Q = Ak @ T
            assert _rel((Q * wts[:, None]).T @ Q, np.eye(3)) < 1e-8


def test_mode_q_planted_truth_is_a_fixed_point():
    """A noiseless, fully revealed planted tensor: one PARAFAC2-ALS iteration
    (= one Mode Q update on an empty model) from the planted factors keeps
    fitness at 1 to round-off."""
    s = PlantedStream(tiny(K0=8, J=7, R=3, steps=0, sigma=0.0,
                           init_rows=("uniform", 6, 12)))
    b = s.batch(0)
    X = [x.numpy() for _, x in b.segments()]
    st, Qn, _ = O.dash_update_q(O.empty_state_q(s.V.numpy(), s.H.numpy()),
                                _segs(b), b.n_new, 1.0)
    # W of new slices starts at 1, so seed them with the planted weights
    st0 = O.StateQ(V=s.V.numpy(), H=s.H.numpy(), W=s.W.numpy()[:8],
                   L=np.zeros((8, 3, 3)), Z=np.zeros((8, 3, 7)))
    st1, Qn, _ = O.dash_update_q(st0, _segs(b), 0, 1.0)
    fit = O.fitness(X, [O.reconstruct_q(Qn[k], st1.H, st1.W[k], st1.V) for k in range(8)])
    # the streamed form sees A only through its R factor L, so Q is accurate
    # to about eps·cond(L) = eps·cond(A); the SVD form of PARAFAC2-ALS to round-off
    kappa = max(np.linalg.cond(st1.L[k]) for k in range(8))
    assert 1 - fit < 10 * O.EPS * kappa
    Q, H, V, W = O.parafac2_als(X, s.H.numpy(), s.V.numpy(), s.W.numpy()[:8], 1)
    fit_svd = O.fitness(X, [O.reconstruct_q(Q[k], H, W[k], V) for k in range(8)])
    assert fit_svd > 1 - 1e-12


def test_mode_q_noiseless_recovery_from_seeded_start():
    """Well-conditioned noiseless planted PARAFAC2 (orthonormal V, H; W in
    [0.5, 1.5]), fully revealed: PARAFAC2-ALS from this seeded start reaches
    fitness 1 within 1e-9 (ALS converges linearly; this start is in the
    basin of the planted solution)."""
    K0, J, R = 30, 8, 3
    s = PlantedStream(tiny(K0=K0, J=J, R=R, steps=0, sigma=0.0,
                           init_rows=("uniform", 6, 12)))
    g = torch.Generator().manual_seed(5)
    s.V = torch.linalg.qr(torch.randn(J, R, generator=g, dtype=torch.float64))[0] * 3
    s.H = torch.linalg.qr(torch.randn(R, R, generator=g, dtype=torch.float64))[0]
    s.W = 0.5 + torch.rand(s.W.shape, generator=g, dtype=torch.float64)
    b = s.batch(0)
    X = [x.numpy() for _, x in b.segments()]
    rng = np.random.default_rng(1)
    Vt, Ht, Wt = s.V.numpy(), s.H.numpy(), s.W.numpy()[:K0]
    V0 = Vt + 0.5 * rng.standard_normal(Vt.shape)
    H0 = Ht + 0.5 * rng.standard_normal(Ht.shape)
    W0 = Wt + 0.5 * rng.standard_normal(Wt.shape)
    Q, H, V, W = O.parafac2_als(X, H0, V0, W0, 250)
    fit = O.fitness(X, [O.reconstruct_q(Q[k], H, W[k], V) for k in range(K0)])
    assert fit > 1 - 1e-9
    # the streaming form run as repeated single-batch updates agrees
    st = O.StateQ(V=V0, H=H0, W=W0, L=np.zeros((K0, R, R)), Z=np.zeros((K0, R, J)))
    for _ in range(250):
        st, Qn, _ = O.dash_update_q(st, _segs(b), 0, 0.0)
    fit2 = O.fitness(X, [O.reconstruct_q(Qn[k], st.H, st.W[k], st.V) for k in range(K0)])
    assert fit2 > 1 - 1e-9


def test_mode_q_cp_sweep_is_monotone():
    """Each PARAFAC2-ALS iteration does not increase the loss."""
    s = PlantedStream(tiny(K0=8, J=7, R=3, steps=0, sigma=0.1,
                           init_rows=("uniform", 6, 12)))
    b = s.batch(0)
    X = [x.numpy() for _, x in b.segments()]
    H, V, W = np.eye(3), RNG.random((7, 3)), np.ones((8, 3))
    prev = np.inf
    for _ in range(20):
        Q, H, V, W = O.parafac2_als(X, H, V, W, 1)
        loss = sum(np.sum((X[k] - O.reconstruct_q(Q[k], H, W[k], V)) ** 2) for k in range(8))
        assert loss <= prev * (1 + 1e-12)
        prev = loss


# ---------------------------------------------------------------------------
# Errors of §3.4 and §4.1
# ---------------------------------------------------------------------------

def test_slice_and_tensor_errors_by_hand():
    """Definitions 1-2: se = mean |X - X̂| per slice; te = mean of se."""
    a = np.array([[1.0, 2.0], [3.0, 4.0]])
    ah = np.array([[1.5, 2.0], [3.0, 3.0]])       # |diff| sum 1.5 over 4
    b = np.array([[0.0, 1.0, 2.0]])
    bh = np.array([[0.0, 0.0, 0.0]])              # sum 3 over 3
    assert O.slice_error(a, ah) == 0.375
    assert O.slice_error(b, bh) == 1.0
    assert O.tensor_error([a, b], [ah, bh]) == (0.375 + 1.0) / 2
    assert O.fitness([a], [a]) == 1.0
    assert abs(O.fitness([a], [np.zeros_like(a)])) < 1e-15


def test_fitness_takes_the_root_of_the_pooled_residual_ratio():
    """fit = 1 - ||X - X̂||_F / ||X||_F worked by hand.  X = [[3, 4]] against
    X̂ = [[3, 0]] leaves a residual of norm 4 against ||X||_F = 5: fit = 0.2
    (the squared ratio would give 0.36).  Over several matrices the squared
    sums pool before the root: residual² 4 + 0 over ||X||² 9 + 16 gives
    1 - 2/5 = 0.6 (the mean of per-matrix fits would give 2/3)."""
    assert abs(O.fitness([np.array([[3.0, 4.0]])], [np.array([[3.0, 0.0]])]) - 0.2) < 1e-15
    X = [np.array([[1.0, 2.0], [2.0, 0.0]]), np.array([[0.0, 4.0]])]
    Xh = [np.array([[1.0, 2.0], [0.0, 0.0]]), np.array([[0.0, 4.0]])]
    assert abs(O.fitness(X, Xh) - 0.6) < 1e-15


def test_init_helpers_q_follow_their_definition():
    """Constrained-mode helpers of an initial tensor (the Q_k H S_k form of
    §2.1, helpers as in Eqs. 6-9): with A_k = X_k V S_k Hᵀ formed entry by
    entry, L_k is upper triangular with a non-negative diagonal and
    L_kᵀL_k = A_kᵀA_k, i.e. L_k is the transposed Cholesky factor of A_kᵀA_k;
    and Z_k = A_kᵀX_k entry by entry.  Weights away from 1 keep S_k visible."""
    rng = np.random.default_rng(7)
    J, R = 5, 3
    X = [rng.standard_normal((n, J)) for n in (7, 4, 3)]    # I_k = R included
    V = rng.random((J, R))
    H = rng.random((R, R))
    W = rng.random((3, R)) + 0.5
    st = O.init_helpers_q(X, H, V, W)
    for k, Xk in enumerate(X):
        I = Xk.shape[0]
        A = np.zeros((I, R))
        for i in range(I):
            for r in range(R):
                A[i, r] = sum(Xk[i, j] * V[j, s] * W[k, s] * H[r, s]
                              for j in range(J) for s in range(R))
        Z = np.zeros((R, J))
        for r in range(R):
            for j in range(J):
                Z[r, j] = sum(A[i, r] * Xk[i, j] for i in range(I))
        L = st.L[k]
        assert np.all(np.tril(L, -1) == 0.0)
        assert np.all(np.diag(L) >= 0.0)
        assert _rel(L.T @ L, A.T @ A) < 1e-12
        assert _rel(L, np.linalg.cholesky(A.T @ A).T) < 1e-10
        assert _rel(st.Z[k], Z) < 1e-13


def test_weighted_fitness_by_hand_and_as_a_batch_fitness():
    """The λ-weighted fitness: a hand case (ages 0 and 1, λ = 1/4) and the
    single-batch special case, where it is the batch fitness."""
    V = np.eye(2)
    rows = [(0, np.array([[3.0, 4.0]]), np.array([[3.0, 0.0]]), np.array([1.0, 1.0])),
            (1, np.array([[0.0, 2.0]]), np.array([[0.0, 1.0]]), np.array([1.0, 2.0]))]
    # residuals 16 (age 0) and 0; norms 25 + 4/4
    assert abs(O.weighted_fitness_p(rows, V, 0.25) - (1.0 - np.sqrt(16.0 / 26.0))) < 1e-15
    X = RNG.standard_normal((6, 4))
    U = RNG.standard_normal((6, 2))
    w = RNG.random(2) + 0.5
    Vr = RNG.standard_normal((4, 2))
    assert abs(O.weighted_fitness_p([(0, X, U, w)], Vr, 0.7)
               - O.fitness([X], [O.reconstruct_p(U, w, Vr)])) < 1e-14


@pytest.mark.parametrize("lam", [1.0, 0.8])
def test_weighted_fitness_equals_the_helper_form(lam):
    """Over a stream, Σ λ^age ||x − (u∘w)Vᵀ||² computed from every stored row
    equals xx − 2 tr(VᵀF) + tr(VᵀV G) from the streamed helpers (Eqs. 20-21),
    xx = Σ λ^age ||x||²: the form the library evaluates."""
    w = tiny(K0=6, J=7, R=3, steps=3, sigma=0.05, lam=lam, new=2)
    s = PlantedStream(w)
    ost = O.OracleStream("P", RNG.random((w.J, w.R)), lam)
    for t in range(4):
        b = s.batch(t)
        ost.update(_segs(b), b.n_new)
    st = ost.state
    T = ost.t
    rows = [(T - 1 - p[0], p[1], p[2], p[3]) for parts in ost.rows for p in parts]
    num = sum(lam ** a * np.sum((X - O.reconstruct_p(U, wv, st.V)) ** 2) for a, X, U, wv in rows)
    xx = sum(lam ** a * np.sum(X ** 2) for a, X, _, _ in rows)
    helper = xx - 2.0 * np.sum(st.V * st.F) + np.sum((st.V.T @ st.V) * st.G)
    assert abs(num - helper) <= 1e-10 * xx
    assert abs(O.weighted_fitness_p(rows, st.V, lam) - (1.0 - np.sqrt(helper / xx))) < 1e-8
