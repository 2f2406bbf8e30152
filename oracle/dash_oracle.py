"""FP64 CPU oracle for Dash, the dual-way streaming PARAFAC2 update
(Jang, Jang and Kang, KDD'23).  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
legs may import this module.  The CUDA library never calls it and it never
calls the library; the two share nothing but the seeded input generator in
synth/.  Everything here is plain numpy float64, slow and literal: one
slice at a time, each step in the paper's order and notation.

Conventions
  * vec() is column-major; the Khatri–Rao product A ⊙ B has column r equal
    to kron(A[:, r], B[:, r])  (Table 1).
  * "⁻¹" in Eqs. 11, 12 and 17 is read as the Moore–Penrose pseudo-inverse,
    computed by SVD with singular values at or below rtol·σ_max treated as
    zero (rtol defaults to n·eps for an n×n matrix).
  * A new slice has no S_k before its first W step; Lemma 1 is then applied
    with S_k = I (w_k = 1).
  * λ multiplies every old term once per update, including slices that got
    no new rows (Eqs. 15, 16, 20, 21 run over all k).

Mode "P" is Algorithm 1 as written (U_k free, §2.1 / §3).  Mode "Q" applies
the same divide-and-compute discipline to the constrained model
U_k = Q_k H S_k with column-orthonormal Q_k (the reparameterisation §2.1
mentions and Dash drops):
  A_new = X_new V S_k Hᵀ,  B_k ← λB_k + A_newᵀA_new,  Z_k ← λZ_k + A_newᵀX_new,
  T_k = B_k^{-1/2} (pseudo-inverse square root),  Q_k,new = A_new T_k,
  Y_k = T_k Z_k  (= Q_kᵀ Λ_k X_k),  then one CP-ALS sweep H → V → W on {Y_k}.
With one batch and an empty model this is one classic PARAFAC2-ALS iteration.
B_k is carried as its triangular square root L_k (B_k = L_kᵀL_k, L_k the R
factor of the λ^{age/2}-weighted stacked A rows), updated by a QR of
[√λ L_k; A_new], and T_k comes from the SVD of L_k: forming B_k itself
squares cond(A_k), and on planted tensors with U(0,1) factors cond(B_k)
reaches 1e9-1e12, where any B-based T_k loses 7-12 digits.

Parity pins (tests/test_oracle_*.py): Lemma 1–3 optimality against direct
least squares, the Khatri–Rao identity of Appendix A.2, λ = 1 exactness of
the streamed summaries, the replay identity for c_k, F, G, single-batch
equality with static ALS written independently, noiseless planted recovery,
the R = 1 reduction to a power iteration, orthonormal Q_k, a two-update
worked example carried out by hand in exact fractions, the fitness's root
on a hand value, and the constrained-mode initial helpers against their
entry-by-entry definition.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------------------
# Linear-algebra readings
# ---------------------------------------------------------------------------

def pinv(A: np.ndarray, rtol: Optional[float] = None) -> np.ndarray:
    """Moore–Penrose pseudo-inverse by SVD: the reading of the '⁻¹' in
    Eqs. 11, 12 and 17 (the paper writes an inverse and is silent on
    singular cases).  Singular values <= rtol·σ_max count as zero."""
    A = np.asarray(A, dtype=np.float64)
    if A.size == 0:
        return np.zeros(A.T.shape)
    u, s, vt = np.linalg.svd(A)
    if rtol is None:
        rtol = max(A.shape) * EPS
    if s.size == 0 or s[0] == 0.0:
        return np.zeros(A.T.shape)
    keep = s > rtol * s[0]
    sinv = np.zeros_like(s)
    sinv[keep] = 1.0 / s[keep]
    return (vt.T * sinv) @ u.T


def inv_sqrt_psd(B: np.ndarray, rtol: Optional[float] = None) -> np.ndarray:
    """T = B^{-1/2} of a symmetric PSD matrix, pseudo-inverse sense: the
    eigenvalues <= rtol·μ_max are dropped.  Q_k = A_k T_k is then the polar
    (Procrustes) factor of A_k."""
    B = 0.5 * (B + B.T)
    mu, E = np.linalg.eigh(B)
    if rtol is None:
        rtol = B.shape[0] * EPS
    top = mu.max() if mu.size else 0.0
    if top <= 0.0:
        return np.zeros_like(B)
    keep = mu > rtol * top
    d = np.zeros_like(mu)
    d[keep] = 1.0 / np.sqrt(mu[keep])
    return (E * d) @ E.T


def r_factor(M: np.ndarray) -> np.ndarray:
    """The R factor of a thin QR of M (rows ≥ 0), as an R×R upper-triangular
    matrix with a non-negative diagonal (zero rows appended when M has fewer
    rows than columns).  It is the unique square root of MᵀM of that shape
    when M has full column rank."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[1]
    out = np.zeros((n, n))
    if M.shape[0] == 0:
        return out
    Rf = np.linalg.qr(M, mode="r")
    sgn = np.where(np.diag(Rf) < 0.0, -1.0, 1.0)
    Rf = Rf * sgn[:, None]
    out[:Rf.shape[0]] = Rf
    return out


def inv_sqrt_from_factor(L: np.ndarray, rtol: Optional[float] = None) -> np.ndarray:
    """T = (LᵀL)^{-1/2} in the pseudo-inverse sense from the SVD
    L = U diag(σ) Pᵀ: T = P diag(1/σ) Pᵀ, with the directions whose
    eigenvalue σ² of LᵀL is <= rtol·σ_max² dropped (the cut of
    inv_sqrt_psd applied to B = LᵀL).  Works on L, whose condition number
    is the square root of B's."""
    L = np.asarray(L, dtype=np.float64)
    n = L.shape[1]
    if rtol is None:
        rtol = n * EPS
    _, sig, Pt = np.linalg.svd(L)
    if sig.size == 0 or sig[0] == 0.0:
        return np.zeros((n, n))
    keep = sig * sig > rtol * sig[0] * sig[0]
    d = np.zeros_like(sig)
    d[keep] = 1.0 / sig[keep]
    return (Pt.T * d) @ Pt


def vec(X: np.ndarray) -> np.ndarray:
    """Column-major vectorisation vec(·) (Table 1)."""
    return np.asarray(X).reshape(-1, order="F")


def khatri_rao(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A ⊙ B: column r is kron(A[:, r], B[:, r]) (Table 1)."""
    I, R = B.shape
    J = A.shape[0]
    out = np.empty((J * I, R))
    for r in range(R):
        out[:, r] = np.kron(A[:, r], B[:, r])
    return out


# ---------------------------------------------------------------------------
# Mode P: the paper's Dash (Algorithm 1, Lemmas 1-3)
# ---------------------------------------------------------------------------

def update_u_new(X_new: np.ndarray, V: np.ndarray, w: np.ndarray,
                 rtol: Optional[float] = None) -> np.ndarray:
    """Lemma 1, Eq. 11: U_k,new = X_k,new V S_k (S_k Vᵀ V S_k)⁻¹."""
    S = np.diag(w)
    return X_new @ V @ S @ pinv(S @ V.T @ V @ S, rtol)


def c_term(X: np.ndarray, V: np.ndarray, U: np.ndarray) -> np.ndarray:
    """vec(X)ᵀ (V ⊙ U), the data term of c_k (Eqs. 6, 13, 15)."""
    if X.shape[0] == 0:
        return np.zeros(V.shape[1])
    return vec(X) @ khatri_rao(V, U)


def solve_w_row(c: np.ndarray, D: np.ndarray, V: np.ndarray,
                rtol: Optional[float] = None) -> np.ndarray:
    """Lemma 2, Eq. 12: W(k,:) = c_kᵀ (VᵀV ∗ D_k)⁻¹."""
    return c @ pinv((V.T @ V) * D, rtol)


@dataclasses.dataclass
class StateP:
    """Factors and helper matrices of Algorithm 1 (inputs/outputs list)."""
    V: np.ndarray          # J×R
    W: np.ndarray          # K×R, row k = diagonal of S_k
    c: np.ndarray          # K×R
    D: np.ndarray          # K×R×R
    F: np.ndarray          # J×R
    G: np.ndarray          # R×R

    @property
    def K(self) -> int:
        return self.W.shape[0]

    def copy(self) -> "StateP":
        return StateP(*(np.array(getattr(self, f.name)) for f in dataclasses.fields(self)))


def empty_state_p(V0: np.ndarray) -> StateP:
    """A model with no slices yet: zero helpers, the given V."""
    J, R = V0.shape
    return StateP(V=np.array(V0, dtype=np.float64), W=np.zeros((0, R)),
                  c=np.zeros((0, R)), D=np.zeros((0, R, R)),
                  F=np.zeros((J, R)), G=np.zeros((R, R)))


def _group(segments, K_before: int, n_new: int, J: int) -> Dict[int, np.ndarray]:
    """Concatenate a batch's segments per slice, in arrival order.  New slice
    ids must be K_before .. K_before+n_new-1."""
    by: Dict[int, List[np.ndarray]] = {}
    for k, X in segments:
        k = int(k)
        if not (0 <= k < K_before + n_new):
            raise ValueError(f"slice id {k} outside 0..{K_before + n_new - 1}")
        by.setdefault(k, []).append(np.asarray(X, dtype=np.float64).reshape(-1, J))
    return {k: np.concatenate(v, axis=0) for k, v in by.items()}


def dash_update_p(state: StateP, segments, n_new: int, lam: float,
                  n_sweeps: int = 1, rtol: Optional[float] = None,
                  freeze_V: bool = False, freeze_W: bool = False
                  ) -> Tuple[StateP, Dict[int, np.ndarray]]:
    """One update of Algorithm 1 for the new tensor {X_k,new}, k = 1..K+L.

    segments: iterable of (k, X_k,new) pairs (0-based k; k >= K are the L =
    n_new new slices).  Returns the new state and U_k,new per touched slice.

    Order (Algorithm 1): U_k,new for all k with the old V and S_k (Eq. 11);
    then for every k: c_k, D_k (Eqs. 15, 16) and W(k,:) (Eq. 12); then F, G
    (Eqs. 20, 21) with the new S_k; then V = F G⁻¹ (Eq. 17).  For
    n_sweeps > 1 the whole sequence is repeated with the old helpers held
    fixed and the new terms recomputed from the latest factors.

    freeze_V / freeze_W are test modes that skip the V (resp. W) step, so
    that the streamed helpers can be compared with a from-scratch recompute.
    """
    J, R = state.V.shape
    K = state.K
    Kn = K + n_new
    X = _group(segments, K, n_new, J)
    old = state
    W = np.vstack([old.W, np.ones((n_new, R))])   # S_k := I for new slices
    V = old.V.copy()
    c_old = np.vstack([old.c, np.zeros((n_new, R))])
    D_old = np.concatenate([old.D, np.zeros((n_new, R, R))], axis=0)
    U: Dict[int, np.ndarray] = {}
    for _ in range(max(1, n_sweeps)):
        # loop 1: U_k,new for every slice with new rows (Eq. 11)
        U = {k: update_u_new(Xk, V, W[k], rtol) for k, Xk in X.items()}
        # loop 2: c_k, D_k (Eqs. 15, 16) then W(k,:) (Eq. 12), all k
        c = lam * c_old
        D = lam * D_old
        for k in range(Kn):
            if k in X:
                c[k] = c[k] + c_term(X[k], V, U[k])
                D[k] = D[k] + U[k].T @ U[k]
            if not freeze_W:
                W[k] = solve_w_row(c[k], D[k], V, rtol)
        # F, G with the new S_k (Eqs. 20, 21), then V (Eq. 17)
        F = lam * old.F
        G = lam * old.G
        for k, Xk in X.items():
            S = np.diag(W[k])
            F = F + Xk.T @ U[k] @ S
            G = G + S @ U[k].T @ U[k] @ S
        if not freeze_V:
            V = F @ pinv(G, rtol)
    return StateP(V=V, W=W, c=c, D=D, F=F, G=G), U


def init_helpers_p(X: Sequence[np.ndarray], U: Sequence[np.ndarray],
                   W: np.ndarray, V: np.ndarray) -> StateP:
    """§3.2.1, Eqs. 6-9: helpers of the initial tensor from its factors."""
    K = len(X)
    J, R = V.shape
    c = np.zeros((K, R))
    D = np.zeros((K, R, R))
    F = np.zeros((J, R))
    G = np.zeros((R, R))
    for k in range(K):
        S = np.diag(W[k])
        c[k] = c_term(X[k], V, U[k])                 # Eq. 6
        D[k] = U[k].T @ U[k]                         # Eq. 7
        F = F + X[k].T @ U[k] @ S                    # Eq. 8
        G = G + S @ U[k].T @ U[k] @ S                # Eq. 9
    return StateP(V=np.array(V), W=np.array(W), c=c, D=D, F=F, G=G)


def static_als_p(X: Sequence[np.ndarray], V0: np.ndarray, W0: np.ndarray,
                 n_iter: int) -> Tuple[List[np.ndarray], np.ndarray, np.ndarray]:
    """Static ALS for Eq. 1 with free U_k, written as direct least squares
    (numpy lstsq) rather than normal equations.  Block order per iteration:
    every U_k, then every row of W, then V.  Used for initialisation (§3.2.1
    with our own static fit in place of SPARTan) and as an independent check
    of the update rules."""
    V = np.array(V0, dtype=np.float64)
    W = np.array(W0, dtype=np.float64)
    K = len(X)
    U: List[np.ndarray] = []
    for _ in range(n_iter):
        # U_k minimises ||X_k - U_k S_k Vᵀ||: U_kᵀ = argmin ||(V S_k) U_kᵀ - X_kᵀ||
        U = [np.linalg.lstsq(V * W[k], X[k].T, rcond=None)[0].T for k in range(K)]
        # W(k,:) minimises ||vec(X_k) - (V ⊙ U_k) W(k,:)ᵀ||
        for k in range(K):
            W[k] = np.linalg.lstsq(khatri_rao(V, U[k]), vec(X[k]), rcond=None)[0]
        # V minimises sum_k ||X_k - (U_k S_k) Vᵀ||: stack the slices
        M = np.vstack([U[k] * W[k] for k in range(K)])
        Xs = np.vstack(X)
        V = np.linalg.lstsq(M, Xs, rcond=None)[0].T
    return U, W, V


# ---------------------------------------------------------------------------
# Mode Q: the constrained model U_k = Q_k H S_k, same streaming discipline
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class StateQ:
    V: np.ndarray          # J×R
    H: np.ndarray          # R×R
    W: np.ndarray          # K×R
    L: np.ndarray          # K×R×R   upper-triangular, L_kᵀL_k = B_k = λ-weighted Σ A_kᵀA_k
    Z: np.ndarray          # K×R×J   λ-weighted Σ A_kᵀX_k

    @property
    def K(self) -> int:
        return self.W.shape[0]

    @property
    def B(self) -> np.ndarray:
        """B_k = L_kᵀL_k (formed only for inspection)."""
        return np.einsum("kij,kil->kjl", self.L, self.L)

    def copy(self) -> "StateQ":
        return StateQ(*(np.array(getattr(self, f.name)) for f in dataclasses.fields(self)))


def empty_state_q(V0: np.ndarray, H0: Optional[np.ndarray] = None) -> StateQ:
    J, R = V0.shape
    H = np.eye(R) if H0 is None else np.array(H0, dtype=np.float64)
    return StateQ(V=np.array(V0, dtype=np.float64), H=H, W=np.zeros((0, R)),
                  L=np.zeros((0, R, R)), Z=np.zeros((0, R, J)))


def cp_sweep(Y: Sequence[np.ndarray], H: np.ndarray, V: np.ndarray, W: np.ndarray,
             rtol: Optional[float] = None):
    """One CP-ALS sweep H → V → W for Y_k ≈ H S_k Vᵀ (normal equations):
      H = (Σ_k Y_k V S_k)(VᵀV ∗ WᵀW)⁻¹
      V = (Σ_k Y_kᵀ H S_k)(HᵀH ∗ WᵀW)⁻¹
      W(k,:) = diag(Hᵀ Y_k V)ᵀ (HᵀH ∗ VᵀV)⁻¹."""
    K = len(Y)
    R = H.shape[0]
    W = np.array(W)
    M = np.zeros((R, R))
    for k in range(K):
        M = M + Y[k] @ V @ np.diag(W[k])
    H = M @ pinv((V.T @ V) * (W.T @ W), rtol)
    N = np.zeros_like(V)
    for k in range(K):
        N = N + Y[k].T @ H @ np.diag(W[k])
    V = N @ pinv((H.T @ H) * (W.T @ W), rtol)
    P = pinv((H.T @ H) * (V.T @ V), rtol)
    for k in range(K):
        W[k] = np.diag(H.T @ Y[k] @ V) @ P
    return H, V, W


def dash_update_q(state: StateQ, segments, n_new: int, lam: float,
                  rtol: Optional[float] = None, a_noise=None
                  ) -> Tuple[StateQ, Dict[int, np.ndarray], Dict[int, np.ndarray]]:
    """One constrained-mode update.  Returns the new state, the new rows of
    Q_k (A_new T_k) and the new rows A_new, per touched slice.

    a_noise (tests only, default None): a function applied to each A_new
    right after it is formed, to each updated L_k and to the swept H, V, W,
    so that a test can measure how far roundings of that size move the
    result; None leaves the arithmetic as written."""
    J, R = state.V.shape
    K = state.K
    Kn = K + n_new
    X = _group(segments, K, n_new, J)
    V, H = state.V, state.H
    W = np.vstack([state.W, np.ones((n_new, R))])   # S_k := I for new slices
    # √λ·L_k is the factor of λB_k; new slices start from zero
    L = np.concatenate([np.sqrt(lam) * state.L, np.zeros((n_new, R, R))], axis=0)
    Z = np.concatenate([lam * state.Z, np.zeros((n_new, R, J))], axis=0)
    A: Dict[int, np.ndarray] = {}
    for k, Xk in X.items():
        A[k] = Xk @ V @ np.diag(W[k]) @ H.T
        if a_noise is not None:
            A[k] = a_noise(A[k])
        L[k] = r_factor(np.vstack([L[k], A[k]]))   # (L')ᵀL' = λB_k + A_newᵀA_new
        if a_noise is not None:
            L[k] = np.triu(a_noise(L[k]))
        Z[k] = Z[k] + A[k].T @ Xk
    T = [inv_sqrt_from_factor(L[k], rtol) for k in range(Kn)]
    Y = [T[k] @ Z[k] for k in range(Kn)]
    H2, V2, W2 = cp_sweep(Y, H, V, W, rtol)
    if a_noise is not None:
        H2, V2, W2 = a_noise(H2), a_noise(V2), a_noise(W2)
    Qnew = {k: A[k] @ T[k] for k in X}
    return StateQ(V=V2, H=H2, W=W2, L=L, Z=Z), Qnew, A


def parafac2_als(X: Sequence[np.ndarray], H0, V0, W0, n_iter: int):
    """Classic constrained PARAFAC2-ALS (Procrustes step by SVD, then one
    CP-ALS sweep with explicit Khatri–Rao MTTKRPs).  Written independently
    of dash_update_q; used for initialisation and as its single-batch check."""
    H = np.array(H0, dtype=np.float64)
    V = np.array(V0, dtype=np.float64)
    W = np.array(W0, dtype=np.float64)
    K = len(X)
    R = H.shape[0]
    Q: List[np.ndarray] = []
    for _ in range(n_iter):
        Q = []
        for k in range(K):
            P, _, Zt = np.linalg.svd(X[k] @ V @ np.diag(W[k]) @ H.T, full_matrices=False)
            Q.append(P @ Zt)
        Y = np.stack([Q[k].T @ X[k] for k in range(K)], axis=2)   # R×J×K
        Y1 = Y.reshape(R, -1, order="F")                          # mode-1
        Y2 = np.transpose(Y, (1, 0, 2)).reshape(V.shape[0], -1, order="F")
        Y3 = np.transpose(Y, (2, 0, 1)).reshape(K, -1, order="F")
        H = Y1 @ khatri_rao(W, V) @ pinv((W.T @ W) * (V.T @ V))
        V = Y2 @ khatri_rao(W, H) @ pinv((W.T @ W) * (H.T @ H))
        W = Y3 @ khatri_rao(V, H) @ pinv((V.T @ V) * (H.T @ H))
    return Q, H, V, W


def init_helpers_q(X: Sequence[np.ndarray], H, V, W, a_noise=None) -> StateQ:
    """Constrained-mode helpers of the initial tensor from its final factors
    (the analogue of Eqs. 6-9): L_k = R factor of A_k (B_k = A_kᵀA_k),
    Z_k = A_kᵀX_k with A_k = X_k V S_k Hᵀ."""
    K = len(X)
    J, R = V.shape
    L = np.zeros((K, R, R))
    Z = np.zeros((K, R, J))
    for k in range(K):
        A = X[k] @ V @ np.diag(W[k]) @ H.T
        if a_noise is not None:                     # tests only (see dash_update_q)
            A = a_noise(A)
        L[k] = r_factor(A)
        if a_noise is not None:
            L[k] = np.triu(a_noise(L[k]))
        Z[k] = A.T @ X[k]
    return StateQ(V=np.array(V), H=np.array(H), W=np.array(W), L=L, Z=Z)


# ---------------------------------------------------------------------------
# Errors (fitness, §3.4 Definitions 1-2, §4.1 local/global error)
# ---------------------------------------------------------------------------

def fitness(X: Sequence[np.ndarray], Xhat: Sequence[np.ndarray]) -> float:
    """1 - ||X - X̂||_F / ||X||_F over a set of matrices (direct residual)."""
    num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(X, Xhat))
    den = sum(float(np.sum(a ** 2)) for a in X)
    return 1.0 - np.sqrt(num / den) if den > 0 else 1.0


def weighted_fitness_p(rows, V: np.ndarray, lam: float) -> float:
    """λ-weighted fitness of stored rows with the current V: every row block
    keeps the U_k,new and the S_k,new (its diagonal w) that its own update
    produced, the products that enter F and G (Eqs. 20-21) and that Lemma 3's
    V step fits (Eq. 17), and counts with weight λ^age:
        1 − sqrt(Σ λ^age ||X − U diag(w) Vᵀ||² / Σ λ^age ||X||²).
    rows: iterable of (age, X, U, w)."""
    num = den = 0.0
    for age, X, U, w in rows:
        a = lam ** age
        num += a * float(np.sum((X - reconstruct_p(U, w, V)) ** 2))
        den += a * float(np.sum(X ** 2))
    return 1.0 - np.sqrt(num / den) if den > 0 else 1.0


def slice_error(X_new: np.ndarray, Xhat_new: np.ndarray) -> float:
    """Definition 1 (Eq. 22): mean absolute reconstruction error of a slice's
    new rows, se = Σ|X - X̂| / (I_k,new J)."""
    if X_new.size == 0:
        return 0.0
    return float(np.abs(X_new - Xhat_new).sum() / X_new.size)


def tensor_error(X_new: Sequence[np.ndarray], Xhat_new: Sequence[np.ndarray]) -> float:
    """Definition 2 (Eq. 23): te = mean over slices of se (the local error
    of §4.1)."""
    errs = [slice_error(a, b) for a, b in zip(X_new, Xhat_new)]
    return float(np.mean(errs)) if errs else 0.0


def reconstruct_p(U: np.ndarray, w: np.ndarray, V: np.ndarray) -> np.ndarray:
    """X̂ = U S Vᵀ."""
    return (U * w) @ V.T


def reconstruct_q(Q: np.ndarray, H: np.ndarray, w: np.ndarray, V: np.ndarray) -> np.ndarray:
    """X̂ = Q H S Vᵀ."""
    return ((Q @ H) * w) @ V.T


# ---------------------------------------------------------------------------
# A streaming driver that also keeps every row (for global checks)
# ---------------------------------------------------------------------------

class OracleStream:
    """Runs Dash (mode 'P' or 'Q') over a sequence of batches and keeps all
    data and factor rows, so that tests can recompute from scratch, weight
    rows by λ^age and measure global errors."""

    def __init__(self, mode: str, V0: np.ndarray, lam: float, H0=None, rtol=None):
        self.mode = mode
        self.lam = lam
        self.rtol = rtol
        self.state = empty_state_p(V0) if mode == "P" else empty_state_q(V0, H0)
        # per slice: (update index, X rows, U rows (P) or A rows (Q))
        self.rows: List[List[Tuple[int, np.ndarray, np.ndarray]]] = []
        self.t = 0
        self.last_new: Dict[int, np.ndarray] = {}
        self.last_X: Dict[int, np.ndarray] = {}

    def update(self, segments, n_new: int, n_sweeps: int = 1, **test_modes):
        J = self.state.V.shape[0]
        X = _group(list(segments), self.state.K, n_new, J)
        segs = list(X.items())
        if self.mode == "P":
            self.state, new = dash_update_p(self.state, segs, n_new, self.lam,
                                            n_sweeps=n_sweeps, rtol=self.rtol, **test_modes)
            keep = new
        else:
            self.state, new, keep = dash_update_q(self.state, segs, n_new, self.lam,
                                                  rtol=self.rtol)
        while len(self.rows) < self.state.K:
            self.rows.append([])
        for k, Xk in X.items():
            self.rows[k].append((self.t, Xk, keep[k], np.array(self.state.W[k])))
        self.t += 1
        self.last_new, self.last_X = new, X
        return new

    def slice_rows(self, k: int):
        """All stored rows of slice k: (X, U rows (P) or A rows (Q), λ^age
        per row, age counted in updates since the row arrived)."""
        parts = self.rows[k]
        if not parts:
            J, R = self.state.V.shape
            return np.zeros((0, J)), np.zeros((0, R)), np.zeros(0)
        Xs = np.vstack([p[1] for p in parts])
        Fs = np.vstack([p[2] for p in parts])
        wts = np.concatenate([np.full(p[1].shape[0], self.lam ** (self.t - 1 - p[0]))
                              for p in parts])
        return Xs, Fs, wts
