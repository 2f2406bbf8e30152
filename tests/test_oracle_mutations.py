"""Planted mistakes in the oracle must fail its pins.

Each case patches one plausible slip into the oracle (on the CPU only) and
checks that at least one pin in test_oracle_pins.py then fails.
"""
import numpy as np
import pytest

from oracle import dash_oracle as O
import tests.test_oracle_pins as P


def _dropped_s_in_lemma1(X_new, V, w, rtol=None):
    return X_new @ V @ O.pinv(V.T @ V, rtol)                  # S_k dropped


def _sum_not_hadamard(c, D, V, rtol=None):
    return c @ O.pinv((V.T @ V) + D, rtol)                    # ∗ read as +


def _transposed_c_term(X, V, U):
    if X.shape[0] == 0:
        return np.zeros(V.shape[1])
    return O.vec(X) @ O.khatri_rao(U, V)                       # operands swapped


def _u_without_pinv_cutoff(X_new, V, w, rtol=None):
    S = np.diag(w)
    return X_new @ V @ S @ np.linalg.inv(S @ V.T @ V @ S + 1e-3 * np.eye(len(w)))


def _lambda_dropped_on_old_f_g(state, segments, n_new, lam, **kw):
    undo = state.copy()
    if lam > 0:
        undo.F = state.F / lam                                 # λ·F_old becomes F_old
        undo.G = state.G / lam
    return _ORIG_UPDATE(undo, segments, n_new, lam, **kw)


_ORIG_UPDATE = O.dash_update_p


def _r_factor_unsquared(M):
    L = _ORIG_R_FACTOR(M)
    return L * L                                               # entrywise square


def _polar_via_transpose(L, rtol=None):
    return _ORIG_INV_SQRT_F(L.T, rtol)                          # factor transposed


def _fitness_without_root(X, Xhat):
    num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(X, Xhat))
    den = sum(float(np.sum(a ** 2)) for a in X)
    return 1.0 - num / den if den > 0 else 1.0                 # sqrt dropped


def _init_helpers_q_without_s(X, H, V, W, a_noise=None):
    return _ORIG_INIT_Q(X, H, V, np.ones_like(np.asarray(W)), a_noise)   # S_k dropped from A_k


_ORIG_INIT_Q = O.init_helpers_q
_ORIG_R_FACTOR = O.r_factor
_ORIG_INV_SQRT_F = O.inv_sqrt_from_factor

CASES = [
    ("update_u_new", _dropped_s_in_lemma1, [P.test_lemma1_u_new_is_the_least_squares_solution]),
    ("solve_w_row", _sum_not_hadamard,
     [lambda: P.test_lemma2_w_minimises_weighted_loss_with_v_frozen(1.0)]),
    ("c_term", _transposed_c_term, [P.test_c_term_equals_explicit_triple_sum]),
    ("update_u_new", _u_without_pinv_cutoff, [P.test_lemma1_u_new_is_the_least_squares_solution]),
    ("dash_update_p", _lambda_dropped_on_old_f_g, [P.test_worked_example_rank_one_exact_fractions]),
    ("r_factor", _r_factor_unsquared, [lambda: P.test_mode_q_summaries_exact_and_q_orthonormal(0.8)]),
    ("inv_sqrt_from_factor", _polar_via_transpose,
     [P.test_mode_q_single_batch_equals_parafac2_als_iteration]),
    ("fitness", _fitness_without_root, [P.test_fitness_takes_the_root_of_the_pooled_residual_ratio]),
    ("init_helpers_q", _init_helpers_q_without_s, [P.test_init_helpers_q_follow_their_definition]),
]


@pytest.mark.parametrize("name,fake,pins", CASES, ids=[f"{c[0]}:{c[1].__name__}" for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, name, fake, pins):
    monkeypatch.setattr(O, name, fake)
    failed = 0
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, np.linalg.LinAlgError):
            failed += 1
    assert failed > 0, f"no pin caught the planted mistake in {name}"
