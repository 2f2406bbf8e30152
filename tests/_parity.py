"""Helpers for the GPU-vs-oracle parity tests: run the same seeded stream
through the FP64 oracle and through the CUDA library (C ABI) and compare."""
from __future__ import annotations

import numpy as np
import torch

from oracle import dash_oracle as O

# tolerances (relative, normwise max): FP64 products ≤ 1e-10; FP32 / mixed
# products ≤ 1e-4 with batch fitness within 1e-3
TOL = {"fp64": 1e-10, "fp32": 1e-4, "f16x3": 1e-4, "f16x3-fused": 1e-4, "f16x3-split": 1e-4,
       "f16x3-split-warp": 1e-4}
FIT_TOL = {"fp64": 1e-10, "fp32": 1e-3, "f16x3": 1e-3, "f16x3-fused": 1e-3, "f16x3-split": 1e-3,
           "f16x3-split-warp": 1e-3}


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    scale = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b))) / scale


def rel_rows(a, b) -> float:
    """Largest normwise relative error over the leading index (per slice for
    W, c and D): a slice whose own entries are small relative to the largest
    slice is judged at its own scale.  A slice whose reference is exactly zero
    is judged against the global scale."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    a2 = a.reshape(a.shape[0], -1)
    b2 = b.reshape(b.shape[0], -1)
    gscale = max(float(np.max(np.abs(b2))), 1e-300)
    scale = np.max(np.abs(b2), axis=1)
    scale = np.where(scale > 0.0, scale, gscale)
    return float(np.max(np.max(np.abs(a2 - b2), axis=1) / scale))


def record(step: str, errors: dict, limits=None):
    """Append one parity record (the measured errors and the limits applied)
    of the running test to the JSON-lines file named by DASH_PARITY_RECORD,
    if set."""
    import json
    import os
    path = os.environ.get("DASH_PARITY_RECORD")
    if not path:
        return
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    fl = lambda d: {k: float(v) for k, v in d.items()} if isinstance(d, dict) else d
    with open(path, "a") as f:
        f.write(json.dumps({"test": test, "step": step, "errors": fl(errors),
                            "limits": fl(limits)}) + "\n")


def segs_np(batch, dtype):
    """(k, X) pairs with X rounded to the GPU's input dtype (the oracle sees
    exactly the values the kernels read)."""
    out = []
    for k, x in batch.segments():
        out.append((k, x.to(dtype).to(torch.float64).numpy()))
    return out


def oracle_fit_p(segs, V0, n_iter: int) -> "O.StateP":
    """The static initial fit as the library runs it (§3.2.1 with our own
    static ALS): n_iter oracle updates on empty helpers (λ = 0), each one
    static ALS iteration (pinned against lstsq in the CPU tests), then the
    helpers of the final factors (Eqs. 6-9).  segs: (k, X_k) of every
    initial slice, k = 0..K0-1 in order."""
    st = O.empty_state_p(V0)
    U = {}
    for it in range(n_iter):
        st, U = O.dash_update_p(st, segs, len(segs) if it == 0 else 0, 0.0)
    X = [x for _, x in segs]
    R = V0.shape[1]
    return O.init_helpers_p(X, [U.get(k, np.zeros((0, R))) for k in range(len(X))], st.W, st.V)


def oracle_batch_fitness_p(state, U, X):
    ks = sorted(X.keys())
    return O.fitness([X[k] for k in ks],
                     [O.reconstruct_p(U[k], state.W[k], state.V) for k in ks])


def gpu_rows_by_slice(rows: np.ndarray, batch):
    """Split the N×R new rows of the library (staging order) per slice."""
    rp = batch.row_ptr.tolist()
    out = {}
    for s, k in enumerate(batch.slice_ids.tolist()):
        out.setdefault(k, []).append(rows[rp[s]:rp[s + 1]])
    return {k: np.concatenate(v, axis=0) for k, v in out.items()}


def compare_state_p(gpu: dict, st: "O.StateP", tol: float, what=""):
    """Normwise relative error of every factor and helper, plus the same per
    slice for W, c and D (each slice at its own scale), all within tol."""
    errs = {
        "V": rel(gpu["V"], st.V), "W": rel(gpu["W"], st.W), "c": rel(gpu["c"], st.c),
        "D": rel(gpu["D"], st.D), "F": rel(gpu["F"], st.F), "G": rel(gpu["G"], st.G),
        "W_slice": rel_rows(gpu["W"], st.W), "c_slice": rel_rows(gpu["c"], st.c),
        "D_slice": rel_rows(gpu["D"], st.D),
    }
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what} state mismatch (tol {tol:g}): {errs}"
    return errs


# Shadow oracle runs (mode Q).  The shadow perturbs every bulk product
# A_new = X_new V S_k Hᵀ, every updated L_k, the swept H, V, W and every
# input row, at the rounding level of the path; the spread between it and the oracle measures how far a correct
# implementation with a different rounding can land.
#   FP64 path: A_new relative noise u·sqrt(J + R), u = 2^-53 (the
#     random-walk size of the rounding of the J- and R-term sums).
#   Mixed path: A_new relative noise u = 2^-24 (A_new held in FP32).
SHADOW_U = {"fp64": 1.1e-16, "fp32": 6.0e-8, "f16x3": 6.0e-8}
SHADOW_FACTOR = 16.0
# quantities that carry the polar factor's conditioning in the mixed path;
# the rest keep the stated mixed tolerance there
SHADOW_MIXED = ("Q", "Y")


def shadow_scale(prec: str, J: int, R: int) -> float:
    u = SHADOW_U[prec]
    return u * np.sqrt(J + R) if prec == "fp64" else u


def shadow_tol(prec: str, spread: dict) -> dict:
    """Per-quantity tolerance.  FP64: the stated 1e-10, or SHADOW_FACTOR
    times the shadow spread, whichever is larger.  Mixed: the stated 1e-4
    for V, H, W, L; for the new Q rows and Y_k (= Q_kᵀΛX_k) the larger of
    1e-4 and SHADOW_FACTOR times the shadow spread.  On ill-conditioned
    slices (cond(A_k) up to 1e6 on planted U(0,1) factors) the polar factor
    Q_k moves by about u·cond(A_k) under a rounding of size u of A_k, so the
    stated tolerance is out of reach of any implementation whose rounding
    differs from the oracle's; the shadow run measures that limit."""
    out = {}
    for k, v in spread.items():
        if prec == "fp64" or k in SHADOW_MIXED:
            out[k] = max(TOL[prec], SHADOW_FACTOR * v)
        else:
            out[k] = TOL[prec]
    return out


def a_noise(scale: float, rng):
    """The shadow run's perturbation of a bulk product (relative `scale`)."""
    return lambda A: A * (1.0 + scale * rng.standard_normal(A.shape))


def perturb(a, u: float, rng) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a * (1.0 + u * rng.standard_normal(a.shape))


def oracle_y(st: "O.StateQ") -> np.ndarray:
    """The projected data Y_k = T_k Z_k (= Q_kᵀΛ_kX_k) of an oracle state,
    T_k = (L_kᵀL_k)^{-1/2} from the oracle's own factor."""
    return np.stack([O.inv_sqrt_from_factor(st.L[k]) @ st.Z[k] for k in range(st.K)]) \
        if st.K else np.zeros((0,) + st.Z.shape[1:])


def state_q_errors(gpu: dict, st: "O.StateQ") -> dict:
    return {"V": rel(gpu["V"], st.V), "H": rel(gpu["H"], st.H), "W": rel(gpu["W"], st.W),
            "L": rel(gpu["L"], st.L), "Y": rel(gpu["Y"], oracle_y(st))}


def compare_state_q(gpu: dict, st: "O.StateQ", tol, what=""):
    """tol: one number, or a per-quantity dict (shadow_tol)."""
    errs = state_q_errors(gpu, st)
    tl = tol if isinstance(tol, dict) else {k: tol for k in errs}
    bad = {k: v for k, v in errs.items() if not v <= tl[k]}
    assert not bad, f"{what} state mismatch: errors {errs} tolerances {tl}"
    return errs
