"""Helpers for the GPU-vs-oracle parity tests: run the same seeded stream
through the FP64 oracle and through the CUDA library (C ABI) and compare."""
from __future__ import annotations

import numpy as np
import torch

from oracle import dash_oracle as O

# tolerances (relative, normwise max): FP64 products ≤ 1e-10; FP32 / mixed
# products ≤ 1e-4 with batch fitness within 1e-3
TOL = {"fp64": 1e-10, "fp32": 1e-4, "f16x3": 1e-4}
FIT_TOL = {"fp64": 1e-10, "fp32": 1e-3, "f16x3": 1e-3}


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    scale = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b))) / scale


def segs_np(batch, dtype):
    """(k, X) pairs with X rounded to the GPU's input dtype (the oracle sees
    exactly the values the kernels read)."""
    out = []
    for k, x in batch.segments():
        out.append((k, x.to(dtype).to(torch.float64).numpy()))
    return out


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
    errs = {
        "V": rel(gpu["V"], st.V), "W": rel(gpu["W"], st.W), "c": rel(gpu["c"], st.c),
        "D": rel(gpu["D"], st.D), "F": rel(gpu["F"], st.F), "G": rel(gpu["G"], st.G),
    }
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what} state mismatch (tol {tol:g}): {errs}"
    return errs
