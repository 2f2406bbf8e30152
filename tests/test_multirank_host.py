"""Slice-sharded Dash on CPU ranks (gloo, world size 2).

Dash shards by slice: every per-slice step (Lemma 1's U_k,new, Eqs. 15-16's
c_k and D_k, Lemma 2's W(k,:); in the constrained mode A_new, L_k, Z_k, T_k,
Y_k and the W rows of the sweep) reads only that slice's rows and the
replicated V (and H), so it runs on the rank that owns the slice.  The only
exchange is one sum over ranks per update of the terms that run over all k:
  mode P:  the F and G increments of Eqs. 20-21 (J·R + R² values);
  mode Q:  Σ Y_k V S_k with WᵀW, then Σ Y_kᵀ H S_k (the two MTTKRPs of the
           sweep's H and V steps).
Each rank composes the oracle's per-slice functions over the slices it owns
and sums over ranks with an all-reduce; rank 0 then checks that the sharded
stream equals the single-rank oracle stream to rounding (the sums are only
regrouped).  No GPU and no library call is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import dash_oracle as O
from synth.planted import PlantedStream, tiny

WORLD = 2
TOL = 1e-11


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _allreduce(a: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _gather_rows(a: np.ndarray, mine: np.ndarray) -> np.ndarray:
    """Rows owned by each rank, assembled on every rank (other rows zero)."""
    z = np.zeros_like(a)
    z[mine] = a[mine]
    return _allreduce(z)


def _sharded_update_p(st: O.StateP, segments, n_new, lam, rank):
    """One update of Algorithm 1 with the slices split k mod WORLD."""
    J, R = st.V.shape
    Kn = st.K + n_new
    mine = np.arange(Kn) % WORLD == rank
    X = {k: x for k, x in O._group(segments, st.K, n_new, J).items() if mine[k]}
    V = st.V
    W = np.vstack([st.W, np.ones((n_new, R))])
    c = lam * np.vstack([st.c, np.zeros((n_new, R))])
    D = lam * np.concatenate([st.D, np.zeros((n_new, R, R))], axis=0)
    U = {k: O.update_u_new(Xk, V, W[k]) for k, Xk in X.items()}     # Eq. 11
    for k in np.flatnonzero(mine):
        if k in X:
            c[k] = c[k] + O.c_term(X[k], V, U[k])                      # Eq. 15
            D[k] = D[k] + U[k].T @ U[k]                                 # Eq. 16
        W[k] = O.solve_w_row(c[k], D[k], V)                             # Eq. 12
    dF = np.zeros((J, R))
    dG = np.zeros((R, R))
    for k, Xk in X.items():
        S = np.diag(W[k])
        dF = dF + Xk.T @ U[k] @ S                                       # Eq. 20 (local part)
        dG = dG + S @ U[k].T @ U[k] @ S                                 # Eq. 21 (local part)
    msg = _allreduce(np.concatenate([dF.ravel(), dG.ravel()]))         # the one exchange
    F = lam * st.F + msg[: J * R].reshape(J, R)
    G = lam * st.G + msg[J * R:].reshape(R, R)
    V = F @ O.pinv(G)                                                   # Eq. 17
    W, c = _gather_rows(W, mine), _gather_rows(c, mine)
    D = _gather_rows(D.reshape(Kn, -1), mine).reshape(Kn, R, R)
    return O.StateP(V=V, W=W, c=c, D=D, F=F, G=G)


def _sharded_update_q(st: O.StateQ, segments, n_new, lam, rank):
    """One constrained-mode update with the slices split k mod WORLD."""
    J, R = st.V.shape
    Kn = st.K + n_new
    mine = np.arange(Kn) % WORLD == rank
    own = np.flatnonzero(mine)
    X = {k: x for k, x in O._group(segments, st.K, n_new, J).items() if mine[k]}
    V, H = st.V, st.H
    W = np.vstack([st.W, np.ones((n_new, R))])
    L = np.concatenate([np.sqrt(lam) * st.L, np.zeros((n_new, R, R))], axis=0)
    Z = np.concatenate([lam * st.Z, np.zeros((n_new, R, J))], axis=0)
    for k, Xk in X.items():
        A = Xk @ V @ np.diag(W[k]) @ H.T
        L[k] = O.r_factor(np.vstack([L[k], A]))
        Z[k] = Z[k] + A.T @ Xk
    Y = {k: O.inv_sqrt_from_factor(L[k]) @ Z[k] for k in own}
    # sweep, H step: Σ Y_k V S_k and WᵀW summed over ranks
    M = sum((Y[k] @ V @ np.diag(W[k]) for k in own), np.zeros((R, R)))
    WtW = sum((np.outer(W[k], W[k]) for k in own), np.zeros((R, R)))
    msg = _allreduce(np.concatenate([M.ravel(), WtW.ravel()]))
    M, WtW = msg[: R * R].reshape(R, R), msg[R * R:].reshape(R, R)
    H = M @ O.pinv((V.T @ V) * WtW)
    # V step: Σ Y_kᵀ H S_k summed over ranks
    N = sum((Y[k].T @ H @ np.diag(W[k]) for k in own), np.zeros((J, R)))
    N = _allreduce(N)
    V = N @ O.pinv((H.T @ H) * WtW)
    # W step: local rows
    P = O.pinv((H.T @ H) * (V.T @ V))
    for k in own:
        W[k] = np.diag(H.T @ Y[k] @ V) @ P
    W = _gather_rows(W, mine)
    L = _gather_rows(L.reshape(Kn, -1), mine).reshape(Kn, R, R)
    Z = _gather_rows(Z.reshape(Kn, -1), mine).reshape(Kn, R, J)
    return O.StateQ(V=V, H=H, W=W, L=L, Z=Z)


def _segs(b):
    return [(k, x.numpy()) for k, x in b.segments()]


def _worker(rank, port, mode, lam, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        w = tiny(K0=5, J=7, R=3, steps=4, sigma=0.05, lam=lam, seed=29)
        s = PlantedStream(w)
        V0 = np.random.default_rng(7).random((7, 3))
        if mode == "P":
            ref, sh = O.empty_state_p(V0), O.empty_state_p(V0)
        else:
            H0 = np.random.default_rng(8).random((3, 3)) + np.eye(3)
            ref, sh = O.empty_state_q(V0, H0), O.empty_state_q(V0, H0)
        err = 0.0
        for t in range(w.steps + 1):
            b = s.batch(t)
            if mode == "P":
                ref, _ = O.dash_update_p(ref, _segs(b), b.n_new, lam)
                sh = _sharded_update_p(sh, _segs(b), b.n_new, lam, rank)
                pairs = [(ref.V, sh.V), (ref.W, sh.W), (ref.c, sh.c), (ref.D, sh.D),
                         (ref.F, sh.F), (ref.G, sh.G)]
            else:
                ref, _, _ = O.dash_update_q(ref, _segs(b), b.n_new, lam)
                sh = _sharded_update_q(sh, _segs(b), b.n_new, lam, rank)
                pairs = [(ref.V, sh.V), (ref.H, sh.H), (ref.W, sh.W), (ref.L, sh.L),
                         (ref.Z, sh.Z)]
            for a, c in pairs:
                err = max(err, float(np.max(np.abs(a - c)) / max(np.max(np.abs(a)), 1e-300)))
        if rank == 0:
            out.put(err)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,lam", [("P", 1.0), ("P", 0.7), ("Q", 1.0), ("Q", 0.8)])
def test_slice_sharded_stream_equals_single_rank(mode, lam):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(_free_port(), mode, lam, q), nprocs=WORLD,
                       join=True, start_method="spawn")
    err = q.get()
    assert err < TOL, err
