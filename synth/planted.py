"""Seeded synthetic dual-way streams of planted PARAFAC2 tensors (inputs only).

This module produces the *inputs* that both the FP64 oracle and the CUDA
library consume: the irregular tensor {X_k} revealed over time as new rows of
existing slices plus whole new slices (the dual-way streaming setting of §2.2,
Problem 1, and the time terms of Figure 3).  It holds none of Dash's
arithmetic: it only draws random factors and multiplies them out.

Planted model (one recipe for every workload):
  * H (R×R), V (J×R) and the slice weights W (K_total×R) have U(0,1) entries;
  * Q_k (I_k,final×R) is the Q factor of a QR of a standard Gaussian matrix,
    with its columns' signs fixed so that diag(R̃) > 0, drawn at the slice's
    *final* length and revealed by row prefix, so new rows continue the same
    planted slice;
  * X_k = Q_k H diag(w_k) Vᵀ + σ·N(0,1)  (absolute noise level σ);
  * a drifting stream (drift > 0) uses V + drift·t·V_d for update t's rows.

Row counts are drawn up front from the workload's distributions, so the
stream is a pure function of (workload, seed, device).  The CPU and CUDA
torch generators give different draws for the same seed; every comparison
therefore generates on one device and copies, never regenerates elsewhere.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import torch

BASE_SEED = 2305183760


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape and arrival recipe of one synthetic stream."""
    name: str
    K0: int                    # slices in the initial tensor
    J: int                     # columns shared by every slice
    R: int                     # target rank
    init_rows: Tuple           # distribution of initial I_k
    steps: int                 # number of updates in the stream
    rows_per_step: Tuple       # rows added to every existing slice per update
    new_slices_per_step: int   # L per update
    new_slice_rows: Tuple      # distribution of a new slice's initial rows
    sigma: float               # absolute Gaussian noise level
    lam: float                 # forgetting factor used by this workload
    seed: int
    drift: float = 0.0         # V of update t is V + drift·t·V_d (a drifting stream)
    touch: Tuple = ()          # () every existing slice gets rows; ("uniform", lo, hi): per
                               # update a fraction f ~ U(lo, hi) of them, each with prob. f
    new_slices_dist: Tuple = ()  # () new_slices_per_step per update; else L drawn per update


def _w(name, idx, **kw):
    return Workload(name=name, seed=BASE_SEED + idx, **kw)


# The five dual-way workloads.  Stock-like shapes: J ∈ {85, 96, 144} in the
# paper's Table 2 are matched by J = 88 (c2) and 64–256 (serving); the row
# growth per update mirrors the update cycle of §4.1.
WORKLOADS = {
    "c1": _w("c1", 0, K0=50, J=100, R=10, init_rows=("uniform", 50, 200), steps=10,
             rows_per_step=("const", 10), new_slices_per_step=5,
             new_slice_rows=("uniform", 50, 200), sigma=0.01, lam=1.0),
    "c2": _w("c2", 1, K0=3000, J=88, R=10, init_rows=("uniform", 500, 3000), steps=200,
             rows_per_step=("const", 1), new_slices_per_step=10,
             new_slice_rows=("uniform", 500, 1000), sigma=0.05, lam=0.98),
    "c3": _w("c3", 2, K0=20000, J=256, R=20, init_rows=("lognormal", 400, 1.0, 1, 20000),
             steps=50, rows_per_step=("uniform", 1, 64), new_slices_per_step=100,
             new_slice_rows=("lognormal", 400, 1.0, 1, 20000), sigma=0.1, lam=0.95),
    "c4": _w("c4", 3, K0=50000, J=512, R=32, init_rows=("lognormal", 400, 1.0, 1, 20000),
             steps=20, rows_per_step=("uniform", 1, 64), new_slices_per_step=100,
             new_slice_rows=("lognormal", 400, 1.0, 1, 20000), sigma=0.1, lam=0.95),
}


def scaled(w: Workload, **changes) -> Workload:
    """A copy of a workload with some fields replaced (e.g. fewer slices)."""
    return dataclasses.replace(w, **changes)


def _draw_counts(dist: Tuple, n: int, gen: torch.Generator) -> torch.Tensor:
    kind = dist[0]
    if n == 0:
        return torch.zeros(0, dtype=torch.int64)
    if kind == "const":
        return torch.full((n,), int(dist[1]), dtype=torch.int64)
    if kind == "uniform":                      # integers lo..hi inclusive
        lo, hi = int(dist[1]), int(dist[2])
        return torch.randint(lo, hi + 1, (n,), generator=gen, dtype=torch.int64)
    if kind == "lognormal":                    # median, sigma_ln, clip lo, clip hi
        med, s, lo, hi = dist[1], dist[2], int(dist[3]), int(dist[4])
        z = torch.randn(n, generator=gen, dtype=torch.float64)
        v = torch.round(torch.exp(math.log(med) + s * z))
        return v.clamp(lo, hi).to(torch.int64)
    raise ValueError(f"unknown row distribution {dist!r}")


@dataclasses.dataclass
class Batch:
    """New data of one update in CSR form: segment s covers rows
    row_ptr[s]..row_ptr[s+1] of X and belongs to slice slice_ids[s].

    Slices with id >= K_before are new; they are numbered consecutively
    K_before .. K_before+n_new-1 and each has exactly one segment.
    """
    slice_ids: torch.Tensor     # (n_seg,) int64, ascending
    row_ptr: torch.Tensor       # (n_seg+1,) int64
    X: torch.Tensor             # (N, J)
    K_before: int
    n_new: int

    @property
    def n_rows(self) -> int:
        return int(self.X.shape[0])

    def segments(self):
        """(slice id, rows) pairs, in order."""
        rp = self.row_ptr.tolist()
        for s, k in enumerate(self.slice_ids.tolist()):
            yield k, self.X[rp[s]:rp[s + 1]]


class PlantedStream:
    """A planted PARAFAC2 stream for one workload.

    batch(0) is the initial tensor (K0 slices, all their initial rows);
    batch(t), t = 1..steps, is update t: rows_per_step new rows for every
    slice that exists before it, then new_slices_per_step new slices.
    """

    def __init__(self, w: Workload, device="cpu", dtype=torch.float64,
                 seed: Optional[int] = None):
        self.w = w
        self.device = torch.device(device)
        self.dtype = dtype
        seed = w.seed if seed is None else seed
        g = torch.Generator(device="cpu").manual_seed(seed)
        T = w.steps
        # new slices per update (extra draws only for a drawn L, so streams
        # with a fixed L are unchanged)
        if w.new_slices_dist:
            self.L_t = [0] + _draw_counts(w.new_slices_dist, T, g).tolist()
        else:
            self.L_t = [0] + [w.new_slices_per_step] * T
        self.K_before_t = [0] * (T + 1)
        for t in range(2, T + 1):
            self.K_before_t[t] = self.K_before_t[t - 1] + self.L_t[t - 1]
        for t in range(1, T + 1):
            self.K_before_t[t] += w.K0
        self.K_total = w.K0 + sum(self.L_t)
        # ---- row counts (host, int64) --------------------------------------
        born = torch.zeros(self.K_total, dtype=torch.int64)   # arrival update
        first = torch.empty(self.K_total, dtype=torch.int64)  # rows at arrival
        first[: w.K0] = _draw_counts(w.init_rows, w.K0, g)
        self.step_rows: List[torch.Tensor] = [first[: w.K0].clone()]
        for t in range(1, T + 1):
            k_exist = self.K_before_t[t]
            L = self.L_t[t]
            grow = _draw_counts(w.rows_per_step, k_exist, g)
            if w.touch:                        # a random fraction of the slices
                kind, flo, fhi = w.touch
                if kind != "uniform":
                    raise ValueError(f"unknown touch distribution {w.touch!r}")
                f = flo + (fhi - flo) * float(torch.rand(1, generator=g, dtype=torch.float64))
                grow = grow * (torch.rand(k_exist, generator=g, dtype=torch.float64) < f)
            lo = k_exist
            first[lo: lo + L] = _draw_counts(w.new_slice_rows, L, g)
            born[lo: lo + L] = t
            self.step_rows.append(torch.cat([grow, first[lo: lo + L]]))
        self.born = born
        final = torch.zeros(self.K_total, dtype=torch.int64)
        for t, rows in enumerate(self.step_rows):
            final[: rows.numel()] += rows
        self.final_len = final
        # prefix offsets of each slice's planted rows inside the flat Q store
        self.q_off = torch.zeros(self.K_total + 1, dtype=torch.int64)
        self.q_off[1:] = torch.cumsum(final, 0)
        # rows of each slice revealed before update t
        self._revealed = torch.zeros(self.K_total, dtype=torch.int64)
        # ---- planted factors (drawn on the target device) -------------------
        dg = torch.Generator(device=self.device).manual_seed(seed + 7919)
        self._dgen = dg
        R, J = w.R, w.J
        kw = dict(generator=dg, device=self.device, dtype=dtype)
        self.H = torch.rand(R, R, **kw)
        self.V = torch.rand(J, R, **kw)
        self.W = torch.rand(self.K_total, R, **kw)
        self.Q = self._planted_q(final, dg)
        # a drifting stream moves V along a fixed random direction (drawn last,
        # so streams without drift are unchanged)
        self.Vd = torch.rand(J, R, **kw) if w.drift else None
        self._next = 0

    # -- planted orthonormal Q_k, bucketed by length ---------------------------
    def _planted_q(self, final: torch.Tensor, dg: torch.Generator) -> torch.Tensor:
        """Q_k = the Q factor, with positive diag(R̃), of a Gaussian matrix of
        the slice's final length.  Computed as a Cholesky QR (R̃ = chol(GᵀG)ᵀ,
        Q = G R̃⁻¹), which is that same unique factor.  A slice shorter than R
        gets orthonormal rows instead (first rows of an orthogonal matrix)."""
        R = self.w.R
        dev = self.device
        total = int(final.sum())
        G = torch.randn(total, R, generator=dg, device=dev, dtype=self.dtype)
        Q = torch.zeros_like(G)
        lens = final.clone()
        offs = self.q_off[:-1]
        short = torch.nonzero((lens > 0) & (lens < R)).flatten().tolist()
        for k in short:                      # rare: fewer rows than the rank
            o, L = int(offs[k]), int(lens[k])
            g = G[o:o + L].T.contiguous().cpu().double()             # R×L
            q, r = torch.linalg.qr(g)                                 # R×L, orthonormal cols
            sgn = torch.sign(torch.diagonal(r))
            sgn[sgn == 0] = 1
            Q[o:o + L] = (q * sgn).T.to(device=dev, dtype=self.dtype)
        tall = torch.nonzero(lens >= R).flatten()
        if tall.numel():
            tl = lens[tall]
            order = torch.argsort(tl)
            tall, tl = tall[order], tl[order]
            i, n = 0, tall.numel()
            cap_rows = 1 << 23
            while i < n:
                l0 = int(tl[i])
                lim = max(int(l0 * 1.25) + 1, l0 + 8)
                j = int(torch.searchsorted(tl, torch.tensor(lim), right=True))
                j = max(j, i + 1)
                j = min(j, i + max(1, cap_rows // max(int(tl[j - 1]), 1)))
                ids = tall[i:j]
                ln = tl[i:j]
                Lmax = int(ln.max())
                ar = torch.arange(Lmax)
                mask = ar[None, :] < ln[:, None]
                idx = (offs[ids][:, None] + ar[None, :]).masked_fill(~mask, 0)
                idx_d, mask_d = idx.to(dev), mask.to(dev)
                pad = G[idx_d] * mask_d[..., None]
                # small R×R factorisations in FP64 on the host; the tall
                # products stay on the device
                gram = (pad.transpose(1, 2) @ pad).cpu().double()
                Linv = torch.linalg.inv(torch.linalg.cholesky(gram))
                q = pad @ Linv.transpose(1, 2).to(device=dev, dtype=self.dtype)
                Q[idx_d[mask_d]] = q[mask_d]
                i = j
        return Q

    def batch(self, t: int) -> Batch:
        """Update t's new data (t = 0: the initial tensor).  Batches must be
        drawn in order 0, 1, 2, ... because rows are revealed by prefix."""
        if t != self._next:
            raise ValueError(f"batches must be drawn in order (next is {self._next})")
        self._next += 1
        w = self.w
        rows = self.step_rows[t]
        k_count = rows.numel()
        K_before = 0 if t == 0 else self.K_before_t[t]
        n_new = w.K0 if t == 0 else self.L_t[t]
        ids = torch.arange(k_count, dtype=torch.int64)
        row_ptr = torch.zeros(k_count + 1, dtype=torch.int64)
        row_ptr[1:] = torch.cumsum(rows, 0)
        N = int(row_ptr[-1])
        # gather the planted Q rows revealed at this update, chunk by chunk
        start = self.q_off[:k_count] + self._revealed[:k_count]
        seg_of_row = torch.repeat_interleave(ids, rows)
        within = torch.arange(N, dtype=torch.int64) - row_ptr[:-1].repeat_interleave(rows)
        src = start.repeat_interleave(rows) + within
        self._revealed[:k_count] += rows
        X = torch.empty(N, w.J, device=self.device, dtype=self.dtype)
        Vt = self.V if self.Vd is None else self.V + (w.drift * t) * self.Vd
        chunk = 1 << 21
        for c0 in range(0, N, chunk):
            c1 = min(N, c0 + chunk)
            q = self.Q.index_select(0, src[c0:c1].to(self.device))
            wk = self.W.index_select(0, seg_of_row[c0:c1].to(self.device))
            torch.matmul((q @ self.H) * wk, Vt.T, out=X[c0:c1])
            if w.sigma:
                X[c0:c1].add_(torch.randn(c1 - c0, w.J, generator=self._dgen,
                                          device=self.device, dtype=self.dtype), alpha=w.sigma)
        if w.touch and t > 0:                  # list only the touched old slices
            keep = (rows > 0) | (ids >= K_before)
            ids = ids[keep]
            row_ptr = torch.zeros(ids.numel() + 1, dtype=torch.int64)
            row_ptr[1:] = torch.cumsum(rows[keep], 0)
        return Batch(slice_ids=ids, row_ptr=row_ptr, X=X,
                     K_before=K_before, n_new=n_new)


def workload(name: str, **changes) -> Workload:
    w = WORKLOADS[name]
    return scaled(w, **changes) if changes else w


def tiny(K0=4, J=6, R=3, steps=3, rows=("uniform", 1, 4), new=2,
         new_rows=("uniform", 2, 6), init_rows=("uniform", 4, 9),
         sigma=0.0, lam=1.0, seed=11) -> Workload:
    """A small stream for exact checks on the CPU."""
    return Workload(name="tiny", K0=K0, J=J, R=R, init_rows=init_rows, steps=steps,
                    rows_per_step=rows, new_slices_per_step=new,
                    new_slice_rows=new_rows, sigma=sigma, lam=lam, seed=seed)


def ragged_batch(K_before: int, n_new: int, J: int, rows: Sequence[int],
                 seed: int, dtype=torch.float64, device="cpu",
                 slice_ids: Optional[Sequence[int]] = None) -> Batch:
    """An unstructured batch with the given per-segment row counts (Gaussian
    entries): for edge cases (empty segments, 1-row slices, ragged tails)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    rows_t = torch.tensor(list(rows), dtype=torch.int64)
    if slice_ids is None:
        slice_ids = list(range(len(rows)))
    row_ptr = torch.zeros(len(rows) + 1, dtype=torch.int64)
    row_ptr[1:] = torch.cumsum(rows_t, 0)
    X = torch.randn(int(row_ptr[-1]), J, generator=g, dtype=torch.float64)
    return Batch(slice_ids=torch.tensor(list(slice_ids), dtype=torch.int64),
                 row_ptr=row_ptr, X=X.to(device=device, dtype=dtype),
                 K_before=K_before, n_new=n_new)
