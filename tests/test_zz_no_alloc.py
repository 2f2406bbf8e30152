"""The allocation-free F increment (dash_f_increment_noalloc), for callers
that cannot allocate device memory, gives the same F_inc as dash_update().

A model whose F starts at zero holds F = λ·0 + F_inc after one update, so its
F is the existing entry point's F_inc; the allocation-free entry point gets
the same rows, their U_k,new and the updated W, through the C ABI.  Two calls
in a row, on batches of different sizes, check that nothing a previous call
left in the shared static array leaks into the next result.  This file is
collected last so that a failure here does not hide the other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream, tiny

pytestmark = pytest.mark.gpu


def _oracle_state(w):
    s = PlantedStream(w, dtype=torch.float32)
    b0 = s.batch(0)
    X0 = [x.double().numpy() for _, x in b0.segments()]
    rng = np.random.default_rng(11)
    U, W, V = O.static_als_p(X0, rng.random((w.J, w.R)), np.ones((len(X0), w.R)), 2)
    return s, O.init_helpers_p(X0, U, W, V)


def test_noalloc_f_increment_matches_update():
    from paper_2305_18376_gb300 import DashModel, _native
    lib = _native.load()
    w = tiny(K0=40, J=70, R=7, steps=2, sigma=0.05, lam=0.9, rows=("uniform", 1, 40),
             new_rows=("uniform", 30, 90), init_rows=("uniform", 10, 30))
    s, st = _oracle_state(w)
    for t in (1, 2):
        b = s.batch(t)
        K_all = b.K_before + b.n_new
        m = DashModel(w.J, w.R, w.lam, precision="fp32", input_dtype="f32", max_slices=128,
                      max_rows=4096, max_segments=256)
        W_pad = np.vstack([st.W, np.ones((max(0, b.K_before - st.K), w.R))])[: b.K_before]
        m.set_state_p(st.V, W_pad, st.c[: b.K_before] if st.K >= b.K_before else
                      np.vstack([st.c, np.zeros((b.K_before - st.K, w.R))]),
                      st.D[: b.K_before] if st.K >= b.K_before else
                      np.concatenate([st.D, np.zeros((b.K_before - st.K, w.R, w.R))]),
                      np.zeros((w.J, w.R)), st.G)
        X = b.X.float().cuda()
        m.update_device(b.slice_ids.numpy(), b.row_ptr.numpy(), X)
        g = m.get_state_p()
        F_ref = g["F"]                                # λ·0 + F_inc
        U = torch.from_numpy(m.new_rows()).float().cuda()
        Wd = torch.from_numpy(g["W"]).cuda()
        seg_row = b.row_ptr.cuda()
        seg_slice = b.slice_ids.to(torch.int32).cuda()
        out = torch.full((w.J, w.R), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        stat = lib.dash_f_increment_noalloc(X.data_ptr(), U.data_ptr(), b.n_rows, w.J, w.R,
                                            seg_row.data_ptr(), seg_slice.data_ptr(),
                                            b.slice_ids.numel(), Wd.data_ptr(), out.data_ptr(),
                                            None)
        assert stat == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = float(np.max(np.abs(got - F_ref)) / np.max(np.abs(F_ref)))
        assert err <= 1e-4, (t, err)
        assert K_all == m.K
        m.close()


def _oracle_f_inc(X, U, seg_row, seg_slice, W):
    """Σ_k X_k,newᵀ U_k,new S_k (Eq. 20's new term) from the oracle: the rows
    grouped by slice and passed to init_helpers_p, whose F is that sum
    (Eq. 8 has the same form)."""
    rows = {}
    for s in range(len(seg_slice)):
        rows.setdefault(int(seg_slice[s]), []).append((seg_row[s], seg_row[s + 1]))
    ks = sorted(rows)
    Xk = [np.concatenate([X[a:b] for a, b in rows[k]]) for k in ks]
    Uk = [np.concatenate([U[a:b] for a, b in rows[k]]) for k in ks]
    Wk = np.stack([W[k] for k in ks])
    return O.init_helpers_p(Xk, Uk, Wk, np.zeros((X.shape[1], U.shape[1]))).F


def test_noalloc_large_then_small_call_on_a_side_stream():
    """A call with every one of the 64 row chunks and J·R = 2^15 (R = 64, the
    largest rank), then a call with fewer rows, another J and R: each equals
    the oracle's F_inc (FP32 products: 1e-4), so nothing the first
    call left in the shared array reaches the second.  Both on a non-default
    stream."""
    from paper_2305_18376_gb300 import _native
    lib = _native.load()
    rng = np.random.default_rng(5)
    side = torch.cuda.Stream()
    for (N, J, R, n_seg) in ((8192, 512, 64, 120), (900, 70, 7, 40)):
        cuts = np.sort(rng.choice(np.arange(1, N), n_seg - 1, replace=False))
        seg_row = np.concatenate([[0], cuts, [N]]).astype(np.int64)
        seg_slice = rng.integers(0, 3 * n_seg, n_seg).astype(np.int32)
        X = rng.random((N, J)).astype(np.float32)
        U = (rng.standard_normal((N, R)) * 0.1).astype(np.float32)
        W = rng.random((3 * n_seg, R)) + 0.5
        with torch.cuda.stream(side):
            Xd, Ud = torch.from_numpy(X).cuda(), torch.from_numpy(U).cuda()
            sr, ss = torch.from_numpy(seg_row).cuda(), torch.from_numpy(seg_slice).cuda()
            Wd = torch.from_numpy(W).cuda()
            out = torch.full((J, R), float("nan"), dtype=torch.float64, device="cuda")
            side.synchronize()
            stat = lib.dash_f_increment_noalloc(Xd.data_ptr(), Ud.data_ptr(), N, J, R, sr.data_ptr(),
                                                ss.data_ptr(), n_seg, Wd.data_ptr(), out.data_ptr(),
                                                C.c_void_p(side.cuda_stream))
            assert stat == 0
            side.synchronize()
        want = _oracle_f_inc(X.astype(np.float64), U.astype(np.float64), seg_row, seg_slice, W)
        err = float(np.max(np.abs(out.cpu().numpy() - want)) / np.max(np.abs(want)))
        assert err <= 1e-4, (N, J, R, err)


def test_noalloc_rejects_sizes_beyond_the_static_array():
    from paper_2305_18376_gb300 import _native
    lib = _native.load()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # J·R = 2^21 + 64·... beyond the 2^21-float array
    assert lib.dash_f_increment_noalloc(None, None, 0, (1 << 21) // 32 + 1, 64, None, None, 0,
                                        None, out.data_ptr(), None) == 2
    assert lib.dash_f_increment_noalloc(None, None, 0, 8, 65, None, None, 0, None,
                                        out.data_ptr(), None) == 1
