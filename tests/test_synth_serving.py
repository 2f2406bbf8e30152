"""The serving input generator (synth.serving) and the serving options of
the planted streams (touched fraction, drawn new-slice counts): seeded,
consistent CSR batches, and arrivals that match each stream's update count.
Inputs only: none of this is Dash arithmetic."""
import torch

from synth.planted import PlantedStream, scaled, workload
from synth.serving import serving_load


def test_serving_load_is_seeded_and_consistent():
    a = serving_load(n_streams=6, duration=0.02, rate=1500.0, K0_range=(10, 20))
    b = serving_load(n_streams=6, duration=0.02, rate=1500.0, K0_range=(10, 20))
    assert a.arrivals == b.arrivals
    assert [w.J for w in a.streams] == [w.J for w in b.streams]
    times = [t for t, _, _ in a.arrivals]
    assert times == sorted(times) and 0 < times[0] and times[-1] <= 0.02
    for s, w in enumerate(a.streams):
        mine = [t for _, s2, t in a.arrivals if s2 == s]
        assert mine == list(range(1, w.steps + 1))
        assert w.J in (64, 128, 256) and w.R in (8, 16, 32) and 10 <= w.K0 <= 20


def test_touched_fraction_and_drawn_new_slices_give_valid_batches():
    w = scaled(workload("c3", K0=30, J=16, R=4, steps=6), touch=("uniform", 0.0, 1.0),
               new_slices_dist=("uniform", 0, 5), rows_per_step=("uniform", 1, 256),
               new_slice_rows=("uniform", 1, 256), sigma=0.0)
    s = PlantedStream(w)
    K = 0
    for t in range(w.steps + 1):
        b = s.batch(t)
        ids = b.slice_ids
        assert b.K_before == K
        assert torch.all(ids[1:] > ids[:-1])                         # one segment per slice
        new = ids[ids >= b.K_before]
        assert torch.equal(new, torch.arange(b.K_before, b.K_before + b.n_new))
        rows = b.row_ptr[1:] - b.row_ptr[:-1]
        if t > 0:
            assert torch.all(rows[ids < b.K_before] > 0)              # only touched old slices listed
            assert b.n_new == s.L_t[t] and 0 <= b.n_new <= 5
        assert int(b.row_ptr[-1]) == b.n_rows
        K = b.K_before + b.n_new if t else b.n_new
    assert s.K_total == K
