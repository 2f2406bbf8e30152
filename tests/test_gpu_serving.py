"""The serving loop on the GPU (configuration of many independent streams,
J ∈ {64, 128, 256}, R ∈ {8, 16, 32}, serving-style updates: a random
fraction of the slices touched with 1-256 rows each plus a few new slices),
scaled so that the FP64 oracle finishes in seconds.

* Each stream's final state is the same, bit for bit, alone and in the mix
  (requests of several streams in flight at once, models created and retired
  under a device-memory budget).
* Each stream's state matches the FP64 oracle (Algorithm 1 after the static
  initial fit) within the path's tolerance: 1e-10 for FP64 products, 1e-4
  for the mixed products.
* A model owns exactly the device bytes dash_config_bytes predicts.
"""
import numpy as np
import pytest
import torch

from oracle import dash_oracle as O
from synth.planted import PlantedStream
from synth.serving import serving_load
from tests._parity import TOL, compare_state_p, segs_np

pytestmark = pytest.mark.gpu

INIT_ITERS = 2
KEYS = "VWcDFG"
# per stream (J, R, updates): (256, 8, 1), (128, 32, 2), (64, 16, 2), (128, 8, 6), (128, 8, 1)
PRECS = ["f16x3", "f16x3", "fp64", "f16x3", "fp64"]


def _load():
    load = serving_load(n_streams=5, duration=0.010, rate=1000.0, K0_range=(12, 30),
                        init_rows=("uniform", 40, 160), new_slices=("uniform", 0, 4))
    streams = []
    for s, w in enumerate(load.streams):
        prec = PRECS[s]
        tdt = torch.float64 if prec == "fp64" else torch.float32
        ps = PlantedStream(w)
        batches = [ps.batch(t) for t in range(w.steps + 1)]
        spec = dict(J=w.J, R=w.R, lam=w.lam, precision=prec,
                    input_dtype="f64" if prec == "fp64" else "f32",
                    max_slices=ps.K_total + 8,
                    max_rows=max(b.n_rows for b in batches) + 16,
                    max_segments=max(b.slice_ids.numel() for b in batches) + 8)
        V0 = np.random.default_rng(100 + s).random((w.J, w.R))
        streams.append(dict(w=w, prec=prec, tdt=tdt, batches=batches, spec=spec, V0=V0))
    return load, streams


def _alone(st):
    from paper_2305_18376_gb300 import DashModel
    from paper_2305_18376_gb300._native import config_bytes
    m = DashModel(**st["spec"])
    assert m.device_bytes() == config_bytes(**st["spec"])[0]
    m.set_factors(st["V0"])
    b0 = st["batches"][0]
    m.append_batch(b0.slice_ids.numpy(), b0.row_ptr.numpy(), b0.X.to(st["tdt"]).numpy())
    m.fit_initial(INIT_ITERS)
    for b in st["batches"][1:]:
        m.append_batch(b.slice_ids.numpy(), b.row_ptr.numpy(), b.X.to(st["tdt"]).numpy())
        m.update()
    m.sync()
    out = m.get_state_p()
    m.close()
    return out


def _oracle(st):
    w = st["w"]
    b0 = st["batches"][0]
    X0 = [x for _, x in segs_np(b0, st["tdt"])]
    U, W, V = O.static_als_p(X0, st["V0"], np.ones((len(X0), w.R)), INIT_ITERS)
    state = O.init_helpers_p(X0, U, W, V)
    for b in st["batches"][1:]:
        X = O._group(segs_np(b, st["tdt"]), state.K, b.n_new, w.J)
        state, _ = O.dash_update_p(state, list(X.items()), b.n_new, w.lam)
    return state


def test_serving_mix_equals_alone_and_matches_the_oracle():
    from paper_2305_18376_gb300.serving import Request, ServingLoop, latency_summary
    from paper_2305_18376_gb300._native import config_bytes
    load, streams = _load()
    alone = [_alone(st) for st in streams]

    # the mix: every request arrives at its Poisson time, as a burst; at most
    # three streams' models fit the budget, four requests run at once
    sizes = sorted(config_bytes(**st["spec"])[0] for st in streams)
    budget = sum(sizes[-3:])
    specs = {s: st["spec"] for s, st in enumerate(streams)}
    finals = {}
    loop = ServingLoop(specs, budget, max_inflight=4,
                       prepare=lambda s, m: m.set_factors(streams[s]["V0"]),
                       on_retire=lambda s, m: finals.setdefault(s, m.get_state_p()))
    reqs = []
    for s, st in enumerate(streams):
        b0 = st["batches"][0]
        reqs.append(Request(stream=s, arrival=0.0, kind="init", slice_ids=b0.slice_ids.numpy(),
                            row_ptr=b0.row_ptr.numpy(), X=b0.X.to(st["tdt"]).numpy(),
                            init_iters=INIT_ITERS, rows=b0.n_rows))
    for (t_arr, s, t) in load.arrivals:
        st = streams[s]
        b = st["batches"][t]
        reqs.append(Request(stream=s, arrival=t_arr, kind="update", slice_ids=b.slice_ids.numpy(),
                            row_ptr=b.row_ptr.numpy(), X=b.X.to(st["tdt"]).numpy(), rows=b.n_rows))
    loop.run(reqs, realtime=False)
    loop.close()
    print("serving mix:", latency_summary(reqs), "peak resident", loop.peak_resident, "of", budget)
    assert loop.peak_resident <= budget
    assert sorted(finals) == list(range(len(streams)))
    assert len(loop.retired) == len(streams)
    # admissions overlapped: some request was admitted while another ran
    ev = sorted(loop.events, key=lambda e: e[0])
    running, most = 0, 0
    for _, what, _ in ev:
        running += {"admit": 1, "done": -1}.get(what, 0)
        most = max(most, running)
    assert most >= 2

    for s, st in enumerate(streams):
        for k in KEYS:
            assert np.array_equal(finals[s][k], alone[s][k]), (s, k)
        ref = _oracle(st)
        errs = compare_state_p(alone[s], ref, TOL[st["prec"]], f"stream {s} ({st['prec']})")
        print(f"  stream {s}: J={st['w'].J} R={st['w'].R} K={ref.K} {st['prec']}", errs)
