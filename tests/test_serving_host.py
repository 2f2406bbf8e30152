"""Host logic of the serving loop (paper_2305_18376_gb300.serving) with fake
models: admission by device-memory budget, per-stream order, the in-flight
limit, retirement of finished streams, head-of-line avoidance, and the
latency summary.  No GPU: the fakes finish after a fixed number of polls."""
import numpy as np
import pytest

from paper_2305_18376_gb300.serving import Request, ServingError, ServingLoop, latency_summary


class NumericFailure(RuntimeError):
    status = 5


class FakeModel:
    def __init__(self, J, R, lam, nbytes=0, polls=2, fail_at=None, **kw):
        self.J, self.R, self.nbytes, self.polls = J, R, nbytes, polls
        self.fail_at = fail_at
        self.busy = 0
        self.work = []
        self.closed = False

    def device_bytes(self):
        return self.nbytes

    def append_batch(self, ids, rp, X):
        assert not self.busy, "work issued to a busy model"
        self.work.append(("append", int(np.asarray(rp)[-1])))

    def fit_initial(self, n):
        self.work.append(("init", n))
        self.busy = self.polls

    def update(self):
        if self.fail_at is not None and sum(w[0] == "update" for w in self.work) == self.fail_at:
            raise NumericFailure("non-finite factors")
        self.work.append(("update",))
        self.busy = self.polls

    def idle(self):
        if self.busy:
            self.busy -= 1
            return False
        return True

    def close(self):
        self.closed = True


def _req(s, t, kind="update", rows=3):
    return Request(stream=s, arrival=t, kind=kind, slice_ids=[0], row_ptr=[0, rows],
                   X=np.zeros((rows, 2), np.float32), rows=rows)


def _loop(nbytes, budget, max_inflight=2, polls=2):
    specs = {s: dict(J=2, R=1, lam=1.0, nbytes=b, polls=polls) for s, b in nbytes.items()}
    retired = {}
    loop = ServingLoop(specs, budget, max_inflight, factory=FakeModel,
                       bytes_of=lambda spec: spec["nbytes"],
                       on_retire=lambda s, m: retired.setdefault(s, m), poll_sleep=0)
    return loop, retired


def _check_invariants(loop, reqs):
    ev = sorted(loop.events, key=lambda e: e[0])
    running, resident = 0, 0
    for _, what, s in ev:
        running += {"admit": 1, "done": -1}.get(what, 0)
        assert running <= loop.max_inflight
    assert loop.peak_resident <= loop.budget
    by_stream = {}
    for r in reqs:
        assert r.done is not None and r.admitted is not None
        assert r.admitted >= 0 and r.done >= r.admitted
        by_stream.setdefault(r.stream, []).append(r)
    for s, rs in by_stream.items():          # a stream's requests run one at a time, in order
        rs.sort(key=lambda r: r.arrival)
        for a, b in zip(rs, rs[1:]):
            assert b.admitted >= a.done


def test_budget_order_inflight_and_retirement():
    nbytes = {s: 5 for s in range(6)}
    loop, retired = _loop(nbytes, budget=10, max_inflight=2)
    reqs = []
    for s in range(6):
        reqs.append(_req(s, 0.0, "init"))
    for t in range(1, 4):
        for s in range(6):
            reqs.append(_req(s, 0.001 * t, "update", rows=t))
    loop.run(reqs, realtime=False)
    _check_invariants(loop, reqs)
    assert loop.peak_resident == 10                       # two models at a time
    assert len(loop.retired) >= 4                        # streams made room for later ones
    loop.close()
    assert sorted(retired) == list(range(6))
    for s, m in retired.items():
        assert m.closed
        kinds = [w[0] for w in m.work if w[0] != "append"]
        assert kinds == ["init", "update", "update", "update"]


def test_waiting_stream_does_not_block_resident_ones():
    # A (6) and B (6) cannot be resident together; C (3) fits beside A.
    loop, _ = _loop({0: 6, 1: 6, 2: 3}, budget=10, max_inflight=4, polls=3)
    reqs = [_req(0, 0.0, "init"), _req(1, 0.0, "init"), _req(2, 0.0, "init"),
            _req(0, 0.0), _req(2, 0.0), _req(2, 0.0)]
    loop.run(reqs, realtime=False)
    _check_invariants(loop, reqs)
    b_init = reqs[1]
    c_reqs = [r for r in reqs if r.stream == 2]
    a_last = max(r.done for r in reqs if r.stream == 0)
    assert c_reqs[0].admitted < b_init.admitted          # C went ahead of the waiting B
    assert b_init.admitted >= a_last                     # B entered once A had finished and left
    assert 0 in loop.retired


def test_stream_larger_than_the_budget_is_an_error():
    loop, _ = _loop({0: 20}, budget=10)
    with pytest.raises(ServingError):
        loop.run([_req(0, 0.0, "init")], realtime=False)


def test_realtime_arrivals_are_respected():
    loop, _ = _loop({0: 1, 1: 1}, budget=10, max_inflight=2, polls=1)
    reqs = [_req(0, 0.0, "init"), _req(1, 0.0, "init"), _req(0, 0.02), _req(1, 0.03)]
    loop.run(reqs, realtime=True)
    _check_invariants(loop, reqs)
    for r in reqs:
        assert r.admitted >= r.arrival


def test_latency_summary():
    rs = [_req(0, 0.0, rows=10), _req(0, 1.0, rows=30)]
    rs[0].admitted, rs[0].done = 0.0, 0.5
    rs[1].admitted, rs[1].done = 1.0, 2.0
    out = latency_summary(rs)
    assert out["requests"] == 2 and out["rows"] == 40
    assert out["p50_ms"] == pytest.approx(750.0)
    assert out["rows_per_s"] == pytest.approx(20.0)


def test_non_final_run_keeps_models_for_the_next_run():
    """A run with final=False retires nothing, so a stream fitted in it keeps
    its model for its updates in the next run; a request that cannot fit
    without retiring is an error instead of a silent restart."""
    loop, retired = _loop({0: 40, 1: 40}, budget=100)
    loop.run([_req(0, 0.0, "init"), _req(1, 0.0, "init")], realtime=False, final=False)
    assert not retired and set(loop.models) == {0, 1}
    m0 = loop.models[0]
    loop.run([_req(0, 0.0), _req(1, 0.0)], realtime=False)
    assert loop.models.get(0, m0) is m0 or retired.get(0) is m0
    assert [w[0] for w in m0.work] == ["append", "init", "append", "update"]
    loop2, retired2 = _loop({0: 60, 1: 60}, budget=100)
    with pytest.raises(ServingError):
        loop2.run([_req(0, 0.0, "init"), _req(1, 0.0, "init")], realtime=False, final=False)


def test_a_numerical_failure_stops_only_its_stream():
    """A stream whose update reports a non-finite state (DASH_ENUMERIC) is
    stopped: that request and its later ones are marked failed, its model
    is closed and its memory released; the other streams are served."""
    specs = {0: dict(J=2, R=1, lam=1.0, nbytes=10, polls=1, fail_at=1),
             1: dict(J=2, R=1, lam=1.0, nbytes=10, polls=1)}
    loop = ServingLoop(specs, 100, 4, factory=FakeModel, bytes_of=lambda spec: spec["nbytes"],
                       poll_sleep=0)
    reqs = [_req(0, 0.0, "init"), _req(1, 0.0, "init")]
    reqs += [_req(s, 0.001 * t) for t in range(1, 5) for s in (0, 1)]
    loop.run(reqs, realtime=False)
    ok0 = [r for r in reqs if r.stream == 0 and r.kind == "update"]
    assert [r.done is not None for r in ok0] == [True, False, False, False]
    assert all(r.failed for r in ok0[1:]) and 0 in loop.failed
    assert all(r.done is not None and not r.failed for r in reqs if r.stream == 1)
    assert 0 not in loop.models and loop.resident == loop.model_bytes.get(1, 0)
