"""Host logic of the serving loop on the CPU (a fake engine, virtual clock):
admission by footprint within the HBM budget, FIFO or least-work-first
order, slot limit, every request finishes with the steps it asked for."""
import numpy as np
import pytest

import lpc_inputs
from paper_2603_22553_b300.serve import Server, serve_sequential, summary


class FakeLattice:
    def __init__(self, req):
        self.req = req
        self.done = 0
        self.closed = False

    def step(self, n):
        self.done += n


class FakeEngine:
    def __init__(self):
        self.live = {}
        self.peak_bytes = 0
        self.bytes = 0
        self.order = []
        self.batches = []

    def footprint(self, req):
        return req.edge ** 3 * 60

    def create(self, req):
        self.order.append(req.rid)
        self.bytes += self.footprint(req)
        self.peak_bytes = max(self.peak_bytes, self.bytes)
        lat = FakeLattice(req)
        self.live[req.rid] = lat
        return lat

    def step_many(self, lats, steps):
        assert len(lats) == len(steps) and all(s > 0 for s in steps)
        self.batches.append(len(lats))
        for l, s in zip(lats, steps):
            assert not l.closed
            l.step(s)

    def finish(self, lat):
        assert lat.done == lat.req.steps
        self.discard(lat)
        return np.arange(lat.done + 1, dtype=float)

    def discard(self, lat):
        lat.closed = True
        self.bytes -= self.footprint(lat.req)
        del self.live[lat.req.rid]


def _stream(n=60, seed=4, rate=2e5):
    reqs = lpc_inputs.request_stream(n=n, seed=seed, edge_lo=8, edge_hi=40, steps_lo=10, steps_hi=900,
                                     rate_per_s=rate)
    return reqs


@pytest.mark.parametrize("budget_edges,max_active", [(60, 8), (200, 48), (41, 3)])
def test_admission_budget_fifo_and_completion(budget_edges, max_active):
    reqs = _stream()
    eng = FakeEngine()
    budget = budget_edges ** 3 * 60
    srv = Server(eng, budget, max_active=max_active, quantum=100, prefetch=1)
    recs = srv.run(reqs, realtime=False)
    assert len(recs) == len(reqs)
    assert eng.peak_bytes <= budget
    assert not eng.live
    # FIFO: creation order is arrival order
    assert eng.order == [r.rid for r in sorted(reqs, key=lambda r: r.arrival_s)]
    assert max(eng.batches) <= max_active
    for r in recs:
        assert r.finish >= r.admit >= r.arrival
        assert len(r.fid) == r.steps + 1
    s = summary(recs)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_batching_overlaps_requests():
    reqs = _stream(40)
    eng = FakeEngine()
    Server(eng, 10 ** 12, max_active=48, quantum=50, prefetch=1).run(reqs, realtime=False)
    assert max(eng.batches) > 1


def test_request_above_budget_rejected():
    reqs = _stream(5)
    eng = FakeEngine()
    with pytest.raises(ValueError):
        Server(eng, 10, max_active=4).run(reqs, realtime=False)


def test_sequential_comparator_runs_in_order():
    reqs = _stream(10)
    eng = FakeEngine()
    recs = serve_sequential(eng, reqs, realtime=False)
    assert [r.rid for r in recs] == [r.rid for r in sorted(reqs, key=lambda r: r.arrival_s)]
    for a, b in zip(recs, recs[1:]):
        assert b.admit >= a.finish


def test_request_stream_recipe():
    reqs = lpc_inputs.request_stream()
    assert len(reqs) == 1000
    edges = np.array([r.edge for r in reqs])
    steps = np.array([r.steps for r in reqs])
    assert edges.min() >= 24 and edges.max() <= 192
    assert steps.min() >= 1000 and steps.max() <= 20000
    gaps = np.diff([r.arrival_s for r in reqs])
    assert np.all(gaps >= 0) and abs(gaps.mean() - 0.02) < 0.003


class FailingEngine(FakeEngine):
    """Creation of one request fails (as a device allocation might)."""

    def __init__(self, bad_rid):
        super().__init__()
        self.bad_rid = bad_rid

    def create(self, req):
        if req.rid == self.bad_rid:
            raise RuntimeError("creation failed")
        return super().create(req)


@pytest.mark.parametrize("prefetch", [1, 3])
def test_failed_creation_releases_every_lattice(prefetch):
    reqs = _stream(30)
    order = sorted(reqs, key=lambda r: r.arrival_s)
    eng = FailingEngine(order[12].rid)
    with pytest.raises(RuntimeError, match="creation failed"):
        Server(eng, 10 ** 12, max_active=8, quantum=50, prefetch=prefetch).run(reqs, realtime=False)
    # resident lattices and those created after the failure were destroyed
    assert eng.order and not eng.live and eng.bytes == 0


def test_sjf_admits_the_least_work_first_and_ages():
    """policy="sjf": among the requests waiting at an admission, the one with
    the least work (sites x steps) goes first; with max_wait_s a request that
    waited that long goes before shorter ones.  Every request still runs its
    steps, and the slot limit holds."""
    reqs = [lpc_inputs.Request(i, 0.0, e, s, 100 + i) for i, (e, s) in
            enumerate([(30, 900), (8, 20), (20, 100), (9, 10), (40, 500), (10, 30)])]
    eng = FakeEngine()
    recs = Server(eng, 1 << 40, max_active=1, quantum=50, prefetch=1, policy="sjf").run(reqs, realtime=False)
    work = {r.rid: r.edge ** 3 * r.steps for r in reqs}
    assert eng.order == sorted(work, key=lambda k: (work[k], k))
    assert all(r.finish >= r.arrival for r in recs)
    # aging: with a virtual clock advancing by the work done, the longest
    # request (arrived first) passes the queue once it has waited max_wait_s
    eng2 = FakeEngine()
    Server(eng2, 1 << 40, max_active=1, quantum=50, prefetch=1, policy="sjf", max_wait_s=1e-8).run(
        reqs, realtime=False)
    assert eng2.order[0] == 3 and eng2.order[1] == 0     # at t = 0 nobody has waited; then rid 0 has
    with pytest.raises(ValueError):
        Server(eng, 1 << 40, policy="lifo")
