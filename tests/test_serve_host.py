"""Host logic of the continuous-batching server, with fake pools (no GPU):
admission by memory budget and per-pool limits, rejection on a full queue,
requests joining while others are in flight, and batching across depths."""
import threading
import time

import numpy as np
import pytest

from paper_2509_01253_gb300 import serve


class FakeClient:
    def __init__(self, rounds):
        self.rounds = rounds
        self.round = 0

    @property
    def done(self):
        return self.round >= self.rounds

    def logits(self):
        return np.array([float(self.round)])


class FakePool:
    """Stands in for a device pool: each 'round' takes `round_s` seconds."""

    def __init__(self, rounds: dict, reserve: dict, round_s: float = 0.01):
        self.rounds, self.reserves, self.round_s = rounds, reserve, round_s
        self.calls = []            # per engine call: [(rid, round)]
        self.lock = threading.Lock()

    def reserve_of(self, net):
        return self.reserves[net]

    def new_client(self, req):
        return FakeClient(self.rounds[req.net])

    def bind_thread(self):
        pass

    def prepare(self, req):
        req.d_in = ("in", req.rid, req.client.round)

    def evaluate(self, batch):
        assert all(req.d_in == ("in", req.rid, req.client.round) for req in batch)
        with self.lock:
            self.calls.append([(req.rid, req.client.round) for req in batch])
        time.sleep(self.round_s)

    def absorb(self, req):
        req.client.round += 1
        req.rounds_run += 1


def _req(i, net="a"):
    return serve.Request(i, net, 0, np.zeros(1), session_seed=i, request_seed=i)


def _wait_idle(srv, limit=10.0):
    t = time.perf_counter() + limit
    while not srv.idle() and time.perf_counter() < t:
        time.sleep(0.005)
    assert srv.idle()


def test_all_admitted_requests_complete_every_round():
    pool = FakePool({"a": 3, "b": 5}, {"a": 10, "b": 10})
    srv = serve.Server({"p": pool}, {"a": "p", "b": "p"}, mem_budget=1000, max_active=4, max_batch=8)
    srv.start()
    for i in range(10):
        assert srv.submit(_req(i, "a" if i % 2 else "b"))
    _wait_idle(srv)
    srv.shutdown()
    assert len(srv.completed) == 10 and not srv.rejected
    for r in srv.completed:
        assert r.rounds_run == (3 if r.net == "a" else 5)
        assert r.logits[0] == r.rounds_run
    # every round of every request ran exactly once, in order
    seen = {}
    for call in pool.calls:
        assert len({rid for rid, _ in call}) == len(call)      # one round per request per call
        for rid, rnd in call:
            assert seen.get(rid, -1) == rnd - 1
            seen[rid] = rnd
    assert max(len(c) for c in pool.calls) <= 4               # max_active


def test_queue_full_rejects_and_budget_limits_admission():
    pool = FakePool({"a": 2}, {"a": 60}, round_s=0.05)
    srv = serve.Server({"p": pool}, {"a": "p"}, mem_budget=100, max_queue=2, max_active=8)
    srv.start()
    ok = [srv.submit(_req(i)) for i in range(6)]
    # budget 100 admits one request (60 each); queue holds 2; the other 3 are rejected
    assert ok == [True, True, True, False, False, False]
    assert len(srv.rejected) == 3
    _wait_idle(srv)
    srv.shutdown()
    assert len(srv.completed) == 3
    # the budget allowed one request in flight at a time
    assert max(len(c) for c in pool.calls) == 1


def test_late_arrivals_join_calls_with_requests_at_other_depths():
    pool = FakePool({"a": 6}, {"a": 1}, round_s=0.03)
    srv = serve.Server({"p": pool}, {"a": "p"}, mem_budget=100, max_active=8)
    srv.start()
    srv.submit(_req(0))
    time.sleep(0.08)                  # request 0 is a few rounds in
    srv.submit(_req(1))
    _wait_idle(srv)
    srv.shutdown()
    mixed = [c for c in pool.calls if len(c) == 2]
    assert mixed, "the late request never shared an engine call"
    assert any(dict(c)[0] != dict(c)[1] for c in mixed)   # different depths in one call


def test_batch_cap_rotates_requests():
    pool = FakePool({"a": 4}, {"a": 1}, round_s=0.005)
    srv = serve.Server({"p": pool}, {"a": "p"}, mem_budget=100, max_active=6, max_batch=2)
    srv.start()
    for i in range(6):
        srv.submit(_req(i))
    _wait_idle(srv)
    srv.shutdown()
    assert len(srv.completed) == 6
    assert max(len(c) for c in pool.calls) <= 2


def test_worker_error_surfaces_on_shutdown():
    class Broken(FakePool):
        def evaluate(self, batch):
            raise ValueError("device failure")
    pool = Broken({"a": 2}, {"a": 1})
    srv = serve.Server({"p": pool}, {"a": "p"}, mem_budget=100)
    srv.start()
    srv.submit(_req(0))
    time.sleep(0.1)
    with pytest.raises(RuntimeError, match="device failure"):
        srv.shutdown()


def test_poisson_arrivals_are_seeded_and_mixed():
    a = serve.poisson_arrivals(50.0, 4.0, {"x": 0.7, "y": 0.3}, 4, seed=3)
    b = serve.poisson_arrivals(50.0, 4.0, {"x": 0.7, "y": 0.3}, 4, seed=3)
    assert a == b
    assert 120 < len(a) < 280
    frac = sum(1 for _, n, _, _ in a if n == "x") / len(a)
    assert 0.55 < frac < 0.85
    assert {k for _, _, k, _ in a} <= {0, 1, 2, 3}
    assert all(t1 < t2 for (t1, *_), (t2, *_) in zip(a, a[1:]))
