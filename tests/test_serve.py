"""Host logic of the continuous-batching server, with a fake batch backend
(no GPU): admission by memory budget, FIFO per qubit count, slots at
different layers advancing together, reuse of freed slots, rejection of
requests that cannot fit, and results routed to the right request."""
import numpy as np
import pytest

from paper_2411_15332_gb300 import inputs
from paper_2411_15332_gb300.serve import Request, Server, requests_from_workload


class FakeBatch:
    """Counts layers per slot; the 'result' of a slot is a function of the
    angles it saw, so misrouting shows up."""

    log = []

    def __init__(self, n, cap):
        self.n, self.cap = n, cap
        self.acc = np.zeros(cap)
        self.count = np.zeros(cap, dtype=int)
        FakeBatch.log.append(("create", n, cap))

    def reset(self, slots):
        for s in slots:
            assert 0 <= s < self.cap
            self.acc[s] = 0.0
            self.count[s] = 0

    def layer(self, slots, rows):
        assert rows.shape == (len(slots), 2, self.n)
        for s, r in zip(slots, rows):
            self.acc[s] += float(np.sum(r))
            self.count[s] += 1

    def observables(self, slots, q):
        return np.array([[1.0, self.acc[s], float(self.count[s])] for s in slots])


def _expected(req):
    return float(np.sum(req.theta))


def test_all_requests_complete_with_their_own_result():
    reqs = requests_from_workload(inputs.qnn_requests(60, seed=4, n_lo=5, n_hi=8, l_lo=2, l_hi=5))
    srv = Server(dtype="c64", mem_budget=1 << 20, slots_per_n=4, make_batch=FakeBatch)
    done = srv.run(reqs)
    assert len(done) == 60
    for r in done:
        assert r.error is None
        assert r.result == pytest.approx(_expected(r))
    st = srv.stats()
    assert st["circuits"] == 60 and st["p99_ms"] >= st["p50_ms"]


def test_memory_budget_limits_slots_and_rejects_oversize():
    FakeBatch.log = []
    # one slot of n=8 (c64) needs 2 * 256 * 8 = 4 KiB
    srv = Server(dtype="c64", mem_budget=3 * 4096, slots_per_n=16, make_batch=FakeBatch)
    reqs = [Request(rid=i, n=8, theta=np.full((3, 2, 8), 0.1 * i)) for i in range(7)]
    reqs.append(Request(rid=99, n=12, theta=np.zeros((1, 2, 12))))     # 64 KiB: never fits
    done = srv.run(reqs)
    assert ("create", 8, 3) in FakeBatch.log          # capacity cut to the budget
    bad = [r for r in done if r.rid == 99][0]
    assert bad.error and "memory" in bad.error
    good = [r for r in done if r.rid != 99]
    assert len(good) == 7 and all(r.result == pytest.approx(_expected(r)) for r in good)


def test_slots_at_different_layers_share_launches():
    srv = Server(dtype="c64", mem_budget=1 << 20, slots_per_n=8, make_batch=FakeBatch)
    a = Request(rid=0, n=6, theta=np.ones((6, 2, 6)))
    srv.submit(a)
    srv.tick()
    srv.tick()
    b = Request(rid=1, n=6, theta=2 * np.ones((2, 2, 6)))
    srv.submit(b)                        # joins while a is at layer 2
    launches_before = srv.launches
    srv.tick()                           # one layer launch for both (+ one reset)
    assert srv.launches - launches_before == 2
    while srv.active():
        srv.tick()
    assert a.result == pytest.approx(_expected(a)) and b.result == pytest.approx(_expected(b))
    assert b.done <= a.done              # the short late request finished first


def test_malformed_request_rejected():
    srv = Server(make_batch=FakeBatch)
    r = Request(rid=0, n=5, theta=np.zeros((2, 3, 5)))
    srv.submit(r)
    assert r.error is not None
