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


class FakeClock:
    """Deterministic server clock: every reading advances it by ``dt``."""

    def __init__(self, dt=2e-4):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_arrivals_are_honoured_and_latencies_non_negative():
    """Poisson arrivals: no request is submitted, admitted or finished
    before its arrival offset, every latency is >= 0, and the run lasts at
    least as long as the arrival window (so the throughput cannot exceed
    the offered rate over that window)."""
    rate = 500.0
    reqs = requests_from_workload(inputs.qnn_requests(40, seed=4, n_lo=5, n_hi=7, l_lo=2, l_hi=4), rate=rate)
    window = max(r.arrival for r in reqs)
    assert window > 0.02
    srv = Server(dtype="c64", mem_budget=1 << 20, slots_per_n=4, make_batch=FakeBatch, clock=FakeClock())
    done = srv.run(reqs)
    assert len(done) == 40
    for r in done:
        assert r.error is None
        assert r.admitted >= r.arrival
        assert r.done >= r.admitted
        assert r.latency >= 0.0
    st = srv.stats()
    assert st["seconds"] >= window
    assert st["circuits_per_s"] <= 40 / window


def test_largest_qubit_count_after_smaller_groups_is_not_starved():
    """Groups are sized at first use; a later, larger qubit count that no
    longer fits takes the memory of idle groups instead of waiting forever."""
    FakeBatch.log = []
    # n=8 slot: 4 KiB; n=10 slot: 16 KiB; budget 64 KiB
    srv = Server(dtype="c64", mem_budget=64 * 1024, slots_per_n=16, make_batch=FakeBatch, clock=FakeClock())
    small = [Request(rid=i, n=n, theta=np.full((2, 2, n), 0.01 * i)) for i, n in enumerate((8, 9, 8, 9, 8, 9))]
    done = srv.run(small, timeout=5.0)
    assert len(done) == 6
    assert srv.used_bytes() > 64 * 1024 - 16 * 1024     # the small groups hold the budget
    big = Request(rid=100, n=10, theta=np.full((3, 2, 10), 0.5))
    done = srv.run([big], timeout=5.0)
    assert done == [big]
    assert big.error is None and big.result == pytest.approx(_expected(big))
    assert any(e[0] == "create" and e[1] == 10 for e in FakeBatch.log)
