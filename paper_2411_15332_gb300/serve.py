"""Continuous-batching server for QNN ansatz circuits.

A request is (n, theta[L, 2, n]); its result is <Z_0> (float64) of the
ansatz state.  The server keeps one batch (``Batch``) per qubit count n.
Requests are admitted into free slots while the device-memory budget
allows, and wait in a FIFO queue otherwise.  Every tick advances every
active slot of a group by one layer in a single launch -- slots sit at
different layers of different circuits -- so requests that arrive while
others run join at the next tick.  A finished circuit is read out, its
slot is freed and immediately reused.  Each circuit's result is the same
alone and in any mix (per-slot arithmetic and reductions do not depend on
the other rows).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    n: int
    theta: np.ndarray                 # [L, 2, n]
    arrival: float = 0.0              # seconds (server clock)
    admitted: Optional[float] = None
    done: Optional[float] = None
    result: Optional[float] = None
    error: Optional[str] = None

    @property
    def layers(self) -> int:
        return int(self.theta.shape[0])

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


@dataclass
class _Group:
    n: int
    batch: object
    capacity: int
    free: List[int] = field(default_factory=list)
    active: Dict[int, Request] = field(default_factory=dict)   # slot -> request
    layer: Dict[int, int] = field(default_factory=dict)        # slot -> next layer


class Server:
    """make_batch(n, capacity) -> object with reset(slots), layer(slots,
    theta_rows) and observables(slots, q); the default builds a CUDA
    ``Batch``.  ``mem_budget`` bounds the bytes of all batches (two states
    per slot: the state and its adjoint work state)."""

    def __init__(self, dtype: str = "c64", mem_budget: int = 8 << 30, slots_per_n: int = 256,
                 make_batch: Optional[Callable] = None, clock: Callable[[], float] = time.perf_counter):
        self.dtype = dtype
        self.elem = 16 if dtype == "c128" else 8
        self.mem_budget = int(mem_budget)
        self.slots_per_n = int(slots_per_n)
        self.clock = clock
        if make_batch is None:
            from .qnn import Batch

            def make_batch(n, cap):
                return Batch(n, cap, dtype)
        self.make_batch = make_batch
        self.groups: Dict[int, _Group] = {}
        self.queue: collections.deque = collections.deque()
        self.finished: List[Request] = []
        self.ticks = 0
        self.launches = 0
        self.t0 = clock()

    # -- memory ------------------------------------------------------------
    def _group_bytes(self, n: int, cap: int) -> int:
        return 2 * cap * (1 << n) * self.elem

    def used_bytes(self) -> int:
        return sum(self._group_bytes(g.n, g.capacity) for g in self.groups.values())

    def _release_idle(self, keep: int) -> bool:
        """Free the batches of groups with no active slot (other than qubit
        count ``keep``), so that their memory can go to a qubit count that
        does not fit; returns whether anything was freed."""
        idle = [m for m, g in self.groups.items() if m != keep and not g.active]
        for m in idle:
            g = self.groups.pop(m)
            close = getattr(g.batch, "close", None)
            if close is not None:
                close()
        return bool(idle)

    def _group(self, n: int) -> Optional[_Group]:
        g = self.groups.get(n)
        if g is not None:
            return g
        per_slot = self._group_bytes(n, 1)
        room = (self.mem_budget - self.used_bytes()) // per_slot
        want = min(self.slots_per_n, self.mem_budget // per_slot)
        if room < want and self._release_idle(n):
            # groups sized for earlier qubit counts would otherwise hold the
            # budget forever: idle ones give their memory back
            room = (self.mem_budget - self.used_bytes()) // per_slot
        cap = int(min(self.slots_per_n, room))
        if cap < 1:
            return None
        g = _Group(n=n, batch=self.make_batch(n, cap), capacity=cap, free=list(range(cap - 1, -1, -1)))
        self.groups[n] = g
        return g

    # -- requests ----------------------------------------------------------
    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request):
        if req.theta.ndim != 3 or req.theta.shape[1:] != (2, req.n):
            req.error = "theta must have shape [L, 2, n]"
            req.done = self.now()
            self.finished.append(req)
            return
        if self._group_bytes(req.n, 1) > self.mem_budget:
            req.error = "request does not fit in the memory budget"
            req.done = self.now()
            self.finished.append(req)
            return
        self.queue.append(req)

    def _admit(self) -> Dict[int, List[int]]:
        """Admit queued requests into free slots; returns the slots to reset
        per group.  FIFO per qubit count; a request whose group is full
        waits without blocking other qubit counts."""
        fresh: Dict[int, List[int]] = collections.defaultdict(list)
        waiting = collections.deque()
        while self.queue:
            req = self.queue.popleft()
            g = self._group(req.n)
            if g is None or not g.free:
                waiting.append(req)
                continue
            slot = g.free.pop()
            g.active[slot] = req
            g.layer[slot] = 0
            req.admitted = self.now()
            fresh[req.n].append(slot)
        self.queue = waiting
        return fresh

    def tick(self) -> int:
        """Admit, advance every active slot by one layer, retire finished
        circuits.  Returns the number of active circuits after the tick."""
        fresh = self._admit()
        for n, slots in fresh.items():
            self.groups[n].batch.reset(slots)
            self.launches += 1
        for g in self.groups.values():
            if not g.active:
                continue
            slots = sorted(g.active)
            rows = np.stack([g.active[s].theta[g.layer[s]] for s in slots])
            g.batch.layer(slots, rows)
            self.launches += 1
            done = []
            for s in slots:
                g.layer[s] += 1
                if g.layer[s] >= g.active[s].layers:
                    done.append(s)
            if done:
                obs = g.batch.observables(done, 0)
                self.launches += 1
                t = self.now()
                for s, row in zip(done, obs):
                    req = g.active.pop(s)
                    del g.layer[s]
                    req.result = float(row[1])
                    req.done = t
                    self.finished.append(req)
                    g.free.append(s)
        self.ticks += 1
        return sum(len(g.active) for g in self.groups.values())

    def active(self) -> int:
        return sum(len(g.active) for g in self.groups.values())

    def run(self, requests: List[Request], timeout: float = 600.0):
        """Serve ``requests``: each is submitted once the server clock
        (seconds since this call) reaches its ``arrival`` offset (all at
        once when every offset is 0).  Returns the requests of this call,
        finished, in completion order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = self.clock()
        total = len(pending)
        base = len(self.finished)
        while len(self.finished) - base < total:
            now = self.now()
            if now > timeout:
                raise TimeoutError(f"serving did not finish in {timeout} s")
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            if not self.queue and not self.active():
                if pending:
                    time.sleep(max(0.0, min(0.001, pending[0].arrival - now)))
                continue
            self.tick()
        return self.finished[base:]

    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.finished if r.error is None and r.latency is not None])
        ok = len(lat)
        span = max((r.done for r in self.finished if r.done is not None), default=0.0)
        return {"circuits": ok, "errors": sum(r.error is not None for r in self.finished),
                "seconds": span, "circuits_per_s": ok / span if span > 0 else None,
                "p50_ms": float(np.percentile(lat, 50) * 1e3) if ok else None,
                "p99_ms": float(np.percentile(lat, 99) * 1e3) if ok else None,
                "ticks": self.ticks, "launches": self.launches}


def requests_from_workload(reqs, rate: Optional[float] = None) -> List[Request]:
    """Requests of ``inputs.qnn_requests``; arrival offsets are the cumulative
    exponential gaps divided by ``rate`` (None: all at time 0)."""
    out, t = [], 0.0
    for r in reqs:
        if rate:
            t += r["gap"] / rate
        out.append(Request(rid=r["id"], n=r["n"], theta=np.asarray(r["theta"], dtype=np.float64),
                           arrival=t if rate else 0.0))
    return out
