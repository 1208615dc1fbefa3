"""Workload accounting used by the benchmark: algorithmic amplitude updates
and bytes of a gate list, from the library's own gate catalogue.

An amplitude update is one amplitude rewritten by one gate: a gate on k
targets with c controls rewrites N / 2^c * (changed rows) / 2^k amplitudes,
where a changed row is a row of its matrix that differs from the identity's
(RZ and H change both rows, Z / S / T one, SWAP two of four, a sign flip of
one basis state changes one amplitude).
"""
from __future__ import annotations

import numpy as np

_cache = {}


def changed_rows(name: str, params=()) -> tuple:
    from .core import gate_matrix
    key = (name, tuple(params))
    if key not in _cache:
        if name == "FLIP":
            _cache[key] = (1, 0)
        else:
            M = gate_matrix(name, params)
            I = np.eye(M.shape[0])
            k = int(round(np.log2(M.shape[0])))
            _cache[key] = (int(np.sum(np.any(M != I, axis=1))), k)
    return _cache[key]


def amplitude_updates(ops, n: int) -> float:
    N = float(1 << n)
    total = 0.0
    for name, targets, controls, params, _cv in ops:
        rows, k = changed_rows(name, params if name in ("RX", "RY", "RZ", "P", "U1", "R", "U", "U2", "U3",
                                                        "RXX", "RYY", "RZZ", "RZX") else ())
        total += N / float(1 << len(controls)) * rows / float(1 << k)
    return total
