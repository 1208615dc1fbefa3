"""Seeded synthetic workloads: gate lists, angles, request mixes.

This module holds no simulation arithmetic.  It only draws random numbers
(numpy PCG64 via ``default_rng``) and writes them down as gate lists, so
that the CPU oracle and the CUDA library consume identical inputs.

An operation is a tuple ``(name, targets, controls, params, ctrl_values)``:

* ``name``     gate name from the catalogue (``"X"``, ``"RZ"``, ``"SWAP"``,
               ``"FLIP"`` ...).  ``FLIP`` is the sign flip of the basis
               states selected by its controls (no targets).
* ``targets``  tuple of qubit indices; the first listed target is the most
               significant bit of the gate's sub-index.
* ``controls`` tuple of control qubits.
* ``params``   tuple of floats (rotation angles).
* ``ctrl_values`` integer; bit ``j`` is the value control ``controls[j]``
               must hold (default: all ones).

Qubit ``q`` is bit ``q`` of the basis index (LSB = qubit 0).

Workload shapes follow the paper's case studies (sparse-gate random
circuits, Sec. IV-B; Hadamard-heavy Grover search, Table IV; QNN ansatz,
Table III) with the sizes fixed in the configuration list below.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

Op = Tuple[str, Tuple[int, ...], Tuple[int, ...], Tuple[float, ...], int]

TWO_PI = 2.0 * math.pi

# Gate names of the random-circuit workload (13 gates).
RANDOM_GATES = ("X", "Y", "Z", "S", "T", "CNOT", "CZ", "SWAP", "TOFFOLI",
                "RZ", "H", "RX", "RY")


def op(name, targets=(), controls=(), params=(), ctrl_values=None) -> Op:
    controls = tuple(int(c) for c in controls)
    if ctrl_values is None:
        ctrl_values = (1 << len(controls)) - 1
    return (name, tuple(int(t) for t in targets), controls,
            tuple(float(p) for p in params), int(ctrl_values))


def random_circuit(n: int = 10, n_gates: int = 200, seed: int = 1) -> List[Op]:
    """Random sparse-gate circuit: each gate uniform over RANDOM_GATES, its
    qubits uniform and distinct, angles uniform on [0, 2*pi)."""
    rng = np.random.default_rng(seed)
    ops: List[Op] = []
    for _ in range(n_gates):
        g = RANDOM_GATES[int(rng.integers(0, len(RANDOM_GATES)))]
        if g in ("X", "Y", "Z", "S", "T", "H"):
            q = rng.choice(n, size=1, replace=False)
            ops.append(op(g, (q[0],)))
        elif g in ("RX", "RY", "RZ"):
            q = rng.choice(n, size=1, replace=False)
            ops.append(op(g, (q[0],), (), (rng.uniform(0.0, TWO_PI),)))
        elif g == "CNOT":
            q = rng.choice(n, size=2, replace=False)
            ops.append(op("X", (q[1],), (q[0],)))
        elif g == "CZ":
            q = rng.choice(n, size=2, replace=False)
            ops.append(op("Z", (q[1],), (q[0],)))
        elif g == "SWAP":
            q = rng.choice(n, size=2, replace=False)
            ops.append(op("SWAP", (q[0], q[1])))
        else:  # TOFFOLI
            q = rng.choice(n, size=3, replace=False)
            ops.append(op("X", (q[2],), (q[0], q[1])))
    return ops


def hadamard_all(n: int) -> List[Op]:
    return [op("H", (q,)) for q in range(n)]


def layered_circuit(n: int = 30, layers: int = 20, seed: int = 2) -> List[Op]:
    """Sparse-gate layered circuit: H on every qubit, then ``layers`` times
    [CNOT ladder (q -> q+1, q = 0..n-2, in that order); CZ on a random
    perfect matching of the qubits; T or S (fair coin) on a random half of
    the qubits; RZ(theta ~ U[0, 2pi)) on every qubit]."""
    rng = np.random.default_rng(seed)
    ops: List[Op] = hadamard_all(n)
    for _ in range(layers):
        for q in range(n - 1):
            ops.append(op("X", (q + 1,), (q,)))
        perm = rng.permutation(n)
        for j in range(n // 2):
            a, b = int(perm[2 * j]), int(perm[2 * j + 1])
            ops.append(op("Z", (b,), (a,)))
        half = rng.choice(n, size=n // 2, replace=False)
        coins = rng.integers(0, 2, size=n // 2)
        for q, c in zip(half, coins):
            ops.append(op("T" if c else "S", (int(q),)))
        thetas = rng.uniform(0.0, TWO_PI, size=n)
        for q in range(n):
            ops.append(op("RZ", (q,), (), (thetas[q],)))
    return ops


def grover_marked(n: int, seed: int = 3) -> int:
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, 1 << n, dtype=np.uint64))


def flip_index(n: int, index: int) -> Op:
    """Sign flip of the single basis state ``index`` (all qubits control)."""
    return op("FLIP", (), tuple(range(n)), (), index)


def grover_circuit(n: int = 33, iterations: int = 8, seed: int = 3) -> Tuple[List[Op], int]:
    """Grover-style Hadamard-heavy circuit: H on all; then ``iterations`` x
    [phase flip of the marked index; H on all; phase flip of |0...0>; H on all]."""
    m = grover_marked(n, seed)
    ops: List[Op] = hadamard_all(n)
    for _ in range(iterations):
        ops.append(flip_index(n, m))
        ops.extend(hadamard_all(n))
        ops.append(flip_index(n, 0))
        ops.extend(hadamard_all(n))
    return ops, m


def ansatz_ops(n: int, theta: np.ndarray) -> List[Op]:
    """Hardware-efficient ansatz.  ``theta`` has shape [L, 2, n]: layer l
    applies RY(theta[l, 0, q]) to every qubit q, then RZ(theta[l, 1, q]) to
    every qubit, then the CNOT ring q -> (q + 1) mod n for q = 0..n-1.  The
    flat parameter index is l*2n + g*n + q, i.e. the order in which the
    parameterised gates appear in the circuit."""
    theta = np.asarray(theta, dtype=np.float64)
    L = theta.shape[0]
    ops: List[Op] = []
    for l in range(L):
        for q in range(n):
            ops.append(op("RY", (q,), (), (theta[l, 0, q],)))
        for q in range(n):
            ops.append(op("RZ", (q,), (), (theta[l, 1, q],)))
        for q in range(n):
            ops.append(op("X", ((q + 1) % n,), (q,)))
    return ops


def qnn_requests(count: int = 4096, seed: int = 4, n_lo: int = 8, n_hi: int = 20,
                 l_lo: int = 4, l_hi: int = 12):
    """Serving workload: ``count`` requests with n ~ U{n_lo..n_hi},
    L ~ U{l_lo..l_hi}, theta ~ U[0, 2pi) of shape [L, 2, n], and unit-rate
    exponential inter-arrival gaps (scale by 1/lambda for a Poisson
    process of rate lambda)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        L = int(rng.integers(l_lo, l_hi + 1))
        theta = rng.uniform(0.0, TWO_PI, size=(L, 2, n))
        gap = float(rng.exponential(1.0))
        reqs.append({"id": i, "n": n, "layers": L, "theta": theta, "gap": gap})
    return reqs


def qnn_batch(batch: int = 1024, n: int = 16, layers: int = 10, seed: int = 5) -> np.ndarray:
    """Training workload: per-circuit angles, shape [B, L, 2, n]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, TWO_PI, size=(batch, layers, 2, n))


def random_state(n: int, seed: int) -> np.ndarray:
    """Normalised complex128 state with i.i.d. Gaussian amplitudes."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (v / np.sqrt(np.vdot(v, v).real)).astype(np.complex128)


def random_unitary(dim: int, seed: int) -> np.ndarray:
    """Haar-like random unitary (QR of a complex Gaussian matrix with the
    phases of R's diagonal divided out)."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def measure_uniforms(k: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=k)


# Configuration sizes of the five workloads.
CONFIGS = {
    "random_n10": dict(n=10, n_gates=200, seed=1),
    "layered_n30": dict(n=30, layers=20, seed=2),
    "grover_n33": dict(n=33, iterations=8, seed=3),
    "qnn_serving": dict(count=4096, seed=4),
    "qnn_training": dict(batch=1024, n=16, layers=10, seed=5),
}
