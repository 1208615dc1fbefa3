"""State vector, operation matrix and readouts, FP64 (Sec. II-A, Eq. 3-7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (the paper's Eq. 6 puts its qubit 1 at the most significant
end of I^{(x)k-1} (x) G (x) I^{(x)n-k}; here qubit q is bit q of the basis
index, so the paper's qubit k is bit n-k):

* a state is a complex128 vector of length N = 2^n (Eq. 3);
* a gate on targets (t_0, ..., t_{k-1}) with controls (c_0, ...) acts
  with the matrix ``controlled(G)`` in the basis |c_0 .. c_{m-1} t_0 ..>,
  first listed qubit most significant.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from . import gates as _g


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def basis_state(n: int, index: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


def op_matrix(name: str, targets, controls, params, ctrl_values) -> np.ndarray:
    """Full matrix of an operation in the basis |controls, targets>."""
    G = _g.matrix(name, params)
    return _g.controlled(G, len(controls), ctrl_values)


# --------------------------------------------------------------------------
# Literal MTP (Eq. 6) and MVM (Eq. 7).  Only for small n: 16 * 4^n bytes.
# --------------------------------------------------------------------------

def mtp_kron(n: int, G: np.ndarray, low: int) -> np.ndarray:
    """Eq. 6 for a gate on the consecutive qubits low .. low+k-1 (its first
    target the highest): U = I_{2^(n-low-k)} (x) G (x) I_{2^low}, built by
    explicit Kronecker products."""
    k = int(round(math.log2(G.shape[0])))
    left = np.eye(1 << (n - low - k), dtype=np.complex128)
    right = np.eye(1 << low, dtype=np.complex128)
    return np.kron(np.kron(left, G), right)


def operation_matrix(n: int, Gfull: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """2^n x 2^n operation matrix of ``Gfull`` acting on ``qubits`` (first
    listed = most significant bit of the sub-index), by the element
    definition U[i][j] = Gfull[sub(i)][sub(j)] * [rest(i) == rest(j)], which
    is Eq. 6 with the gate's qubits in any position."""
    N = 1 << n
    m = len(qubits)
    qs = list(qubits)
    mask = 0
    for q in qs:
        mask |= 1 << q
    rows = np.arange(N, dtype=np.int64)
    sub_r = np.zeros(N, dtype=np.int64)
    for pos, q in enumerate(qs):
        sub_r |= ((rows >> q) & 1) << (m - 1 - pos)
    U = np.zeros((N, N), dtype=np.complex128)
    rest = rows & ~mask
    for s in range(1 << m):
        cols = rest.copy()
        for pos, q in enumerate(qs):
            cols |= ((s >> (m - 1 - pos)) & 1) << q
        U[rows, cols] = Gfull[sub_r, s]
    return U


def operation_matrix_op(n: int, o) -> np.ndarray:
    name, targets, controls, params, cv = o
    return operation_matrix(n, op_matrix(name, targets, controls, params, cv),
                            list(controls) + list(targets))


def mvm(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Eq. 7: the next state is the operation matrix times the state."""
    return U @ psi


# --------------------------------------------------------------------------
# Per-gate application without the operation matrix (any n).
# --------------------------------------------------------------------------

def apply_matrix(psi: np.ndarray, n: int, G: np.ndarray, targets: Sequence[int],
                 controls: Sequence[int] = (), ctrl_values: int | None = None) -> np.ndarray:
    """Apply the 2^k x 2^k matrix G to ``targets`` on the sub-space where
    every control c_j holds bit j of ``ctrl_values``.  The state is viewed
    as an n-axis tensor (axis n-1-q is qubit q); the control axes are fixed
    to their values and G is contracted with the target axes.  In place;
    returns ``psi``."""
    k = len(targets)
    if ctrl_values is None:
        ctrl_values = (1 << len(controls)) - 1
    if len(controls) == n:                   # a single basis state
        flat = 0
        for j, c in enumerate(controls):
            flat |= ((ctrl_values >> j) & 1) << c
        psi[flat] *= G[0, 0]
        return psi
    t = psi.reshape((2,) * n)
    idx = [slice(None)] * n
    for j, c in enumerate(controls):
        idx[n - 1 - c] = (ctrl_values >> j) & 1
    sub = t[tuple(idx)]                      # view of the controlled slice
    remaining = [n - 1 - a for a in range(n) if (n - 1 - a) not in set(controls)]
    if k == 0:
        sub *= G[0, 0]
        return psi
    axes = [remaining.index(q) for q in targets]
    Gt = G.reshape((2,) * (2 * k))
    new = np.tensordot(Gt, sub, axes=(list(range(k, 2 * k)), axes))
    new = np.moveaxis(new, list(range(k)), axes)
    sub[...] = new
    return psi


def apply_op(psi: np.ndarray, n: int, o) -> np.ndarray:
    name, targets, controls, params, cv = o
    G = _g.matrix(name, params)
    return apply_matrix(psi, n, G, targets, controls, cv)


def apply_ops(psi: np.ndarray, n: int, ops) -> np.ndarray:
    for o in ops:
        apply_op(psi, n, o)
    return psi


def simulate(n: int, ops, psi0: np.ndarray | None = None) -> np.ndarray:
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
    return apply_ops(psi, n, ops)


# --------------------------------------------------------------------------
# Readouts (Eq. 4-5): probabilities are squared magnitudes.
# --------------------------------------------------------------------------

def probabilities(psi: np.ndarray) -> np.ndarray:
    """|alpha_i|^2 as re*re + im*im (two products, one sum, no fused
    multiply-add), the rounding every integer decision below uses."""
    return psi.real * psi.real + psi.imag * psi.imag


def norm2(psi: np.ndarray) -> float:
    return float(math.fsum(probabilities(psi)))


def expect_z(psi: np.ndarray, n: int, q: int) -> float:
    """<Z_q> = sum_i (1 - 2 bit_q(i)) |alpha_i|^2."""
    p = probabilities(psi)
    bit = (np.arange(p.size, dtype=np.int64) >> q) & 1
    return float(math.fsum(p[bit == 0]) - math.fsum(p[bit == 1]))


def expect_z_sum(psi: np.ndarray, n: int) -> float:
    """sum_q <Z_q> = sum_i (n - 2 popcount(i)) |alpha_i|^2."""
    p = probabilities(psi)
    idx = np.arange(p.size, dtype=np.int64)
    pc = np.zeros(p.size, dtype=np.int64)
    for q in range(n):
        pc += (idx >> q) & 1
    return float(math.fsum((n - 2 * pc) * p))


def argmax(psi: np.ndarray) -> int:
    """Most probable basis index; the lowest index wins a tie."""
    return int(np.argmax(probabilities(psi)))


def measure(psi: np.ndarray, us) -> np.ndarray:
    """Inverse-CDF sampling: for each u in [0, 1) the smallest i with
    C_i > u * C_{N-1}, where C is the running sum of |alpha_i|^2."""
    c = np.cumsum(probabilities(psi))
    total = c[-1]
    out = np.empty(len(us), dtype=np.int64)
    for j, u in enumerate(us):
        out[j] = int(np.searchsorted(c, u * total, side="right"))
        out[j] = min(out[j], c.size - 1)
    return out
