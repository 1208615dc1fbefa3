"""Circuit-level oracle routines, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``simulate``: gate after gate on the full state (Eq. 7 with the
  operation matrix never formed: ``statevector.apply_op``).
* ``monomial_amplitude``: one amplitude of a circuit made of monomial
  gates (one non-zero per row: permutations times phases) after a known
  initial state, by following the single path back through the gates.
  This reaches states far too large for the host (n = 30, 33).
* ``grover_amplitudes``: closed form of the Grover-style circuit.
* QNN: expectation of the ansatz and its gradient by the parameter-shift
  rule (exact for RY / RZ, whose generators have eigenvalues +-1/2) and
  by central finite differences.
"""
from __future__ import annotations

import math

import numpy as np

from . import gates as _g
from . import statevector as sv


def simulate(n, ops, psi0=None):
    return sv.simulate(n, ops, psi0)


def _sub_index(i: int, qubits) -> int:
    m = len(qubits)
    s = 0
    for pos, q in enumerate(qubits):
        s |= ((i >> q) & 1) << (m - 1 - pos)
    return s


def _with_sub(i: int, qubits, s: int) -> int:
    m = len(qubits)
    for pos, q in enumerate(qubits):
        bit = (s >> (m - 1 - pos)) & 1
        i = (i & ~(1 << q)) | (bit << q)
    return i


def monomial_amplitude(n: int, ops, index: int, initial) -> complex:
    """<index| U_G ... U_1 |psi0> for monomial gates U_g, where ``initial``
    maps a basis index j to <j|psi0>.  Row sub(i) of a monomial matrix
    holds exactly one non-zero v at column s', so
    (U psi)[i] = v * psi[i with sub bits replaced by s']."""
    amp = 1.0 + 0.0j
    i = index
    for (name, targets, controls, params, cv) in reversed(list(ops)):
        G = sv.op_matrix(name, targets, controls, params, cv)
        qs = list(controls) + list(targets)
        r = _sub_index(i, qs)
        nz = np.nonzero(G[r])[0]
        if nz.size != 1:
            raise ValueError(f"gate {name} is not monomial")
        s = int(nz[0])
        amp *= G[r, s]
        i = _with_sub(i, qs, s)
    return amp * initial(i)


def grover_amplitudes(n: int, k: int):
    """Amplitudes after H on all qubits and k iterations of
    [flip marked; H all; flip |0>; H all].  H (I - 2|0><0|) H = I - 2|s><s|
    = -(2|s><s| - I), so each iteration is minus the textbook Grover
    iterate and the textbook result picks up (-1)^k:
      marked:  (-1)^k sin((2k+1) theta),
      other:   (-1)^k cos((2k+1) theta) / sqrt(N - 1),
    with sin(theta) = N^{-1/2}."""
    N = float(1 << n)
    theta = math.asin(1.0 / math.sqrt(N))
    sgn = -1.0 if (k % 2) else 1.0
    a_m = sgn * math.sin((2 * k + 1) * theta)
    a_o = sgn * math.cos((2 * k + 1) * theta) / math.sqrt(N - 1.0)
    return a_m, a_o


# ------------------------------------------------------------------ QNN ---

def ansatz_state(n: int, theta: np.ndarray, ops_fn) -> np.ndarray:
    return sv.simulate(n, ops_fn(n, theta))


def expectation(n: int, psi: np.ndarray, observable: str) -> float:
    """'z0' -> <Z_0>;  'zsum' -> sum_q <Z_q>."""
    if observable == "z0":
        return sv.expect_z(psi, n, 0)
    if observable == "zsum":
        return sv.expect_z_sum(psi, n)
    raise ValueError(observable)


def qnn_value(n, theta, ops_fn, observable="zsum") -> float:
    return expectation(n, ansatz_state(n, theta, ops_fn), observable)


def param_shift_grad(n, theta, ops_fn, observable="zsum") -> np.ndarray:
    """d f / d theta_p = [f(theta_p + pi/2) - f(theta_p - pi/2)] / 2."""
    theta = np.asarray(theta, dtype=np.float64)
    flat = theta.reshape(-1)
    g = np.zeros_like(flat)
    for p in range(flat.size):
        tp = flat.copy()
        tp[p] += math.pi / 2
        fp = qnn_value(n, tp.reshape(theta.shape), ops_fn, observable)
        tp[p] -= math.pi
        fm = qnn_value(n, tp.reshape(theta.shape), ops_fn, observable)
        g[p] = 0.5 * (fp - fm)
    return g.reshape(theta.shape)


def finite_diff_grad(n, theta, ops_fn, observable="zsum", h=1e-6) -> np.ndarray:
    """Central differences, error O(h^2)."""
    theta = np.asarray(theta, dtype=np.float64)
    flat = theta.reshape(-1)
    g = np.zeros_like(flat)
    for p in range(flat.size):
        tp = flat.copy()
        tp[p] += h
        fp = qnn_value(n, tp.reshape(theta.shape), ops_fn, observable)
        tp[p] -= 2 * h
        fm = qnn_value(n, tp.reshape(theta.shape), ops_fn, observable)
        g[p] = (fp - fm) / (2 * h)
    return g.reshape(theta.shape)


def hadamard_layer(psi: np.ndarray, n: int, mask: int) -> np.ndarray:
    """H on every qubit whose bit is set in ``mask`` (in place)."""
    H = _g.matrix("H")
    for q in range(n):
        if (mask >> q) & 1:
            sv.apply_matrix(psi, n, H, [q])
    return psi
