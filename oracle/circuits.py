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


def _monomial_rows(G: np.ndarray):
    """For each row r of a monomial matrix: its one non-zero column and
    value."""
    d = G.shape[0]
    col = np.empty(d, dtype=np.int64)
    val = np.empty(d, dtype=np.complex128)
    for r in range(d):
        nz = np.nonzero(G[r])[0]
        if nz.size != 1:
            raise ValueError("gate is not monomial")
        col[r] = nz[0]
        val[r] = G[r, nz[0]]
    return col, val


def monomial_amplitudes(n: int, ops, indices, initial) -> np.ndarray:
    """``monomial_amplitude`` for many indices at once: the same backward
    path through the gates, followed for every index in the array
    ``indices``; ``initial`` maps an int64 array of basis indices to the
    complex array of <j|psi0>."""
    idx = np.array(indices, dtype=np.int64).reshape(-1)
    amp = np.ones(idx.shape, dtype=np.complex128)
    for (name, targets, controls, params, cv) in reversed(list(ops)):
        G = sv.op_matrix(name, targets, controls, params, cv)
        qs = list(controls) + list(targets)
        m = len(qs)
        col, val = _monomial_rows(G)
        r = np.zeros(idx.shape, dtype=np.int64)
        for pos, q in enumerate(qs):
            r |= ((idx >> q) & 1) << (m - 1 - pos)
        amp *= val[r]
        s = col[r]
        for pos, q in enumerate(qs):
            bit = (s >> (m - 1 - pos)) & 1
            idx = (idx & ~(np.int64(1) << q)) | (bit << q)
    return amp * np.asarray(initial(idx), dtype=np.complex128)


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


_PAULI = {"RX": np.array([[0, 1], [1, 0]], dtype=np.complex128),
          "RY": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          "RZ": np.array([[1, 0], [0, -1]], dtype=np.complex128)}


def _apply_observable(psi: np.ndarray, n: int, observable: str) -> np.ndarray:
    """O psi for O = Z_0 ('z0') or sum_q Z_q ('zsum'); both are diagonal
    in the computational basis."""
    idx = np.arange(psi.size, dtype=np.int64)
    if observable == "z0":
        return (1 - 2 * (idx & 1)) * psi
    if observable == "zsum":
        pc = np.zeros(psi.size, dtype=np.int64)
        for q in range(n):
            pc += (idx >> q) & 1
        return (n - 2 * pc) * psi
    raise ValueError(observable)


def adjoint_grad(n, theta, ops_fn, observable="zsum"):
    """f = <psi|O|psi>, psi = U_G ... U_1 |0>, and df/dtheta for every
    rotation angle by the reverse sweep of adjoint differentiation (Jones &
    Gacon 2020): start from psi and lambda = O psi; for g = G .. 1 undo the
    gate on psi (psi <- U_g^dagger psi, the state before gate g); if gate g
    is a rotation exp(-i theta P / 2), its derivative is
    dU_g/dtheta = (-i/2) P U_g and df/dtheta = 2 Re <lambda| dU_g/dtheta |psi>;
    then lambda <- U_g^dagger lambda.  The k-th rotation of the gate list
    holds flat parameter k.  Returns (f, grad with theta's shape)."""
    theta = np.asarray(theta, dtype=np.float64)
    ops = list(ops_fn(n, theta))
    psi = sv.simulate(n, ops)
    lam = _apply_observable(psi, n, observable)
    f = float(np.vdot(psi, lam).real)
    rot = [j for j, o in enumerate(ops) if o[0] in _PAULI]
    if len(rot) != theta.size:
        raise ValueError("one rotation per angle expected")
    slot = {j: k for k, j in enumerate(rot)}
    g = np.zeros(theta.size, dtype=np.float64)
    for j in range(len(ops) - 1, -1, -1):
        name, targets, controls, params, cv = ops[j]
        U = sv.op_matrix(name, targets, controls, params, cv)
        Ud = U.conj().T
        qs = list(controls) + list(targets)
        sv.apply_matrix(psi, n, Ud, qs)
        if j in slot:
            dU = -0.5j * (_PAULI[name] @ _g.matrix(name, params))
            d = sv.apply_matrix(psi.copy(), n, dU, list(targets))
            g[slot[j]] = 2.0 * float(np.vdot(lam, d).real)
        sv.apply_matrix(lam, n, Ud, qs)
    return f, g.reshape(theta.shape)


def hadamard_layer(psi: np.ndarray, n: int, mask: int) -> np.ndarray:
    """H on every qubit whose bit is set in ``mask`` (in place)."""
    H = _g.matrix("H")
    for q in range(n):
        if (mask >> q) & 1:
            sv.apply_matrix(psi, n, H, [q])
    return psi
