"""Pins for the oracle's state-vector routines: the literal MTP (Eq. 6) and
MVM (Eq. 7), per-gate application, closed forms and readouts.  CPU only."""
import math

import numpy as np
import pytest

from oracle import circuits as oc
from oracle import gates as g
from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs

RNG = np.random.default_rng(99)


def _rand_state(n, seed):
    return inputs.random_state(n, seed)


def test_mtp_kron_equals_element_definition():
    """np.kron (library routine) pins the element definition of Eq. 6 for
    gates on consecutive qubits, first target most significant."""
    n = 5
    for name, k in (("H", 1), ("Y", 1), ("ISWAP", 2), ("RZX", 2)):
        G = g.matrix(name, (0.37,) * g.GATE_ARITY[name][1])
        for low in range(n - k + 1):
            targets = [low + k - 1 - j for j in range(k)]
            np.testing.assert_array_equal(sv.mtp_kron(n, G, low), sv.operation_matrix(n, G, targets))
    U3 = g.controlled(g.matrix("X"), 2)
    np.testing.assert_array_equal(sv.mtp_kron(n, U3, 1), sv.operation_matrix(n, U3, [3, 2, 1]))


def _perm_matrix(n, perm):
    """P|i> = |i'> with bit perm[q] of i' equal to bit q of i."""
    N = 1 << n
    P = np.zeros((N, N))
    for i in range(N):
        j = 0
        for q in range(n):
            j |= ((i >> q) & 1) << perm[q]
        P[j, i] = 1
    return P


def test_element_definition_equals_conjugated_kron():
    """A gate on arbitrary qubits is the Kronecker form on consecutive qubits
    conjugated by the qubit permutation that moves them there (brute force)."""
    n = 5
    G = g.matrix("RXX", (0.9,))
    Gc = g.controlled(G, 1)
    qubits = [0, 4, 2]          # control 0, targets 4, 2
    # permutation sending qubits[j] -> position 2 - j (consecutive block 2,1,0)
    perm = [None] * n
    dest = {qubits[0]: 2, qubits[1]: 1, qubits[2]: 0}
    free = [p for p in range(n) if p not in dest.values()]
    rest = [q for q in range(n) if q not in dest]
    for q, p in zip(rest, free):
        dest[q] = p
    for q in range(n):
        perm[q] = dest[q]
    P = _perm_matrix(n, perm)
    U = P.T @ sv.mtp_kron(n, Gc, 0) @ P
    np.testing.assert_allclose(sv.operation_matrix(n, Gc, qubits), U, atol=0)


@pytest.mark.parametrize("seed", range(6))
def test_apply_matrix_equals_operation_matrix(seed):
    """Two independent routes: tensor contraction vs literal matrix."""
    rng = np.random.default_rng(seed)
    n = 6
    for k in (1, 2, 3):
        for nc in (0, 1, 2):
            qs = rng.choice(n, size=k + nc, replace=False)
            controls, targets = list(qs[:nc]), list(qs[nc:])
            G = inputs.random_unitary(1 << k, seed * 10 + k)
            cv = int(rng.integers(0, 1 << nc))
            psi = _rand_state(n, seed)
            U = sv.operation_matrix(n, g.controlled(G, nc, cv), controls + targets)
            ref = sv.mvm(U, psi)
            got = sv.apply_matrix(psi.copy(), n, G, targets, controls, cv)
            np.testing.assert_allclose(got, ref, atol=1e-14)


def _bit_permute_reference(psi, n, fn):
    """out[fn(i)] = psi[i] for a bijection fn on basis indices."""
    out = np.empty_like(psi)
    for i in range(1 << n):
        out[fn(i)] = psi[i]
    return out


def test_permutation_gates_exact():
    n = 7
    psi = _rand_state(n, 5)
    flip = lambda i, q: i ^ (1 << q)
    bit = lambda i, q: (i >> q) & 1
    cases = [
        (("X", (3,), (), (), 0), lambda i: flip(i, 3)),
        (("X", (1,), (5,), (), 1), lambda i: flip(i, 1) if bit(i, 5) else i),
        (("X", (6,), (0, 2), (), 3), lambda i: flip(i, 6) if bit(i, 0) and bit(i, 2) else i),
        (("SWAP", (2, 5), (), (), 0),
         lambda i: (i & ~((1 << 2) | (1 << 5))) | (bit(i, 2) << 5) | (bit(i, 5) << 2)),
    ]
    for o, fn in cases:
        got = sv.apply_op(psi.copy(), n, o)
        assert np.array_equal(got, _bit_permute_reference(psi, n, fn)), o


def test_diagonal_gates_exact():
    n = 6
    psi = _rand_state(n, 6)
    got = psi.copy()
    for _ in range(4):
        sv.apply_op(got, n, ("S", (2,), (), (), 0))
    assert np.array_equal(got, psi)
    got = sv.apply_op(psi.copy(), n, ("Z", (4,), (1,), (), 1))      # CZ
    ref = psi.copy()
    for i in range(1 << n):
        if (i >> 4) & 1 and (i >> 1) & 1:
            ref[i] = -ref[i]
    assert np.array_equal(got, ref)


def test_hadamard_all_uniform_and_involution():
    for n in (1, 4, 9):
        psi = sv.simulate(n, inputs.hadamard_all(n))
        np.testing.assert_allclose(psi, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-15)
        back = sv.apply_ops(psi, n, inputs.hadamard_all(n))
        np.testing.assert_allclose(back, sv.zero_state(n), atol=1e-15)


def test_ghz():
    n = 8
    ops = [inputs.op("H", (0,))] + [inputs.op("X", (q,), (0,)) for q in range(1, n)]
    psi = sv.simulate(n, ops)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-15)


def qft_ops(n):
    """Textbook QFT: for qubits from the most significant down, H then
    controlled phases pi/2^d from each lower qubit; finally reverse the
    qubit order with swaps."""
    ops = []
    for i in range(n - 1, -1, -1):
        ops.append(inputs.op("H", (i,)))
        for j in range(i - 1, -1, -1):
            ops.append(inputs.op("P", (i,), (j,), (math.pi / 2 ** (i - j),)))
    for i in range(n // 2):
        ops.append(inputs.op("SWAP", (i, n - 1 - i)))
    return ops


@pytest.mark.parametrize("j", [0, 1, 5, 37, 63])
def test_qft_of_basis_state(j):
    """QFT|j> = sum_k e^{2 pi i jk/N}/sqrt(N) |k>, pinned by numpy's FFT."""
    n = 6
    N = 1 << n
    psi = sv.simulate(n, qft_ops(n), sv.basis_state(n, j))
    ref = np.fft.ifft(sv.basis_state(n, j)) * math.sqrt(N)
    np.testing.assert_allclose(psi, ref, atol=1e-14)


def test_norm_preserved_random_circuit():
    n = 10
    psi = sv.simulate(n, inputs.random_circuit(n, 200, seed=11))
    assert abs(sv.norm2(psi) - 1.0) < 1e-13


def test_random_circuit_every_gate_against_literal_mtp():
    """The 200-gate n=10 random circuit: after every gate, the per-gate
    route equals the brute-force 2^10 x 2^10 operation matrix times the
    state (Eq. 6-7)."""
    n = 10
    ops = inputs.random_circuit(n, 200, seed=1)
    psi_a = sv.zero_state(n)
    psi_b = sv.zero_state(n)
    for o in ops:
        psi_a = sv.mvm(sv.operation_matrix_op(n, o), psi_a)
        sv.apply_op(psi_b, n, o)
        assert np.max(np.abs(psi_a - psi_b)) < 1e-13, o


def test_readouts():
    n = 5
    psi = _rand_state(n, 7)
    p = np.abs(psi) ** 2
    for q in range(n):
        Zq = np.diag([1.0 - 2.0 * ((i >> q) & 1) for i in range(1 << n)])
        assert sv.expect_z(psi, n, q) == pytest.approx(np.real(np.vdot(psi, Zq @ psi)), abs=1e-15)
    assert sv.expect_z_sum(psi, n) == pytest.approx(sum(sv.expect_z(psi, n, q) for q in range(n)), abs=1e-14)
    assert sv.norm2(psi) == pytest.approx(float(np.sum(p)), abs=1e-15)
    tie = np.zeros(1 << n, dtype=complex)
    tie[[3, 9, 20]] = 0.5
    tie[1] = 0.1
    assert sv.argmax(tie) == 3
    us = np.array([0.0, 0.05, 0.3, 0.999])
    got = sv.measure(psi, us)
    c = np.cumsum(p) / np.sum(p)
    for u, i in zip(us, got):
        brute = min(k for k in range(1 << n) if c[k] > u)
        assert i == brute


def test_monomial_amplitude_trace():
    """Path tracing through monomial gates equals full simulation."""
    n = 8
    ops = inputs.layered_circuit(n, 3, seed=2)
    psi = sv.simulate(n, ops)
    body = ops[n:]                     # gates after the H layer
    for i in [0, 1, 77, 200, 255]:
        a = oc.monomial_amplitude(n, body, i, lambda j: 2.0 ** (-n / 2))
        assert abs(a - psi[i]) < 1e-14
