"""The complex128 fused path keeps the state as int64 fixed point across a
circuit's tile passes (global scale from a norm bound).  These tests pin
what that format must preserve: exact results where the mathematics gives
exact values, exact zeros, the norm over long circuits, and states that are
not normalised."""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from paper_2411_15332_gb300.inputs import op
from tests.gpu_helpers import lib_ready, max_err, new_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


@pytest.mark.parametrize("n", [20, 21, 24, 25])
def test_hadamard_layer_is_uniform(n):
    """H on every qubit of |0>: every amplitude is 2^(-n/2) (exact for even
    n, within a few units in the last place for odd n)."""
    s = new_state(n)
    s.apply_circuit(inputs.hadamard_all(n), mode="fused")
    got = s.to_numpy()
    s.close()
    exact = 2.0 ** (-n / 2)
    assert np.max(np.abs(got.imag)) == 0.0
    assert np.max(np.abs(got.real - exact)) <= 1e-14 * exact


def test_vanishing_amplitudes_stay_exactly_zero():
    """H on qubits 0..20 of n = 24 (two passes, one with an odd number of
    levels): amplitudes with any of bits 21..23 set are exactly 0."""
    n = 24
    s = new_state(n)
    s.apply_circuit([op("H", (q,)) for q in range(21)], mode="fused")
    got = s.to_numpy()
    s.close()
    idx = np.arange(1 << n)
    assert np.all(got[(idx >> 21) != 0] == 0)
    assert np.max(np.abs(got[(idx >> 21) == 0] - 2.0 ** -10.5)) <= 1e-14 * 2.0 ** -10.5


def test_norm_and_probabilities_over_a_long_circuit():
    """Layered circuit, n = 22, 20 layers (61 passes): after the H layer
    every gate is a phase times a permutation, so every probability stays
    2^-n, the norm stays 1 and <Z_0> = 0."""
    n = 22
    ops = inputs.layered_circuit(n, 20, seed=2)
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    nrm, z0, _ = s.observables(0)
    s.close()
    assert abs(nrm - 1.0) <= 1e-13
    assert abs(z0) <= 1e-13
    assert np.max(np.abs(np.abs(got) ** 2 * (1 << n) - 1.0)) <= 1e-11
    ref = sv.simulate(n, ops)
    assert max_err(got, ref) <= 1e-13


@pytest.mark.parametrize("scale", [1e-3, 3.7, 1e5])
def test_unnormalised_state(scale):
    """The format's scale follows the state's norm: a random state times
    `scale` through rotations on every qubit followed by a monomial body
    (CNOT ladders, CZ, T/S, RZ) matches the oracle within 1e-12 relative to
    the norm."""
    n = 14
    psi = inputs.random_state(n, seed=9) * scale
    rng = np.random.default_rng(10)
    prefix = [op("RY", (q,), (), (float(rng.uniform(0, 6.28)),)) for q in range(n)]
    ops = prefix + inputs.layered_circuit(n, 6, seed=11)[n:]
    s = new_state(n, psi=psi)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    ref = sv.simulate(n, ops, psi0=psi)
    assert max_err(got, ref) <= 1e-12 * scale


def test_permutations_on_loads_and_stores_in_place():
    """Rotations, then CNOT ladders and rotations about Z only: the ladders
    ride on gathered loads and scattered stores of single-phase passes that
    move amplitudes between threads of a tile in place (every load must
    precede every store).  Checked against the oracle amplitude by
    amplitude."""
    n = 20
    rng = np.random.default_rng(21)
    ops = [op("RY", (q,), (), (float(rng.uniform(0, 6.28)),)) for q in range(n)]
    for _ in range(6):
        ops += [op("X", (q + 1,), (q,)) for q in range(n - 1)]
        ops += [op("RZ", (q,), (), (float(rng.uniform(0, 6.28)),)) for q in range(n)]
        ops += [op("X", (q,), (q + 1,)) for q in range(n - 2, -1, -1)]
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    ref = sv.simulate(n, ops)
    assert max_err(got, ref) <= 1e-13


@pytest.mark.parametrize("layers", [2, 3])
def test_runs_split_by_per_gate_ops(layers):
    """A three-target gate runs as a per-gate kernel between two runs of
    fixed-point passes; each run alternates between the state and a second
    buffer and must end in the state (odd and even pass counts)."""
    n = 16
    rng = np.random.default_rng(30 + layers)
    ops = [op("RY", (q,), (), (float(rng.uniform(0, 6.28)),)) for q in range(n)]
    body = inputs.layered_circuit(n, layers, seed=31)[n:]
    half = len(body) // 2
    perm8 = np.roll(np.eye(8, dtype=np.complex128), 1, axis=0)   # a three-qubit permutation
    first = ops + body[:half]
    second = body[half:]
    s = new_state(n)
    s.apply_circuit(first + [(perm8, (9, 2, 13), (), (), 0)] + second, mode="fused")
    got = s.to_numpy()
    s.close()
    ref = sv.simulate(n, first)
    ref = sv.apply_matrix(ref, n, perm8, (9, 2, 13))
    ref = sv.simulate(n, second, psi0=ref)
    assert max_err(got, ref) <= 1e-13


def _grover_split(n):
    """Hadamard layers after sign flips, split into two runs by a
    three-target gate; the partial layer on even qubits gives the first run
    an odd level count somewhere."""
    m = inputs.grover_marked(n, seed=7)
    perm8 = np.roll(np.eye(8, dtype=np.complex128), 1, axis=0)
    first = inputs.hadamard_all(n) + [inputs.flip_index(n, m)] + [op("H", (q,)) for q in range(0, n, 2)]
    second = ([inputs.flip_index(n, 0)] + inputs.hadamard_all(n) + [inputs.flip_index(n, m)]
              + inputs.hadamard_all(n))
    return first, perm8, second


@pytest.mark.parametrize("n", [14, 17])
def test_hadamard_runs_split_by_per_gate_ops(n):
    """Mixing gates after sign flips keep float64 storage; the Hadamard
    passes (per-tile int64, scaling at phase exits, an odd level count
    ending in a rounded 1/sqrt(2) product) on both sides of a per-gate op."""
    first, perm8, second = _grover_split(n)
    s = new_state(n)
    s.apply_circuit(first + [(perm8, (n - 1, 3, 6), (), (), 0)] + second, mode="fused")
    got = s.to_numpy()
    s.close()
    ref = sv.simulate(n, first)
    ref = sv.apply_matrix(ref, n, perm8, (n - 1, 3, 6))
    ref = sv.simulate(n, second, psi0=ref)
    assert max_err(got, ref) <= 1e-13


def test_hadamard_passes_on_a_general_state():
    """Per-tile int64 Hadamard passes on arbitrary doubles (not a basis
    state): block exponents from every tile's own maximum."""
    n = 16
    rng = np.random.default_rng(44)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    ops, _ = inputs.grover_circuit(n, 2, seed=3)
    s = new_state(n, psi=psi)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    ref = sv.simulate(n, ops, psi0=psi)
    assert max_err(got, ref) <= 1e-13


def test_hadamard_passes_are_deterministic():
    """Rounding depends only on the values and the plan: the same circuit
    gives bitwise the same state."""
    n = 20
    ops, _ = inputs.grover_circuit(n, 3, seed=3)
    outs = []
    for _ in range(2):
        s = new_state(n)
        s.apply_circuit(ops, mode="fused")
        outs.append(s.to_numpy())
        s.close()
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
