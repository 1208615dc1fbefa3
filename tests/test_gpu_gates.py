"""GPU parity: per-gate and fused gate application against the FP64 oracle.

Tolerance: max |amp_gpu - amp_oracle| <= 1e-12 (complex128), <= 2e-5
(complex64).  Permutation and unit-phase gates must be bit-exact."""
import math

import numpy as np
import pytest

from oracle import gates as og
from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import TOL, lib_ready, max_err, new_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_random_circuit_every_gate_per_gate(dtype):
    """The n=10, 200-gate random circuit, checked after every gate."""
    n = 10
    ops = inputs.random_circuit(n, 200, seed=1)
    s = new_state(n, dtype)
    ref = sv.zero_state(n)
    worst = 0.0
    for o in ops:
        s.apply_circuit([o], mode="per_gate")
        sv.apply_op(ref, n, o)
        e = max_err(s.to_numpy(), ref)
        worst = max(worst, e)
        assert e <= TOL[dtype], (o, e)
    print(f"random n=10 {dtype} per-gate worst |d amp| = {worst:.3e}")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_random_circuit_fused_prefixes(dtype):
    n = 10
    ops = inputs.random_circuit(n, 200, seed=1)
    for cut in (1, 7, 50, 133, 200):
        s = new_state(n, dtype)
        s.apply_circuit(ops[:cut], mode="fused")
        ref = sv.simulate(n, ops[:cut])
        assert max_err(s.to_numpy(), ref) <= TOL[dtype]


def _random_ops(n, count, seed, names=None):
    rng = np.random.default_rng(seed)
    names = names or [g for g in og.GATE_ARITY]
    ops = []
    for _ in range(count):
        g = names[int(rng.integers(0, len(names)))]
        k, npar = og.GATE_ARITY[g]
        nc = int(rng.integers(0, min(3, n - k) + 1)) if g != "FLIP" else int(rng.integers(1, n + 1))
        qs = rng.choice(n, size=k + nc, replace=False)
        cv = int(rng.integers(0, 1 << nc))
        params = tuple(rng.uniform(0, 2 * math.pi, size=npar))
        if g in ("U", "U3"):
            params = params + (float(rng.uniform(0, 6.0)),)
        ops.append(inputs.op(g, qs[nc:], qs[:nc], params, cv))
    return ops


@pytest.mark.parametrize("n", [5, 6, 11, 14])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["per_gate", "fused"])
def test_catalogue_random_controls(n, dtype, mode):
    """Every catalogue gate with random qubits, 0-3 controls and random
    control values, on a random state; spans one tile (n <= 12) and several
    tiles with a ragged mix of targets (n = 14)."""
    ops = _random_ops(n, 150, seed=n * 7 + (mode == "fused"))
    psi0 = inputs.random_state(n, seed=n)
    s = new_state(n, dtype, psi0)
    s.apply_circuit(ops, mode=mode)
    ref = sv.simulate(n, ops, psi0)
    assert max_err(s.to_numpy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_long_fused_circuit_many_tiles(dtype):
    n = 17
    ops = _random_ops(n, 400, seed=5)
    psi0 = inputs.random_state(n, seed=3)
    s = new_state(n, dtype, psi0)
    s.apply_circuit(ops, mode="fused")
    ref = sv.simulate(n, ops, psi0)
    assert max_err(s.to_numpy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_matrix_gate(k, dtype):
    n = 9
    rng = np.random.default_rng(k)
    psi0 = inputs.random_state(n, seed=k)
    ref = psi0.copy()
    s = new_state(n, dtype, psi0)
    for j in range(6):
        U = inputs.random_unitary(1 << k, seed=10 * k + j)
        qs = rng.choice(n, size=k + 1, replace=False)
        s.apply_matrix(U, list(qs[1:]), [int(qs[0])])
        sv.apply_matrix(ref, n, U, list(qs[1:]), [int(qs[0])])
    assert max_err(s.to_numpy(), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["per_gate", "fused"])
def test_permutation_gates_bit_exact(dtype, mode):
    """X, Y, Z, S, CNOT, CZ, SWAP, Toffoli, DCX, iSWAP, FLIP move amplitudes
    and flip signs only: bit-exact against the oracle."""
    n = 15
    names = ["X", "Y", "Z", "S", "SDG", "SWAP", "DCX", "ISWAP", "FLIP"]
    ops = _random_ops(n, 200, seed=11, names=names)
    psi0 = inputs.random_state(n, seed=4)
    if dtype == "c64":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    s = new_state(n, dtype, psi0)
    s.apply_circuit(ops, mode=mode)
    ref = sv.simulate(n, ops, psi0)
    got = s.to_numpy().astype(np.complex128)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [5, 7, 13, 18])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_hadamard_layer(n, dtype):
    rng = np.random.default_rng(n)
    psi0 = inputs.random_state(n, seed=n + 1)
    for mask in [(1 << n) - 1, int(rng.integers(1, 1 << n)), 1, 1 << (n - 1)]:
        s = new_state(n, dtype, psi0)
        s.hadamard_layer(mask)
        ref = psi0.copy()
        for q in range(n):
            if (mask >> q) & 1:
                sv.apply_op(ref, n, ("H", (q,), (), (), 0))
        assert max_err(s.to_numpy(), ref) <= TOL[dtype]


def test_hadamard_all_uniform():
    n = 20
    s = new_state(n, "c128")
    s.hadamard_layer((1 << n) - 1)
    a = s.to_numpy()
    assert np.max(np.abs(a - 2.0 ** (-n / 2))) <= 1e-15


def test_empty_and_identity_circuits():
    n = 8
    psi0 = inputs.random_state(n, seed=9)
    s = new_state(n, "c128", psi0)
    s.apply_circuit([], mode="fused")
    s.apply_circuit([inputs.op("I", (3,)), inputs.op("RZ", (2,), (), (0.0,))], mode="fused")
    assert np.array_equal(s.to_numpy(), psi0)


def test_invalid_ops_leave_state_unchanged():
    from paper_2411_15332_gb300 import _lib as L
    n = 8
    psi0 = inputs.random_state(n, seed=12)
    s = new_state(n, "c128", psi0)
    bad = [
        [inputs.op("X", (8,))],                         # qubit >= n
        [inputs.op("X", (3,), (3,))],                   # target is a control
        [inputs.op("SWAP", (2, 2))],                    # duplicate target
        [inputs.op("RX", (1,), (), (float("nan"),))],   # NaN angle
        [inputs.op("H", (0,)), inputs.op("X", (9,))],   # valid op before a bad one
    ]
    for ops in bad:
        for mode in ("per_gate", "fused"):
            with pytest.raises(L.MeraError) as ei:
                s.apply_circuit(ops, mode=mode)
            assert ei.value.code == L.MERA_EINVAL
    assert np.array_equal(s.to_numpy(), psi0)


def test_diagonal_gates_on_both_product_paths():
    """Per-gate complex128 diagonals with general unit phases, controls and
    several targets, and a non-unitary diagonal (|Re| > 1)."""
    n = 16
    rng = np.random.default_rng(12)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    mats = [(np.diag(np.exp(1j * rng.uniform(0, 6.28, 2))), (3,), (), 0),
            (np.diag(np.exp(1j * rng.uniform(0, 6.28, 4))), (15, 0), (7,), 1),
            (np.diag([2.0 + 0.0j, 0.5j]), (9,), (), 0),
            (np.diag(np.exp(1j * rng.uniform(0, 6.28, 2))), (12,), (1, 4), 2)]
    s = new_state(n, "c128", psi=psi)
    s.apply_circuit([(G, t, c, (), cv) for G, t, c, cv in mats], mode="per_gate")
    got = s.to_numpy()
    s.close()
    ref = psi.copy()
    for G, t, c, cv in mats:
        sv.apply_matrix(ref, n, G, t, c, cv)
    assert max_err(got, ref) <= 1e-13
