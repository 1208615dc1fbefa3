"""Monomial run passes against the oracle: a run of permutation gates whose
index maps are affine over GF(2) (X, CNOT with either control value, SWAP,
DCX) followed by diagonal gates (phases, RZ, RZZ, CZ, CCZ, index flips) is
one monomial operator (a product of DAX matrices) applied by one streaming
pass that gathers each output amplitude from F^-1(i).  The circuits start
with a Hadamard layer so that the complex128 state is resident and every
amplitude is nonzero."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from paper_2411_15332_gb300.inputs import op
from tests.gpu_helpers import TOL as _TOL, lib_ready, max_err, new_state

TOL = _TOL["c128"]

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


def _amp_lines(n, ops):
    from paper_2411_15332_gb300 import core
    return [l for l in core.plan_summary(n, ops).splitlines()[1:] if " amp " in l]


def _run(n, ops):
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    return got


def _monomial_run(rng, n, nperm, ndiag):
    """Permutations (affine index maps) then diagonals on random qubits."""
    ops = []
    for _ in range(nperm):
        g = int(rng.integers(0, 4))
        a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
        if g == 0:
            ops.append(op("X", (a,)))
        elif g == 1:
            ops.append(op("X", (b,), (a,), (), int(rng.integers(0, 2))))
        elif g == 2:
            ops.append(op("SWAP", (a, b)))
        else:
            ops.append(op("DCX", (a, b)))
    for _ in range(ndiag):
        g = int(rng.integers(0, 8))
        q = rng.choice(n, size=3, replace=False)
        a, b, c = int(q[0]), int(q[1]), int(q[2])
        t = float(rng.uniform(0.0, 2.0 * np.pi))
        if g == 0:
            ops.append(op("RZ", (a,), (), (t,)))
        elif g == 1:
            ops.append(op(["T", "S", "Z", "SDG", "TDG"][int(rng.integers(0, 5))], (a,)))
        elif g == 2:
            ops.append(op("P", (a,), (), (t,)))
        elif g == 3:
            ops.append(op("Z", (b,), (a,)))
        elif g == 4:
            ops.append(op("Z", (c,), (a, b)))
        elif g == 5:
            ops.append(op("RZZ", (a, b), (), (t,)))
        elif g == 6:
            ops.append(op("S", (b,), (a,), (), int(rng.integers(0, 2))))
        else:
            ops.append(inputs.flip_index(n, int(rng.integers(0, 1 << n))))
    return ops


@pytest.mark.parametrize("n,seed", [(13, 1), (14, 2), (16, 3), (18, 4), (20, 5)])
def test_random_monomial_runs(n, seed):
    rng = np.random.default_rng(seed)
    ops = inputs.hadamard_all(n)
    for _ in range(3):
        ops += _monomial_run(rng, n, 40, 40)
    assert len(_amp_lines(n, ops)) >= 2
    got = _run(n, ops)
    assert max_err(got, sv.simulate(n, ops)) <= TOL


@pytest.mark.parametrize("n", [13, 16, 19])
def test_layered_circuit_one_pass_per_layer(n):
    ops = inputs.layered_circuit(n, 6, seed=n)
    lines = _amp_lines(n, ops)
    assert len(lines) == 6
    got = _run(n, ops)
    assert max_err(got, sv.simulate(n, ops)) <= TOL


def test_run_shortened_when_phases_do_not_fit():
    """General two-qubit phases between local bits and more than eight
    distinct tile bits: the run is cut where table A's selection runs out,
    and the rest goes to later passes."""
    n = 22
    ops = inputs.hadamard_all(n)
    ops += [op("X", (q + 1,), (q,)) for q in range(n - 1)]
    ops += [op("RZZ", (q % 12, 12 + q), (), (0.3 + 0.1 * q,)) for q in range(n - 12)]
    ops += [op("RZ", (q,), (), (0.7 * q,)) for q in range(n)]
    lines = _amp_lines(n, ops)
    assert lines and all(int(l.split("sel_a=")[1].split()[0]) <= 8 for l in lines)
    got = _run(n, ops)
    assert max_err(got, sv.simulate(n, ops)) <= TOL


def test_matches_tile_planner(tmp_path):
    """The same layered circuit with monomial runs and with the tile planner
    alone (MERA_AMP=0, another process) agrees to the tolerance."""
    n = 22
    ops = inputs.layered_circuit(n, 8, seed=3)
    assert len(_amp_lines(n, ops)) == 8
    got = _run(n, ops)
    out = tmp_path / "tile.npy"
    code = ("import numpy as np\n"
            "from paper_2411_15332_gb300 import inputs, core\n"
            f"ops = inputs.layered_circuit({n}, 8, seed=3)\n"
            f"assert ' amp ' not in core.plan_summary({n}, ops)\n"
            f"s = core.State({n})\n"
            "s.apply_circuit(ops, mode='fused')\n"
            f"np.save({str(out)!r}, s.to_numpy())\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], cwd=root, env={**os.environ, "MERA_AMP": "0"}, check=True,
                   timeout=600)
    ref = np.load(out)
    assert np.max(np.abs(got - ref)) <= TOL
    # the magnitudes of a layered circuit stay 2^(-n/2)
    assert np.max(np.abs(np.abs(got) - 2.0 ** (-n / 2))) <= 1e-15


def test_repeated_circuit_reuses_its_passes():
    """A cached plan with monomial runs runs again on the same state (the
    second buffer is kept) and gives the same amplitudes."""
    n = 17
    ops = inputs.layered_circuit(n, 4, seed=9)
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    first = s.to_numpy()
    s.set_basis(0)
    s.apply_circuit(ops, mode="fused")
    second = s.to_numpy()
    s.close()
    assert np.array_equal(first, second)
    assert max_err(first, sv.simulate(n, ops)) <= TOL


@pytest.mark.parametrize("layers", [2, 3])
def test_run_of_monomial_passes_after_a_per_gate_op(layers):
    """A three-qubit permutation (a per-gate kernel) splits the circuit; the
    run after it is monomial run passes only, each out of place: with an odd
    count the run ends in the second buffer and is copied into the state."""
    n = 15
    perm8 = np.roll(np.eye(8, dtype=np.complex128), 1, axis=0)
    body = inputs.layered_circuit(n, layers, seed=40 + layers)[n:]
    ops = inputs.hadamard_all(n) + [(perm8, (9, 2, 13), (), (), 0)] + body
    assert len(_amp_lines(n, ops)) == layers
    got = _run(n, ops)
    ref = sv.simulate(n, inputs.hadamard_all(n))
    ref = sv.apply_matrix(ref, n, perm8, (9, 2, 13))
    ref = sv.simulate(n, body, psi0=ref)
    assert max_err(got, ref) <= TOL


def test_64bit_index_variant(tmp_path):
    """The variant with 64-bit index arithmetic (states above 2^32
    amplitudes) on a small state (MERA_AMP_IX64=1, another process)
    gives the same bits as the 32-bit one."""
    n = 18
    rng = np.random.default_rng(11)
    ops = inputs.hadamard_all(n)
    for _ in range(2):
        ops += _monomial_run(rng, n, 30, 30)
    got = _run(n, ops)
    import pickle
    out = tmp_path / "ix64.npy"
    ops_file = tmp_path / "ops.pkl"
    with open(ops_file, "wb") as f:
        pickle.dump(ops, f)
    code = ("import pickle\n"
            "import numpy as np\n"
            "from paper_2411_15332_gb300 import core\n"
            f"ops = pickle.load(open({str(ops_file)!r}, 'rb'))\n"
            f"s = core.State({n})\n"
            "s.apply_circuit(ops, mode='fused')\n"
            f"np.save({str(out)!r}, s.to_numpy())\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], cwd=root, env={**os.environ, "MERA_AMP_IX64": "1"}, check=True,
                   timeout=600)
    assert np.array_equal(got.view(np.uint64), np.load(out).view(np.uint64))
    assert max_err(got, sv.simulate(n, ops)) <= TOL
