"""GPU parity of the readouts (Eq. 4-5) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import lib_ready, new_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


@pytest.mark.parametrize("n", [1, 3, 8, 13, 21])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_observables(n, dtype):
    psi = inputs.random_state(n, seed=100 + n)
    if dtype == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    s = new_state(n, dtype, psi)
    tol = 1e-13
    assert abs(s.norm2() - sv.norm2(psi)) <= tol
    for q in sorted({0, n // 2, n - 1}):
        assert abs(s.expect_z(q) - sv.expect_z(psi, n, q)) <= tol
        nrm, ez, zs = s.observables(q)
        assert abs(ez - sv.expect_z(psi, n, q)) <= tol
    assert abs(s.expect_z_sum() - sv.expect_z_sum(psi, n)) <= tol * n


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_argmax_ties_lowest_index(dtype):
    n = 12
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[[7, 300, 2049, 4000]] = 0.5
    psi[5] = 0.25
    s = new_state(n, dtype, psi)
    i, p = s.argmax()
    assert i == sv.argmax(psi) == 7
    assert p == 0.25
    psi2 = inputs.random_state(n, seed=3)
    s2 = new_state(n, "c128", psi2)
    assert s2.argmax()[0] == sv.argmax(psi2)


def _safe_uniforms(psi, k, seed):
    """u values at least 1e-9 (relative) away from every CDF boundary."""
    c = np.cumsum(sv.probabilities(psi))
    c /= c[-1]
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < k:
        u = rng.uniform()
        if np.min(np.abs(c - u)) > 1e-9:
            out.append(u)
    return np.array(out)


@pytest.mark.parametrize("n", [4, 10, 17])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_measure_inverse_cdf(n, dtype):
    psi = inputs.random_state(n, seed=n)
    if dtype == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    us = _safe_uniforms(psi, 64, seed=n)
    s = new_state(n, dtype, psi)
    got = s.measure(us)
    assert np.array_equal(got, sv.measure(psi, us))


def test_measure_dyadic_ghz():
    n = 16
    ops = [inputs.op("H", (0,))] + [inputs.op("X", (q,), (0,)) for q in range(1, n)]
    s = new_state(n, "c128")
    s.apply_circuit(ops)
    got = s.measure([0.1, 0.49, 0.51, 0.9])
    assert list(got) == [0, 0, (1 << n) - 1, (1 << n) - 1]


def test_gather_amplitudes():
    n = 14
    psi = inputs.random_state(n, seed=1)
    s = new_state(n, "c128", psi)
    idx = np.array([0, 1, 5, 1000, (1 << n) - 1])
    assert np.array_equal(s.amplitudes(idx), psi[idx])


def test_async_upload_overlaps_and_matches():
    """mera_state_copy_from_host_async: two states on two streams, one
    uploading while the other runs a circuit; both give the oracle's
    result."""
    import torch
    from oracle import statevector as sv
    from paper_2411_15332_gb300 import State, inputs
    n = 16
    ops = inputs.layered_circuit(n, 3, seed=5)
    host = torch.zeros((1 << n) * 2, dtype=torch.float64).pin_memory()
    host[0] = 1.0
    hp = host.numpy().view(np.complex128)
    a = State(n, stream=torch.cuda.Stream())
    b = State(n, stream=torch.cuda.Stream())
    a.from_host_async(hp)
    a.apply_circuit(ops, mode="fused")
    b.from_host_async(hp)
    b.apply_circuit(ops, mode="fused")
    ref = sv.simulate(n, ops)
    for s in (a, b):
        got = s.to_numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12
        s.close()
    with pytest.raises(ValueError):
        State(n).from_host_async(np.zeros(1 << n, dtype=np.complex64))


def _readouts(psi, n, q):
    """norm^2, <Z_q> and sum_q <Z_q> of a state vector (numpy, float64)."""
    p = np.abs(np.asarray(psi, dtype=np.complex128)) ** 2
    idx = np.arange(p.size, dtype=np.uint64)
    bit = ((idx >> np.uint64(q)) & np.uint64(1)).astype(bool)
    pc = np.array([bin(i).count("1") for i in range(p.size)], dtype=np.float64)
    return float(p.sum()), float(p[~bit].sum() - p[bit].sum()), float((p * (n - 2.0 * pc)).sum())


def _check_readout(got, ref, n, dtype="c128"):
    from tests.gpu_helpers import obs_tol
    assert abs(got[0] - ref[0]) <= obs_tol(dtype, 1.0)
    assert abs(got[1] - ref[1]) <= obs_tol(dtype, 1.0)
    assert abs(got[2] - ref[2]) <= obs_tol(dtype, float(n))


@pytest.mark.parametrize("q", [0, 4, 9, 12, 15])
def test_apply_circuit_observe_in_the_last_pass(q):
    """mera_apply_circuit_observe on a layered circuit: the last pass (a
    monomial run pass writing doubles) sums the readout while it stores the
    state.  Same state as mera_apply_circuit; readouts as mera_observables
    and as the oracle's."""
    from paper_2411_15332_gb300 import core
    n = 16
    ops = inputs.layered_circuit(n, 4, seed=21)
    last = core.plan_summary(n, ops).splitlines()[-1]
    assert " amp " in last and "q_out=0" in last
    a = new_state(n)
    got = a.apply_circuit_observe(ops, q)
    b = new_state(n)
    b.apply_circuit(ops, mode="fused")
    ref = b.observables(q)
    psi = a.to_numpy()
    assert np.array_equal(psi, b.to_numpy())
    a.close()
    b.close()
    _check_readout(got, ref, n)
    _check_readout(got, _readouts(sv.simulate(n, ops), n, q), n)
    # a second call on the same state (cached passes) gives the same sums
    c = new_state(n)
    c.apply_circuit_observe(ops, q)
    c.set_basis(0)
    assert c.apply_circuit_observe(ops, q) == got
    c.close()


@pytest.mark.parametrize("case", ["grover", "per_gate", "c64"])
def test_apply_circuit_observe_without_a_readout_pass(case):
    """Where the last pass cannot sum the readout (a Hadamard pass, the
    per-gate mode, a complex64 state) the readout reduction runs after the
    circuit: the results equal mera_observables'."""
    n = 14
    dtype, mode = "c128", "fused"
    if case == "grover":
        ops = inputs.grover_circuit(n, 2, seed=3)[0]
    else:
        ops = inputs.layered_circuit(n, 3, seed=5)
        if case == "per_gate":
            mode = "per_gate"
        else:
            dtype = "c64"
    q = 3
    a = new_state(n, dtype)
    got = a.apply_circuit_observe(ops, q, mode=mode)
    b = new_state(n, dtype)
    b.apply_circuit(ops, mode=mode)
    ref = b.observables(q)
    a.close()
    b.close()
    assert got == ref
    _check_readout(got, _readouts(sv.simulate(n, ops), n, q), n, dtype)


def test_apply_circuit_observe_rejects_a_bad_qubit():
    from paper_2411_15332_gb300 import _lib as L
    n = 13
    s = new_state(n)
    with pytest.raises(L.MeraError) as e:
        s.apply_circuit_observe(inputs.layered_circuit(n, 1, seed=1), n)
    assert e.value.code == L.MERA_EINVAL
    s.close()
