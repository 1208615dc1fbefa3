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
