"""Pins for circuit-level oracle routines: Grover closed form, monomial path
tracing and QNN gradients.  CPU only."""
import math

import numpy as np
import pytest

from oracle import circuits as oc
from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs


@pytest.mark.parametrize("n", [3, 4, 6, 9])
def test_grover_closed_form(n):
    """Simulated Grover-style circuit equals the closed form at every
    iteration count, sign included (not up to a global phase)."""
    m = inputs.grover_marked(n, seed=3)
    for k in range(0, 9):
        ops = inputs.hadamard_all(n)
        for _ in range(k):
            ops = ops + [inputs.flip_index(n, m)] + inputs.hadamard_all(n) \
                + [inputs.flip_index(n, 0)] + inputs.hadamard_all(n)
        psi = sv.simulate(n, ops)
        a_m, a_o = oc.grover_amplitudes(n, k)
        ref = np.full(1 << n, a_o, dtype=complex)
        ref[m] = a_m
        np.testing.assert_allclose(psi, ref, atol=1e-13)


def test_grover_generator_matches():
    ops, m = inputs.grover_circuit(6, 3, seed=3)
    psi = sv.simulate(6, ops)
    a_m, a_o = oc.grover_amplitudes(6, 3)
    assert abs(psi[m] - a_m) < 1e-13
    assert abs(psi[(m + 1) % 64] - a_o) < 1e-13


def test_monomial_trace_layered_against_simulation():
    n = 10
    ops = inputs.layered_circuit(n, 4, seed=2)
    psi = sv.simulate(n, ops)
    rng = np.random.default_rng(0)
    for i in rng.integers(0, 1 << n, size=20):
        a = oc.monomial_amplitude(n, ops[n:], int(i), lambda j: 2.0 ** (-n / 2))
        assert abs(a - psi[i]) < 1e-14


def test_monomial_trace_rejects_dense():
    with pytest.raises(ValueError):
        oc.monomial_amplitude(2, [inputs.op("H", (0,))], 0, lambda j: 1.0)


def test_qnn_single_qubit_closed_form():
    """One layer of the n = 2 ansatz, against expectations derived by hand
    (below)."""
    n = 2
    rng = np.random.default_rng(3)
    theta = rng.uniform(0, 2 * math.pi, size=(1, 2, n))
    psi = sv.simulate(n, inputs.ansatz_ops(n, theta))
    # product state after RY: qubit q has P(1) = sin^2(a_q / 2); RZ does
    # not change populations; CNOT(0->1) then CNOT(1->0) maps |b1 b0> to
    # bits (b0' = b0 xor b1 xor b0 = b1, b1' = b0 xor b1) so Z_0 afterwards
    # reads the old qubit 1: <Z_0> = cos(a_1), and Z_1 reads b0 xor b1.
    a0, a1 = theta[0, 0, 0], theta[0, 0, 1]
    assert sv.expect_z(psi, n, 0) == pytest.approx(math.cos(a1), abs=1e-14)
    assert sv.expect_z(psi, n, 1) == pytest.approx(math.cos(a0) * math.cos(a1), abs=1e-14)


def test_param_shift_closed_form_and_fd():
    n = 2
    rng = np.random.default_rng(4)
    theta = rng.uniform(0, 2 * math.pi, size=(1, 2, n))
    g = oc.param_shift_grad(n, theta, inputs.ansatz_ops, "zsum")
    a0, a1 = theta[0, 0, 0], theta[0, 0, 1]
    # f = cos(a1) + cos(a0) cos(a1)
    assert g[0, 0, 0] == pytest.approx(-math.sin(a0) * math.cos(a1), abs=1e-14)
    assert g[0, 0, 1] == pytest.approx(-math.sin(a1) - math.cos(a0) * math.sin(a1), abs=1e-14)
    assert np.allclose(g[0, 1], 0.0, atol=1e-14)       # RZ does not move populations here
    fd = oc.finite_diff_grad(n, theta, inputs.ansatz_ops, "zsum")
    np.testing.assert_allclose(g, fd, atol=1e-8)


def test_param_shift_matches_fd_deeper():
    n = 4
    theta = inputs.qnn_batch(1, n, 2, seed=9)[0]
    for obs in ("zsum", "z0"):
        g = oc.param_shift_grad(n, theta, inputs.ansatz_ops, obs)
        fd = oc.finite_diff_grad(n, theta, inputs.ansatz_ops, obs)
        np.testing.assert_allclose(g, fd, atol=1e-8)


def test_monomial_amplitudes_vectorised_equals_trace_and_simulation():
    """The array form of the single-path trace gives the scalar trace's
    value for every index, and the full simulation's."""
    n = 10
    ops = inputs.layered_circuit(n, 4, seed=2)
    psi = sv.simulate(n, ops)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 1 << n, size=64)
    init = lambda j: np.full(np.shape(j), 2.0 ** (-n / 2), dtype=complex)
    got = oc.monomial_amplitudes(n, ops[n:], idx, init)
    np.testing.assert_allclose(got, psi[idx], atol=1e-14, rtol=0)
    for i, a in zip(idx[:8], got[:8]):
        assert abs(a - oc.monomial_amplitude(n, ops[n:], int(i), lambda j: 2.0 ** (-n / 2))) <= 1e-16


def test_monomial_amplitudes_rejects_dense():
    with pytest.raises(ValueError):
        oc.monomial_amplitudes(2, [inputs.op("H", (0,))], [0, 1], lambda j: np.ones(np.shape(j)))


@pytest.mark.parametrize("n,L", [(2, 1), (3, 2), (5, 2)])
@pytest.mark.parametrize("obs", ["zsum", "z0"])
def test_adjoint_grad_matches_parameter_shift(n, L, obs):
    """The reverse sweep gives the value and every derivative of the exact
    parameter-shift rule (RY / RZ generators have eigenvalues +-1/2), and
    agrees with central differences."""
    theta = inputs.qnn_batch(1, n, L, seed=n * 10 + L)[0]
    f, g = oc.adjoint_grad(n, theta, inputs.ansatz_ops, obs)
    assert f == pytest.approx(oc.qnn_value(n, theta, inputs.ansatz_ops, obs), abs=1e-13)
    ps = oc.param_shift_grad(n, theta, inputs.ansatz_ops, obs)
    np.testing.assert_allclose(g, ps, atol=1e-12, rtol=0)
    fd = oc.finite_diff_grad(n, theta, inputs.ansatz_ops, obs)
    np.testing.assert_allclose(g, fd, atol=1e-8, rtol=0)


def test_adjoint_grad_closed_form_n2():
    """n = 2, one layer: f = cos(a1) + cos(a0) cos(a1) (derived in
    test_qnn_single_qubit_closed_form), so df/da0 = -sin(a0) cos(a1),
    df/da1 = -sin(a1) (1 + cos(a0)) and the RZ angles have zero gradient."""
    rng = np.random.default_rng(4)
    theta = rng.uniform(0, 2 * math.pi, size=(1, 2, 2))
    f, g = oc.adjoint_grad(2, theta, inputs.ansatz_ops, "zsum")
    a0, a1 = theta[0, 0, 0], theta[0, 0, 1]
    assert f == pytest.approx(math.cos(a1) + math.cos(a0) * math.cos(a1), abs=1e-14)
    assert g[0, 0, 0] == pytest.approx(-math.sin(a0) * math.cos(a1), abs=1e-14)
    assert g[0, 0, 1] == pytest.approx(-math.sin(a1) * (1 + math.cos(a0)), abs=1e-14)
    np.testing.assert_allclose(g[0, 1], 0.0, atol=1e-14)
