"""GPU parity on the paper-shaped workloads: the layered sparse-gate
circuit (n = 30, complex128, 16 GiB) and the Grover-style Hadamard-heavy
circuit (n = 33, complex128, 128 GiB), at reduced sizes against the full
oracle state and at full size on sampled amplitudes the oracle computes one
by one (monomial path tracing; Grover closed form)."""
import gc

import numpy as np
import pytest

from oracle import circuits as oc
from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import TOL, lib_ready, max_err, new_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


def _free():
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["per_gate", "fused"])
def test_layered_reduced(dtype, mode):
    n = 18
    ops = inputs.layered_circuit(n, 20, seed=2)
    s = new_state(n, dtype)
    s.apply_circuit(ops, mode=mode)
    ref = sv.simulate(n, ops)
    err = max_err(s.to_numpy(), ref)
    print(f"layered n={n} {dtype} {mode}: max |d amp| = {err:.3e}")
    assert err <= TOL[dtype]
    nrm, z0, _ = s.observables(0)
    tol = 1e-12 if dtype == "c128" else 1e-5
    assert abs(nrm - 1.0) <= tol
    assert abs(z0 - sv.expect_z(ref, n, 0)) <= tol


@pytest.mark.parametrize("mode", ["fused", "per_gate"])
def test_layered_full_n30_sampled(mode):
    """Full size, the launch configuration the benchmark times (fused)."""
    n = 30
    ops = inputs.layered_circuit(n, 20, seed=2)
    s = new_state(n, "c128")
    s.apply_circuit(ops, mode=mode)
    nrm, z0, _ = s.observables(0)
    rng = np.random.default_rng(7)
    idx = np.concatenate([[0, 1, (1 << n) - 1], rng.integers(0, 1 << n, size=29)])
    got = s.amplitudes(idx)
    s.close()
    del s
    _free()
    body = ops[n:]
    amp0 = lambda j: 2.0 ** (-n / 2)
    worst = 0.0
    for i, a in zip(idx, got):
        ref = oc.monomial_amplitude(n, body, int(i), amp0)
        worst = max(worst, abs(a - ref))
    print(f"layered n=30 {mode}: sampled max |d amp| = {worst:.3e}, norm-1 = {nrm - 1:.3e}, <Z0> = {z0:.3e}")
    assert worst <= 1e-12
    assert abs(nrm - 1.0) <= 1e-12
    # every gate after the H layer is a phase times a permutation, so all
    # probabilities stay 2^-n and <Z_0> = 0
    assert abs(z0) <= 1e-12


@pytest.mark.parametrize("n", [12, 20])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_grover_reduced(n, dtype):
    ops, m = inputs.grover_circuit(n, 8, seed=3)
    s = new_state(n, dtype)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    ref = sv.simulate(n, ops)
    assert max_err(got, ref) <= TOL[dtype]
    a_m, a_o = oc.grover_amplitudes(n, 8)
    assert abs(got[m] - a_m) <= TOL[dtype]
    assert s.argmax()[0] == m


def test_grover_full_n33_closed_form():
    n = 33
    ops, m = inputs.grover_circuit(n, 8, seed=3)
    s = new_state(n, "c128")
    s.apply_circuit(ops, mode="fused")
    nrm = s.norm2()
    am = s.argmax()[0]
    rng = np.random.default_rng(33)
    idx = np.concatenate([[m, 0, 1, (1 << n) - 1], rng.integers(0, 1 << n, size=60)])
    got = s.amplitudes(idx)
    s.close()
    del s
    _free()
    a_m, a_o = oc.grover_amplitudes(n, 8)
    ref = np.where(idx == m, a_m, a_o)
    abs_err = np.max(np.abs(got - ref))
    rel_err = np.max(np.abs(got - ref) / np.abs(ref))
    print(f"grover n=33: max |d amp| = {abs_err:.3e}, max rel = {rel_err:.3e}, norm-1 = {nrm - 1:.3e}")
    assert abs_err <= 1e-12
    assert rel_err <= 1e-9
    assert am == m
    assert abs(nrm - 1.0) <= 1e-12
