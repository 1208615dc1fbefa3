"""Capacity: complex128 states of n = 34 qubits (256 GiB, 2^34 amplitudes),
the GPU counterpart of the paper's 34-qubit runs (Sec. IV-B Fig. 5, Table
IV).  There is no room for a second state-sized buffer, so every pass runs
in place.  Grover is checked on all 2^34 amplitudes against its closed
form; the layered circuit on all 2^34 magnitudes (every amplitude keeps
2^-17 after the H layer) and on 4096 amplitudes traced by the oracle."""
import gc

import numpy as np
import pytest

from oracle import circuits as oc
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import lib_ready, new_state
from tests.test_gpu_workloads import _max_abs_dev, grover_full_state_error

pytestmark = pytest.mark.gpu

N_CAP = 34


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()
    import torch
    free, total = torch.cuda.mem_get_info()
    if total < (16 << N_CAP) + (8 << 30):
        pytest.skip(f"needs a device with more than {(16 << N_CAP) >> 30} GiB")


def _free():
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_grover_n34_in_place():
    n = N_CAP
    ops, m = inputs.grover_circuit(n, 8, seed=3)
    s = new_state(n, "c128")
    s.apply_circuit(ops, mode="fused")
    nrm = s.norm2()
    am = s.argmax()[0]
    s.close()
    a_m, a_o = oc.grover_amplitudes(n, 8)
    abs_err, rel_err = grover_full_state_error(s.tensor, n, m, a_m, a_o)
    s.tensor = None
    del s
    _free()
    print(f"grover n=34: max |d amp| = {abs_err:.3e}, max rel = {rel_err:.3e} (all 2^34), norm-1 = {nrm - 1:.3e}")
    assert abs_err <= 1e-12
    assert rel_err <= 1e-9
    assert am == m
    assert abs(nrm - 1.0) <= 1e-12


def test_layered_n34_in_place():
    n = N_CAP
    ops = inputs.layered_circuit(n, 20, seed=2)
    s = new_state(n, "c128")
    s.apply_circuit(ops, mode="fused")
    nrm, z0, _ = s.observables(0)
    rng = np.random.default_rng(34)
    idx = np.concatenate([[0, 1, (1 << n) - 1], rng.integers(0, 1 << n, size=4093)])
    got = s.amplitudes(idx)
    s.close()
    mag = _max_abs_dev(s.tensor, 2.0 ** (-n / 2))
    s.tensor = None
    del s
    _free()
    init = lambda j: np.full(np.shape(j), 2.0 ** (-n / 2), dtype=complex)
    ref = oc.monomial_amplitudes(n, ops[n:], idx, init)
    worst = float(np.max(np.abs(got - ref)))
    print(f"layered n=34: traced max |d amp| = {worst:.3e} (4096), max ||amp| - 2^-17| = {mag:.3e} (all 2^34), "
          f"norm-1 = {nrm - 1:.3e}, <Z0> = {z0:.3e}")
    assert worst <= 1e-12
    assert mag <= 1e-12
    assert abs(nrm - 1.0) <= 1e-12
    assert abs(z0) <= 1e-12
