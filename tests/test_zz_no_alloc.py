"""The allocation-free readout entry point (mera_observables_noalloc) for
callers that cannot let the library call cudaMalloc: it must give the same
norm^2, <Z_q> and sum_q <Z_q> as mera_observables, call after call, although
every call reuses one fixed device scratch array.  Collected last on
purpose."""
import ctypes as C

import numpy as np
import pytest

from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import lib_ready, new_state, obs_tol

pytestmark = pytest.mark.gpu


def _noalloc(state, q):
    import torch
    from paper_2411_15332_gb300 import _lib as L
    out = (C.c_double * 3)()
    code = L.MERA_C128 if state.dtype == "c128" else L.MERA_C64
    L.check(L.lib().mera_observables_noalloc(C.c_void_p(state.tensor.data_ptr()), state.n, code, q,
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream), out))
    return tuple(out)


def test_noalloc_matches_observables_on_consecutive_calls():
    """Same sums as the allocating entry point, call after call, and as the
    FP64 oracle's readouts of the same host state."""
    lib_ready()
    host = {14: inputs.random_state(14, seed=21), 9: inputs.random_state(9, seed=22).astype(np.complex64),
            22: inputs.random_state(22, seed=23)}
    a = new_state(14, "c128", host[14])
    b = new_state(9, "c64", host[9])
    c = new_state(22, "c128", host[22])
    for st, q in ((a, 3), (b, 8), (c, 0), (a, 13)):       # consecutive calls share the scratch array
        got = _noalloc(st, q)
        ref = st.observables(q)
        for g, r in zip(got, ref):
            assert abs(g - r) <= 1e-13, (st.n, q, got, ref)
        # the oracle reads the very amplitudes the device holds (complex64
        # states widened exactly), so only the summation order differs
        psi = host[st.n].astype(np.complex128)
        oref = (sv.norm2(psi), sv.expect_z(psi, st.n, q), sv.expect_z_sum(psi, st.n))
        for g, r, onorm in zip(got, oref, (1, 1, st.n)):
            assert abs(g - r) <= obs_tol("c128", onorm), (st.n, q, got, oref)


def test_noalloc_rejects_bad_sizes():
    lib_ready()
    from paper_2411_15332_gb300 import _lib as L
    a = new_state(6, "c128")
    out = (C.c_double * 3)()
    st = L.lib().mera_observables_noalloc(C.c_void_p(a.tensor.data_ptr()), 40, L.MERA_C128, 0, None, out)
    assert st == L.MERA_EINVAL
    assert b"outside" in L.lib().mera_last_error()
