"""Helpers shared by the GPU parity tests."""
import numpy as np

# max |d amp| against the FP64 oracle, per state dtype
TOL = {"c128": 1e-12, "c64": 2e-5}


def obs_tol(dtype, onorm):
    """Bound for a quantity read from a state whose amplitudes meet TOL: an
    expectation <psi|O|psi> or an adjoint derivative 2 Re <lambda|dU|psi>
    with observable O of operator norm ``onorm`` (1 for Z_q, n for
    sum_q Z_q) is held to onorm * TOL[dtype]."""
    return onorm * TOL[dtype]


def lib_ready():
    from paper_2411_15332_gb300.build import build
    build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def new_state(n, dtype="c128", psi=None):
    from paper_2411_15332_gb300 import State
    s = State(n, dtype)
    if psi is not None:
        s.from_numpy(psi)
    return s


def max_err(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - np.asarray(b, dtype=np.complex128))))
