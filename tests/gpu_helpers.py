"""Helpers shared by the GPU parity tests."""
import numpy as np

TOL = {"c128": 1e-12, "c64": 2e-5}


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
