"""The C ABI library loads and exports every function include/mera.h
declares; host-only calls behave (no GPU needed).  CPU only."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import gates as og
from tests.conftest import ROOT

HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s+\**\s*(mera_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2411_15332_gb300.build import build
    build()
    from paper_2411_15332_gb300 import _lib as L
    return L


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("mera_state_create", "mera_apply_gate", "mera_apply_circuit", "mera_hadamard_layer",
                 "mera_expect_z", "mera_norm2"):
        assert must in names


def test_every_declared_symbol_exported(lib):
    so = C.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    assert set(declared_functions()) <= set(lib.PROTOS), set(declared_functions()) - set(lib.PROTOS)


def test_version_and_errors(lib):
    L = lib.lib()
    assert b"sm_103a" in L.mera_version()
    st = L.mera_apply_gate(None, 1, None, 0, None, 0, None)
    assert st == lib.MERA_EINVAL
    assert b"NULL" in L.mera_last_error()
    out = C.c_void_p()
    assert L.mera_state_create(0, 1, C.byref(out)) == lib.MERA_EINVAL
    assert L.mera_state_create(5, 7, C.byref(out)) == lib.MERA_EUNSUPPORTED


GATES = [g for g in og.GATE_ARITY if g not in ("FLIP",)]


@pytest.mark.parametrize("name", GATES)
def test_gate_matrix_matches_oracle(name, lib):
    """The library's catalogue equals the oracle's textbook matrices."""
    from paper_2411_15332_gb300 import core
    k, npar = og.GATE_ARITY[name]
    rng = np.random.default_rng(hash(name) % 2 ** 32)
    params = tuple(rng.uniform(0, 6.2, size=npar))
    got = core.gate_matrix(name, params)
    np.testing.assert_allclose(got, og.matrix(name, params), atol=1e-15)


def test_gate_matrix_rejects_nan(lib):
    from paper_2411_15332_gb300 import core
    with pytest.raises(lib.MeraError):
        core.gate_matrix("RX", (float("nan"),))
