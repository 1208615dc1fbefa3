"""The paper's four RH sign methods as GPU kernels (Sec. III-B.2, Table II,
Algorithm 1): results against the oracle's own four methods and against
the butterfly path, sign-computation counts against the oracle's counters,
Table II and the n = 5 worked examples."""
import numpy as np
import pytest

from oracle import rh as orh
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import TOL, lib_ready, max_err, new_state

pytestmark = pytest.mark.gpu

ORACLE = {"nonopt": orh.mvm_nonopt, "quarter": orh.mvm_quarter, "block": orh.mvm_block, "log": orh.mvm_log}


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


def _run(n, method, psi, block=0):
    from paper_2411_15332_gb300 import rh_mvm
    src = new_state(n, "c128", psi)
    dst = new_state(n, "c128")
    cnt = rh_mvm(src, dst, method, block)
    out = dst.to_numpy()
    src.close()
    dst.close()
    return out, cnt


def _default_b(n):
    return 1 << ((n - 1) // 2)


@pytest.mark.parametrize("method", ["nonopt", "quarter", "block", "log"])
@pytest.mark.parametrize("n", [2, 3, 5, 7, 8])
def test_methods_match_oracle_methods(method, n):
    """Same S_next and the same number of compute_sign calls as the oracle's
    literal implementation of each method."""
    psi = inputs.random_state(n, seed=40 + n)
    got, cnt = _run(n, method, psi)
    ref, rcnt = ORACLE[method](orh.RH(n), psi)
    assert max_err(got, ref) <= TOL["c128"]
    assert cnt == rcnt


@pytest.mark.parametrize("n", [12, 14, 16, 18])
def test_methods_match_butterflies_and_table2(n):
    """At the paper's sizes (Fig. 8 spans n = 12..17): every method equals
    H^(x)n applied by the butterfly path, and its count is Table II's."""
    psi = inputs.random_state(n, seed=n)
    ref = new_state(n, "c128", psi)
    ref.hadamard_layer((1 << n) - 1)
    want = ref.to_numpy()
    ref.close()
    for method in (["quarter", "block", "log"] if n == 18 else ["nonopt", "quarter", "block", "log"]):
        got, cnt = _run(n, method, psi)
        assert max_err(got, want) <= TOL["c128"], method
        b = _default_b(n)
        assert cnt == orh.sign_count_formula(method, n, b if method == "block" else None), method


def test_n5_worked_examples(golden):
    """Fig. 4 (n = 5): quarter-based 16 rows x 16 signs; block-based 9 signs
    per row with b = 2 and 7 with b = 4; logarithm-based 5 per row counting
    the trivial sign at column 0."""
    n, h = 5, 16
    psi = inputs.random_state(n, seed=5)
    for row in golden("rh_examples.txt"):
        kind = row[0]
        if kind == "quarter":
            _, cnt = _run(n, "quarter", psi)
            assert cnt == int(row[2]) * int(row[3])
        elif kind == "block":
            _, cnt = _run(n, "block", psi, block=int(row[2]))
            assert cnt == h * int(row[3])
        elif kind == "log":
            _, cnt = _run(n, "log", psi)
            assert cnt + h == h * int(row[2])


def test_block_sizes():
    """Any power-of-two block size gives the same result and the count
    2^(n-1) (2^(n-1)/b + b - 1); Theorem 3's b = sqrt(2^(n-1)) is the
    smallest count."""
    n = 9
    psi = inputs.random_state(n, seed=9)
    ref, _ = _run(n, "quarter", psi)
    counts = {}
    for b in (1, 2, 4, 16, 64, 256):
        got, cnt = _run(n, "block", psi, block=b)
        assert max_err(got, ref) <= TOL["c128"]
        assert cnt == orh.sign_count_formula("block", n, b)
        counts[b] = cnt
    assert min(counts, key=counts.get) == 16          # sqrt(2^8)


def test_rejects_bad_arguments():
    from paper_2411_15332_gb300 import _lib as L
    from paper_2411_15332_gb300 import rh_mvm
    a, b = new_state(6, "c128"), new_state(6, "c128")
    with pytest.raises(L.MeraError):
        rh_mvm(a, a, "log")                          # out of place only
    with pytest.raises(L.MeraError):
        rh_mvm(a, b, "block", block=3)               # not a power of two
    c64 = new_state(6, "c64")
    with pytest.raises(L.MeraError):
        rh_mvm(c64, b, "log")
    big_a, big_b = new_state(19, "c128"), new_state(19, "c128")
    with pytest.raises(L.MeraError):
        rh_mvm(big_a, big_b, "log")
