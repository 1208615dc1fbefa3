"""GPU parity of the DAX / DAS structures (Sec. III-A): device MTP against
the oracle's MTP (index maps and distance words bit-exact, values within
1e-15), and the materialised MVM against the oracle's MVM."""
import numpy as np
import pytest

from oracle import dax as odx
from oracle import gates as og
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import TOL, lib_ready, max_err, new_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


def _dev(kind, M):
    from paper_2411_15332_gb300 import DAS, DAX
    return (DAX if kind == "dax" else DAS).from_dense(M)


def _check_dax(dev, ref):
    idx, val = dev.export()
    assert np.array_equal(idx, ref.index.astype(np.uint64))
    np.testing.assert_allclose(val, ref.value, rtol=0, atol=1e-15)


def _check_das(dev, ref):
    dist, val = dev.export()
    assert np.array_equal(dist, ref.dist.astype(np.uint64))
    np.testing.assert_allclose(val, ref.value, rtol=0, atol=1e-15)


def test_yx_example():
    Y, X = og.matrix("Y"), og.matrix("X")
    d = _dev("dax", Y).kron(_dev("dax", X))
    idx, val = d.export()
    assert list(idx) == [3, 6, 9, 12]
    assert list(val) == [-1j, -1j, 1j, 1j]
    assert d.nbytes == 96
    s = _dev("das", Y).kron(_dev("das", X))
    _check_das(s, odx.das_mtp(odx.das_encode(Y), odx.das_encode(X)))


def _rand_sparse(dim, density, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))
    M[rng.uniform(size=(dim, dim)) > density] = 0
    for r in range(dim):
        if not M[r].any():
            M[r, rng.integers(0, dim)] = 1.0
    return M


MATS = [og.matrix("Y"), og.matrix("H"), og.matrix("SWAP"), og.controlled(og.matrix("X"), 1),
        og.controlled(og.matrix("X"), 2), og.controlled(og.matrix("H"), 1), og.matrix("RXX", (0.3,)),
        _rand_sparse(4, 0.4, 1), _rand_sparse(8, 0.2, 2), _rand_sparse(16, 0.1, 3)]


@pytest.mark.parametrize("a", range(len(MATS)))
@pytest.mark.parametrize("b", [0, 2, 4, 7, 9])
def test_mtp_pairs(a, b):
    A, B = MATS[a], MATS[b]
    _check_dax(_dev("dax", A).kron(_dev("dax", B)), odx.dax_mtp(odx.dax_encode(A), odx.dax_encode(B)))
    _check_das(_dev("das", A).kron(_dev("das", B)), odx.das_mtp(odx.das_encode(A), odx.das_encode(B)))


@pytest.mark.parametrize("name,k,m", [("X", 1, 20), ("Y", 1, 12), ("SWAP", 2, 8), ("CNOT", 2, 6),
                                      ("TOFFOLI", 3, 4), ("H", 1, 9)])
def test_m_identical_gates_chain(name, k, m):
    """The Sec. IV-B workload: MTP of m identical gates, built on the device
    as a chain of pairwise MTPs; DAX index maps bit-exact at n = k * m."""
    G = {"CNOT": og.controlled(og.matrix("X"), 1), "TOFFOLI": og.controlled(og.matrix("X"), 2)}.get(name)
    if G is None:
        G = og.matrix(name)
    g = _dev("dax", G)
    acc = g
    ref = odx.dax_encode(G)
    for _ in range(m - 1):
        acc = acc.kron(g)
        ref = odx.dax_mtp(ref, odx.dax_encode(G))
    assert acc.nq == k * m
    _check_dax(acc, ref)
    if k * m <= 10:
        gs = _dev("das", G)
        acs = gs
        refs = odx.das_encode(G)
        for _ in range(m - 1):
            acs = acs.kron(gs)
            refs = odx.das_mtp(refs, odx.das_encode(G))
        _check_das(acs, refs)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["dax", "das"])
def test_mvm(dtype, kind):
    """Materialised MVM of a mixed layer operator, out of place."""
    factors = [og.controlled(og.matrix("X"), 2), og.matrix("H"), og.matrix("SWAP"), _rand_sparse(8, 0.3, 5)]
    M = factors[0]
    for f in factors[1:]:
        M = np.kron(M, f)
    nq = int(np.log2(M.shape[0]))
    dev = _dev(kind, factors[0])
    for f in factors[1:]:
        dev = dev.kron(_dev(kind, f))
    psi = inputs.random_state(nq, seed=nq)
    src = new_state(nq, dtype, psi)
    dst = new_state(nq, dtype)
    dev.mvm(src, dst)
    ref = odx.dax_mvm(odx.dax_encode(M), psi)
    assert max_err(dst.to_numpy(), ref) <= TOL[dtype]


def test_mvm_large_monomial_layer():
    """n = 24 monomial layer (Y on every qubit): one entry per row."""
    n = 24
    Y = og.matrix("Y")
    dev = _dev("dax", Y)
    for _ in range(n - 1):
        dev = dev.kron(_dev("dax", Y))
    assert dev.nnz == 1 << n
    psi = inputs.random_state(n, seed=2)
    src = new_state(n, "c128", psi)
    dst = new_state(n, "c128")
    dev.mvm(src, dst)
    # Y^(x)n |j> = i^n (-1)^popcount(~j) ... check against per-qubit oracle
    from oracle import statevector as sv
    ref = psi.copy()
    for q in range(n):
        sv.apply_op(ref, n, ("Y", (q,), (), (), 0))
    assert max_err(dst.to_numpy(), ref) <= 1e-12


def test_invalid_inputs():
    from paper_2411_15332_gb300 import DAS, DAX
    from paper_2411_15332_gb300 import _lib as L
    with pytest.raises(L.MeraError):
        DAX.from_host(2, [3, 1], [1.0, 1.0])          # not ascending
    with pytest.raises(L.MeraError):
        DAS.from_host(1, [0], [1.0])                  # row 0 never ends
    a = DAX.from_dense(np.eye(4))
    s1 = new_state(2, "c128")
    with pytest.raises(L.MeraError):
        a.mvm(s1, s1)                                 # in place is rejected
