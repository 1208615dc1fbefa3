"""Pins for the oracle's DAX / DAS structures (Sec. III-A) and the RH
structure with its four MVM methods (Sec. III-B).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import circuits as oc
from oracle import dax as dx
from oracle import gates as g
from oracle import rh
from tests.conftest import read_golden

YX = {r[0]: r[1:] for r in read_golden("yx_example.txt") if r[0] != "dense_row"}


def _c(s):
    re, im = (float(v) for v in s.split(","))
    return re + 1j * im


# ------------------------------------------------------------------ DAX ---

def test_yx_dax_example():
    d = dx.dax_mtp(dx.dax_encode(g.matrix("Y")), dx.dax_encode(g.matrix("X")))
    assert [int(v) for v in d.index] == [int(v) for v in YX["dax_indices"]]
    assert d.nbytes == int(YX["dax_bytes"][0])
    assert 16 * 16 == int(YX["dense_bytes"][0])
    s = dx.das_mtp(dx.das_encode(g.matrix("Y")), dx.das_encode(g.matrix("X")))
    assert s.nbytes == int(YX["das_bytes"][0])


def test_fig2a_single_entry():
    """-i at index 1 of DAX(Y) times 1 at index 2 of DAX(X) -> index 6."""
    ia, ib, out, val = YX["mtp_entry"]
    A = dx.DAX(2, np.array([int(ia)], dtype=np.uint64), np.array([g.matrix("Y").flat[int(ia)]]))
    B = dx.DAX(2, np.array([int(ib)], dtype=np.uint64), np.array([g.matrix("X").flat[int(ib)]]))
    C = dx.dax_mtp(A, B)
    assert int(C.index[0]) == int(out)
    assert C.value[0] == _c(val)


def test_das_y_row0():
    before, behind, last = YX["das_y_row0"]
    s = dx.das_encode(g.matrix("Y"))
    w = s.dist[0]
    assert int(w & dx.DIST_MASK) == int(before)
    assert bool(w & dx.LAST_FLAG) == (last == "last")
    assert dx.das_rows(s)[0][1] == [1]
    assert 2 - 1 - 1 == int(behind)


def _random_sparse(dim, density, seed):
    rng = np.random.default_rng(seed)
    M = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim)))
    M[rng.uniform(size=(dim, dim)) > density] = 0
    for r in range(dim):          # no empty row (unitaries have none)
        if not M[r].any():
            M[r, rng.integers(0, dim)] = 1.0
    return M


MATS = [g.matrix("Y"), g.matrix("H"), g.matrix("SWAP"), g.controlled(g.matrix("H"), 1),
        g.controlled(g.matrix("X"), 2), g.matrix("RXX", (0.4,)), _random_sparse(4, 0.5, 1),
        _random_sparse(8, 0.3, 2), _random_sparse(2, 0.6, 3)]


@pytest.mark.parametrize("a", range(len(MATS)))
@pytest.mark.parametrize("b", range(len(MATS)))
def test_mtp_equals_kron(a, b):
    """DAX and DAS MTP decode to np.kron (library routine); entry count is
    the product (Theorem 1 in entry form); DAX order is row-major."""
    A, B = MATS[a], MATS[b]
    ref = np.kron(A, B)
    d = dx.dax_mtp(dx.dax_encode(A), dx.dax_encode(B))
    s = dx.das_mtp(dx.das_encode(A), dx.das_encode(B))
    nnzA, nnzB = np.count_nonzero(A), np.count_nonzero(B)
    assert d.nnz == s.nnz == nnzA * nnzB == np.count_nonzero(ref)
    # values: complex products may round differently by one ulp
    np.testing.assert_allclose(dx.dax_decode(d), ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(dx.das_decode(s), ref, rtol=0, atol=1e-15)
    assert np.array_equal(dx.dax_decode(d) != 0, ref != 0)
    assert np.array_equal(dx.das_decode(s) != 0, ref != 0)
    assert np.all(np.diff(d.index.astype(np.int64)) > 0)
    # DAS MTP equals DAS encoding of the dense product, bit for bit
    e = dx.das_encode(ref)
    np.testing.assert_array_equal(s.dist, e.dist)
    np.testing.assert_allclose(s.value, e.value, rtol=0, atol=1e-15)
    c = dx.das_to_dax(s)
    np.testing.assert_array_equal(c.index, d.index)


@pytest.mark.parametrize("m", range(len(MATS)))
def test_mvm_equals_dense(m):
    rng = np.random.default_rng(m)
    M = np.kron(MATS[m], MATS[(m + 1) % len(MATS)])
    S = rng.standard_normal(M.shape[0]) + 1j * rng.standard_normal(M.shape[0])
    np.testing.assert_allclose(dx.dax_mvm(dx.dax_encode(M), S), M @ S, atol=1e-12)
    np.testing.assert_allclose(dx.das_mvm(dx.das_encode(M), S), M @ S, atol=1e-12)


def test_layer_chain_m_identical():
    """m identical gates (Sec. IV-B): the DAX chain equals the Kronecker
    power and has (1-R)^m 4^n entries (Property 1)."""
    for name, k in (("X", 1), ("Y", 1), ("SWAP", 2)):
        G = g.matrix(name)
        for m in (1, 2, 3):
            d = dx.layer_dax([G] * m)
            ref = G
            for _ in range(m - 1):
                ref = np.kron(ref, G)
            np.testing.assert_array_equal(dx.dax_decode(d), ref)
            n = k * m
            assert d.nnz == round((1 - g.zero_ratio(G)) ** m * 4 ** n)


MEM = {r[0]: r[1:] for r in read_golden("memory_figures.txt")}


def test_memory_figures():
    n = int(MEM["table3_stage_kib"][0])
    N = 1 << n
    # a monomial stage has one entry per row
    assert dx.memory_model_bytes(N, N) == int(MEM["table3_stage_kib"][1]) * 1024
    dense = 16 * 4 ** n
    assert dense == int(MEM["table3_matrix_mib"][1]) * 2 ** 20
    assert dense / dx.memory_model_bytes(N, N) == pytest.approx(float(MEM["table3_saving"][0]))
    n = int(MEM["table4_matrix_gib"][0])
    assert 16 * 4 ** n == int(MEM["table4_matrix_gib"][1]) * 2 ** 30
    n = int(MEM["table4_dax_tb"][0])
    tib = dx.memory_model_bytes(1 << n, 1 << n) / 2 ** 40
    assert round(tib, 1) == pytest.approx(float(MEM["table4_dax_tb"][1]), abs=0.05)
    n = int(MEM["fig5_saving"][0])
    ratio = 16 * 4 ** n / (dx.ENTRY_BYTES * (1 << n))
    assert float(f"{ratio:.1e}") == float(MEM["fig5_saving"][1])


# ------------------------------------------------------------------- RH ---

RHX = read_golden("rh_examples.txt")


def test_rh_sign_example():
    for r in RHX:
        if r[0] == "sign":
            n, row, col, s = (int(v) for v in r[1:])
            assert rh.compute_sign(row, col, n) == s


def test_rh_sign_closed_form_and_sylvester():
    """The quadrant recursion equals (-1)^popcount(r & c) and the sign of
    scipy's Sylvester Hadamard matrix."""
    for n in range(1, 7):
        Hs = scipy.linalg.hadamard(1 << n)
        for r in range(1 << n):
            for c in range(1 << n):
                s = rh.compute_sign(r, c, n)
                assert s == (-1) ** bin(r & c).count("1")
                assert s == Hs[r, c]


def test_rh_value():
    for n in (1, 5, 17, 35):
        assert rh.RH(n).value == pytest.approx(2.0 ** (-n / 2), rel=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_rh_methods_equal_dense(n):
    rng = np.random.default_rng(n)
    S = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    ref = scipy.linalg.hadamard(1 << n) @ S / math.sqrt(1 << n)
    R = rh.RH(n)
    outs = {"nonopt": rh.mvm_nonopt(R, S), "quarter": rh.mvm_quarter(R, S), "log": rh.mvm_log(R, S)}
    for b in [1 << j for j in range(n)]:
        if (1 << (n - 1)) % b == 0 and b <= (1 << (n - 1)):
            outs[f"block{b}"] = rh.mvm_block(R, S, b)
    for name, (out, count) in outs.items():
        np.testing.assert_allclose(out, ref, atol=1e-13, err_msg=name)
        if name.startswith("block"):
            assert count == rh.sign_count_formula("block", n, int(name[5:]))
        else:
            assert count == rh.sign_count_formula(name, n)
    # and the butterfly route of the state-vector oracle
    psi = oc.hadamard_layer(S.copy(), n, (1 << n) - 1)
    np.testing.assert_allclose(psi, ref, atol=1e-13)


def test_table2_n5_examples():
    for r in RHX:
        kind = r[0]
        if kind == "quarter":
            n, rows, per = (int(v) for v in r[1:])
            h = 1 << (n - 1)
            assert (rows, per) == (h, h)
            assert rh.sign_count_formula("quarter", n) == rows * per
        elif kind == "block":
            n, b, per = (int(v) for v in r[1:])
            h = 1 << (n - 1)
            assert rh.sign_count_formula("block", n, b) == h * per
        elif kind == "log":
            n, per = (int(v) for v in r[1:])
            h = 1 << (n - 1)
            # Table II counts n-1 per row; the example also counts column 0
            assert rh.sign_count_formula("log", n) == h * (per - 1)
            _, count = rh.mvm_log(rh.RH(n), np.ones(1 << n, dtype=complex))
            assert count == h * (per - 1)


def test_theorem3_block_optimum():
    """b = sqrt(2^{n-1}) minimises 2^{n-1}/b + b - 1 (odd n: exact power)."""
    for n in (3, 5, 7, 9, 11):
        h = 1 << (n - 1)
        costs = {b: h // b + b - 1 for b in [1 << j for j in range(n)]}
        best = min(costs, key=costs.get)
        assert best == int(math.isqrt(h))
