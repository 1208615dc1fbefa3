"""Pins for the oracle's gate matrices (Table I catalogue) and the sparsity
theorems of Sec. II-C.  CPU only."""
import math

import numpy as np
import pytest

from oracle import gates as g
from oracle import statevector as sv
from tests.conftest import read_golden

RNG = np.random.default_rng(1234)


def _params(k):
    return tuple(RNG.uniform(0.1, 6.0, size=k))


@pytest.mark.parametrize("name", sorted(n for n in g.GATE_ARITY if n != "FLIP"))
def test_unitary(name):
    k, npar = g.GATE_ARITY[name]
    M = g.matrix(name, _params(npar))
    assert M.shape == (1 << k, 1 << k)
    np.testing.assert_allclose(M.conj().T @ M, np.eye(1 << k), atol=1e-14)


def test_paper_yx_dense():
    """The Y (x) X matrix printed in Sec. III-A.1 fixes Y, X and the
    Kronecker order (left factor on the most significant bit)."""
    rows = [r for r in read_golden("yx_example.txt") if r[0] == "dense_row"]
    M = np.zeros((4, 4), dtype=complex)
    for r in rows:
        i = int(r[1])
        for j, e in enumerate(r[2:]):
            re, im = (float(v) for v in e.split(","))
            M[i, j] = re + 1j * im
    assert np.array_equal(np.kron(g.matrix("Y"), g.matrix("X")), M)


def test_basis_actions():
    """Action on basis states, fixed by the definitions (not by the
    matrices' own code)."""
    k0 = np.array([1, 0], dtype=complex)
    k1 = np.array([0, 1], dtype=complex)
    assert np.array_equal(g.matrix("X") @ k0, k1)
    assert np.array_equal(g.matrix("Y") @ k0, 1j * k1)
    assert np.array_equal(g.matrix("Y") @ k1, -1j * k0)
    assert np.array_equal(g.matrix("Z") @ k1, -k1)
    assert np.array_equal(g.matrix("S") @ k1, 1j * k1)
    np.testing.assert_allclose(g.matrix("T") @ k1, (1 + 1j) / math.sqrt(2) * k1, atol=1e-16)
    np.testing.assert_allclose(g.matrix("H") @ k0, (k0 + k1) / math.sqrt(2), atol=1e-16)
    np.testing.assert_allclose(g.matrix("H") @ k1, (k0 - k1) / math.sqrt(2), atol=1e-16)
    th = 0.7
    # RY(theta)|0> = cos(theta/2)|0> + sin(theta/2)|1>
    np.testing.assert_allclose(g.matrix("RY", (th,)) @ k0,
                               math.cos(th / 2) * k0 + math.sin(th / 2) * k1, atol=1e-16)
    # RX(theta)|0> = cos(theta/2)|0> - i sin(theta/2)|1>
    np.testing.assert_allclose(g.matrix("RX", (th,)) @ k0,
                               math.cos(th / 2) * k0 - 1j * math.sin(th / 2) * k1, atol=1e-16)
    # RZ(theta) = diag(e^{-i theta/2}, e^{i theta/2})
    np.testing.assert_allclose(np.diag(g.matrix("RZ", (th,))),
                               [np.exp(-0.5j * th), np.exp(0.5j * th)], atol=1e-16)


def test_textbook_identities():
    H, X, Y, Z = (g.matrix(n) for n in "HXYZ")
    S, T = g.matrix("S"), g.matrix("T")
    np.testing.assert_allclose(H @ X @ H, Z, atol=1e-15)
    np.testing.assert_allclose(g.matrix("SX") @ g.matrix("SX"), X, atol=1e-15)
    np.testing.assert_allclose(g.matrix("SXDG") @ g.matrix("SX"), np.eye(2), atol=1e-15)
    assert np.array_equal(S @ S, Z)
    np.testing.assert_allclose(T @ T, S, atol=1e-15)
    np.testing.assert_allclose(g.matrix("TDG") @ T, np.eye(2), atol=1e-15)
    np.testing.assert_allclose(g.matrix("RX", (math.pi,)), -1j * X, atol=1e-15)
    np.testing.assert_allclose(g.matrix("RY", (math.pi,)), -1j * Y, atol=1e-15)
    th = 1.3
    np.testing.assert_allclose(g.matrix("RZ", (th,)), np.exp(-0.5j * th) * g.matrix("P", (th,)), atol=1e-15)
    np.testing.assert_allclose(g.matrix("U", (math.pi / 2, 0.0, math.pi)), H, atol=1e-15)
    np.testing.assert_allclose(g.matrix("U2", (0.3, 0.4)), g.matrix("U", (math.pi / 2, 0.3, 0.4)), atol=1e-15)
    np.testing.assert_allclose(g.matrix("R", (th, 0.0)), g.matrix("RX", (th,)), atol=1e-15)
    np.testing.assert_allclose(g.matrix("R", (th, math.pi / 2)), g.matrix("RY", (th,)), atol=1e-15)
    np.testing.assert_allclose(g.matrix("RXX", (math.pi,)), -1j * np.kron(X, X), atol=1e-15)
    np.testing.assert_allclose(g.matrix("RZZ", (th,)),
                               np.diag(np.exp(-0.5j * th * np.array([1, -1, -1, 1]))), atol=1e-15)
    # iSWAP^2 = Z (x) Z
    np.testing.assert_allclose(g.matrix("ISWAP") @ g.matrix("ISWAP"), np.kron(Z, Z), atol=1e-15)
    # SWAP exchanges |01> and |10>
    sw = g.matrix("SWAP")
    assert sw[2, 1] == 1 and sw[1, 2] == 1 and sw[0, 0] == 1 and sw[3, 3] == 1
    # DCX: |a b> -> |b, a xor b>
    dcx = g.matrix("DCX")
    for a in (0, 1):
        for b in (0, 1):
            assert dcx[b * 2 + (a ^ b), a * 2 + b] == 1
    # ECR is its own inverse
    np.testing.assert_allclose(g.matrix("ECR") @ g.matrix("ECR"), np.eye(4), atol=1e-15)


def test_controlled():
    X = g.matrix("X")
    cx = g.controlled(X, 1)
    assert np.array_equal(cx, np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]]))
    # control on |0>
    cx0 = g.controlled(X, 1, ctrl_values=0)
    assert np.array_equal(cx0, np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]]))
    ccx = g.controlled(X, 2)
    perm = np.arange(8)
    perm[[6, 7]] = [7, 6]
    assert np.array_equal(ccx, np.eye(8)[perm])


@pytest.mark.parametrize("row", read_golden("table1_zero_ratio.txt"), ids=lambda r: r[0])
def test_table1_zero_ratio(row):
    num, base, nc, npar, shape, ratio = row
    M = g.controlled(g.matrix(base, _params(int(npar))), int(nc))
    assert M.shape == (int(shape), int(shape))
    assert g.zero_ratio(M) == pytest.approx(float(ratio) / 100.0)


def test_theorem1_corollary_theorem2_property1():
    """Sec. II-C: R(A(x)B) = R(A) + (1 - R(A)) R(B) = R(B(x)A) >= max;
    R(A^(x)m) = 1 - (1 - R(A))^m, on catalogue gates."""
    mats = [g.matrix(n, _params(g.GATE_ARITY[n][1])) for n in ("H", "X", "S", "SWAP", "RXX", "ISWAP")]
    mats.append(g.controlled(g.matrix("H"), 1))
    for A in mats:
        for B in mats:
            rA, rB = g.zero_ratio(A), g.zero_ratio(B)
            rAB = g.zero_ratio(np.kron(A, B))
            assert rAB == pytest.approx(rA + (1 - rA) * rB)
            assert rAB == pytest.approx(g.zero_ratio(np.kron(B, A)))
            assert rAB >= max(rA, rB) - 1e-15
        for m in range(1, 4):
            Am = A
            for _ in range(m - 1):
                Am = np.kron(Am, A)
            assert g.zero_ratio(Am) == pytest.approx(1 - (1 - g.zero_ratio(A)) ** m)


@pytest.mark.parametrize("ratio,k,base,imprv", [
    (0.5, 1, 2.0, 2.0), (0.5, 2, 1.4142135623730951, 2.0 ** 0.5),
    (0.625, 2, 1.632993161855452, (8 / 3) ** 0.5), (0.75, 2, 2.0, 2.0), (0.875, 3, 2.0, 2.0)])
def test_table1_sparsity_and_memory_columns(ratio, k, base, imprv):
    """Table I 'Sparsity (n)' = 1 - 1/base^n and 'Mem imprv.' = 2/3 * imprv^n
    for m = n/k identical gates: Property 1 and 16 B dense vs 24 B DAX."""
    for n in (k, 2 * k, 3 * k, 6 * k):
        m = n // k
        sparsity = 1 - (1 - ratio) ** m
        assert sparsity == pytest.approx(1 - 1 / base ** n)
        dense = 16.0 * 4.0 ** n
        nnz = (1 - ratio) ** m * 4.0 ** n
        assert dense / (24.0 * nnz) == pytest.approx(2.0 / 3.0 * imprv ** n)


def test_flip_gate():
    psi = np.arange(8, dtype=complex) + 1
    sv.apply_matrix(psi, 3, g.matrix("FLIP"), [], [0, 1, 2], 0b101)
    ref = np.arange(8, dtype=complex) + 1
    ref[5] *= -1
    assert np.array_equal(psi, ref)
