"""Gate matrices of the paper's forty-gate survey (Table I), FP64 complex.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper prints only Pauli-X and Pauli-Y (Sec. III-A.1, the Y (x) X
example).  Every other matrix is the textbook definition:

* rotations are exponentials of Paulis, ``R_P(theta) = exp(-i theta P / 2)
  = cos(theta/2) I - i sin(theta/2) P`` (valid because P^2 = I);
* RZ is the rotation above, so RZ != Phase (Table I lists RZ and Phase /
  U1 as distinct gates);
* a gate on k targets is a 2^k x 2^k matrix in the basis |t_0 t_1 ...>,
  where the first listed target is the most significant bit;
* controlled gates are not separate matrices here: a control list is
  attached to the base gate by ``controlled``.  Table I's CH, CSX, CU, CU3,
  CX, CY, CZ, CPhase, CRZ, CU1, CSwap and CCX are H, SX, U, U, X, Y, Z, P,
  RZ, P, SWAP and X with one or two controls.
"""
from __future__ import annotations

import math

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def _rot(P: np.ndarray, theta: float) -> np.ndarray:
    """exp(-i theta P / 2) for a Pauli product P (P @ P = I)."""
    d = P.shape[0]
    return math.cos(theta / 2) * np.eye(d, dtype=np.complex128) - 1j * math.sin(theta / 2) * P


def _u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def _cnot(n_ctrl_first: bool) -> np.ndarray:
    """CNOT on two qubits |a b>: control a, target b if n_ctrl_first, else
    control b, target a."""
    m = np.zeros((4, 4), dtype=np.complex128)
    for a in (0, 1):
        for b in (0, 1):
            if n_ctrl_first:
                a2, b2 = a, b ^ a
            else:
                a2, b2 = a ^ b, b
            m[a2 * 2 + b2, a * 2 + b] = 1.0
    return m


# name -> (number of targets, number of params)
GATE_ARITY = {
    "I": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0), "H": (1, 0),
    "S": (1, 0), "SDG": (1, 0), "T": (1, 0), "TDG": (1, 0),
    "SX": (1, 0), "SXDG": (1, 0),
    "P": (1, 1), "U1": (1, 1), "RX": (1, 1), "RY": (1, 1), "RZ": (1, 1),
    "R": (1, 2), "U2": (1, 2), "U": (1, 3), "U3": (1, 3),
    "SWAP": (2, 0), "ISWAP": (2, 0), "DCX": (2, 0), "ECR": (2, 0),
    "RXX": (2, 1), "RYY": (2, 1), "RZZ": (2, 1), "RZX": (2, 1),
    "FLIP": (0, 0),
}


def matrix(name: str, params=()) -> np.ndarray:
    """2^k x 2^k matrix of the base gate ``name``."""
    p = [float(v) for v in params]
    if name == "I":
        return I2.copy()
    if name == "X":
        return X.copy()
    if name == "Y":
        return Y.copy()
    if name == "Z":
        return Z.copy()
    if name == "H":
        return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    if name == "S":
        return np.diag([1.0, 1j]).astype(np.complex128)
    if name == "SDG":
        return np.diag([1.0, -1j]).astype(np.complex128)
    if name == "T":
        return np.diag([1.0, np.exp(1j * math.pi / 4)]).astype(np.complex128)
    if name == "TDG":
        return np.diag([1.0, np.exp(-1j * math.pi / 4)]).astype(np.complex128)
    if name == "SX":   # square root of Pauli-X, SX @ SX = X
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
    if name == "SXDG":
        return 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]], dtype=np.complex128)
    if name in ("P", "U1"):
        return np.diag([1.0, np.exp(1j * p[0])]).astype(np.complex128)
    if name == "RX":
        return _rot(X, p[0])
    if name == "RY":
        return _rot(Y, p[0])
    if name == "RZ":
        return _rot(Z, p[0])
    if name == "R":    # rotation by theta about cos(phi) X + sin(phi) Y
        return _rot(math.cos(p[1]) * X + math.sin(p[1]) * Y, p[0])
    if name == "U2":
        return _u3(math.pi / 2, p[0], p[1])
    if name in ("U", "U3"):
        m = _u3(p[0], p[1], p[2])
        if len(p) > 3:     # optional global phase gamma (CU carries it)
            m = m * np.exp(1j * p[3])
        return m
    if name == "SWAP":
        m = np.zeros((4, 4), dtype=np.complex128)
        for a in (0, 1):
            for b in (0, 1):
                m[b * 2 + a, a * 2 + b] = 1.0
        return m
    if name == "ISWAP":
        m = matrix("SWAP")
        m[1, 2] = m[2, 1] = 1j
        return m
    if name == "DCX":   # CNOT(t0 -> t1) followed by CNOT(t1 -> t0)
        return _cnot(False) @ _cnot(True)
    if name == "ECR":   # (I(x)X - X(x)Y) / sqrt(2)
        return (np.kron(I2, X) - np.kron(X, Y)) / math.sqrt(2.0)
    if name == "RXX":
        return _rot(np.kron(X, X), p[0])
    if name == "RYY":
        return _rot(np.kron(Y, Y), p[0])
    if name == "RZZ":
        return _rot(np.kron(Z, Z), p[0])
    if name == "RZX":
        return _rot(np.kron(Z, X), p[0])
    if name == "FLIP":
        return -np.ones((1, 1), dtype=np.complex128)
    raise ValueError(f"unknown gate {name}")


def controlled(G: np.ndarray, nc: int, ctrl_values: int | None = None) -> np.ndarray:
    """Matrix of G with ``nc`` controls, in the basis |c_0 ... c_{nc-1} t ...>
    (controls most significant, c_0 first).  G acts when control c_j holds
    bit j of ``ctrl_values`` (default all ones); identity elsewhere."""
    k = G.shape[0]
    if ctrl_values is None:
        ctrl_values = (1 << nc) - 1
    dim = k << nc
    m = np.eye(dim, dtype=np.complex128)
    # block index of the active control pattern: c_0 is the most significant
    blk = 0
    for j in range(nc):
        blk = (blk << 1) | ((ctrl_values >> j) & 1)
    m[blk * k:(blk + 1) * k, blk * k:(blk + 1) * k] = G
    return m


def zero_ratio(M: np.ndarray) -> float:
    """Fraction of exactly-zero entries (Table I column 'Ratio')."""
    return float(np.count_nonzero(M == 0)) / M.size


# Table I catalogue: number, name, (base gate, number of controls, params).
TABLE_I = [
    (1, "Hadamard", "H", 0, 0), (2, "SX", "SX", 0, 0), (3, "SXdg", "SXDG", 0, 0),
    (4, "R", "R", 0, 2), (5, "RX", "RX", 0, 1), (6, "RY", "RY", 0, 1),
    (7, "U", "U", 0, 3), (8, "U2", "U2", 0, 2), (9, "Identity", "I", 0, 0),
    (10, "Pauli-X", "X", 0, 0), (11, "Pauli-Y", "Y", 0, 0), (12, "Pauli-Z", "Z", 0, 0),
    (13, "S", "S", 0, 0), (14, "T", "T", 0, 0), (15, "T-adjoint", "TDG", 0, 0),
    (16, "Phase", "P", 0, 1), (17, "RZ", "RZ", 0, 1), (18, "U1", "U1", 0, 1),
    (19, "CCX", "X", 2, 0), (20, "CSwap", "SWAP", 1, 0),
    (21, "RXX", "RXX", 0, 1), (22, "RYY", "RYY", 0, 1), (23, "RZX", "RZX", 0, 1),
    (24, "ECR", "ECR", 0, 0), (25, "CH", "H", 1, 0), (26, "CSX", "SX", 1, 0),
    (29, "CU", "U", 1, 4), (30, "CU3", "U3", 1, 3),
    (31, "RZZ", "RZZ", 0, 1), (32, "Swap", "SWAP", 0, 0), (33, "iSwap", "ISWAP", 0, 0),
    (34, "Controlled-X", "X", 1, 0), (35, "Controlled-Y", "Y", 1, 0),
    (36, "Controlled-Z", "Z", 1, 0), (37, "DCX", "DCX", 0, 0), (38, "CPhase", "P", 1, 1),
    (39, "CRZ", "RZ", 1, 1), (40, "CU1", "U1", 1, 1),
]
