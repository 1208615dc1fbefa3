"""DAX and DAS compressed structures, their MTP and MVM (Sec. III-A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

DAX (Sec. III-A.1, Fig. 1a): one entry per non-zero element holding the
element's real and imaginary parts (float64) and its "decimal" index, the
row-major linear index row * cols + col (int64); 24 bytes per entry.

DAS (Sec. III-A.1, Fig. 1b): one entry per non-zero holding the value and a
64-bit distance word.  Reading of the paper (its Fig. 1b is not
available): the low 63 bits count the zeros between this non-zero and the
previous non-zero of the same row (or the row start), and the top bit
(bit 63) is set when the element is the last non-zero of its row.  Zeros
after the last non-zero are implicit (cols - 1 - last column).

MTP (Sec. III-A.2, Fig. 2): the result has nnz(A) * nnz(B) entries (the
count the paper states, Theorem 1 in entry form); values are products;
the DAX index is the binary concatenation of the row indices and of the
column indices; the DAS distance follows the paper's three-case distance
equation.  Reading: the result is in canonical row-major order (ascending
linear index), which is also the order of the DAS row-pair traversal.

MVM (Sec. III-A.2): for every entry parse row r and column c and add
value * S[c] into S_next[r].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LAST_FLAG = np.uint64(1) << np.uint64(63)
DIST_MASK = LAST_FLAG - np.uint64(1)
ENTRY_BYTES = 24          # re (8) + im (8) + index or distance (8)


@dataclass
class DAX:
    dim: int                   # square matrix of dim x dim
    index: np.ndarray          # int64 (uint64 for dim > 2^31), row-major linear index
    value: np.ndarray          # complex128

    @property
    def nnz(self) -> int:
        return int(self.index.size)

    @property
    def nbytes(self) -> int:
        return ENTRY_BYTES * self.nnz


@dataclass
class DAS:
    dim: int
    dist: np.ndarray           # uint64: zeros before the element | LAST_FLAG
    value: np.ndarray          # complex128

    @property
    def nnz(self) -> int:
        return int(self.dist.size)

    @property
    def nbytes(self) -> int:
        return ENTRY_BYTES * self.nnz


# ------------------------------------------------------------------- DAX ---

def dax_encode(M: np.ndarray) -> DAX:
    """Scan the matrix row by row and keep each non-zero with its index
    (np.nonzero walks a C-ordered array in row-major order)."""
    dim = M.shape[0]
    r, c = np.nonzero(M)
    idx = r.astype(np.uint64) * np.uint64(dim) + c.astype(np.uint64)
    return DAX(dim, idx, M[r, c].astype(np.complex128))


def dax_decode(d: DAX) -> np.ndarray:
    M = np.zeros((d.dim, d.dim), dtype=np.complex128)
    r = (d.index // np.uint64(d.dim)).astype(np.int64)
    c = (d.index % np.uint64(d.dim)).astype(np.int64)
    M[r, c] = d.value
    return M


def dax_mtp(A: DAX, B: DAX) -> DAX:
    """A (x) B.  Every pair (a, b) of entries gives one result entry: value
    a * b; row (r_a r_b)_2 = r_a * B.dim + r_b; column (c_a c_b)_2; index
    row * (A.dim * B.dim) + column.  The entries are then put in ascending
    index order (row-major)."""
    dB = np.uint64(B.dim)
    dC = np.uint64(A.dim) * dB
    ra, ca = A.index // np.uint64(A.dim), A.index % np.uint64(A.dim)
    rb, cb = B.index // dB, B.index % dB
    # all pairs, a outer and b inner
    ra2, ca2 = np.repeat(ra, B.nnz), np.repeat(ca, B.nnz)
    rb2, cb2 = np.tile(rb, A.nnz), np.tile(cb, A.nnz)
    row = ra2 * dB + rb2
    col = ca2 * dB + cb2
    idx = row * dC + col
    val = np.repeat(A.value, B.nnz) * np.tile(B.value, A.nnz)
    order = np.argsort(idx, kind="stable")
    return DAX(int(dC), idx[order], val[order])


def dax_mvm(d: DAX, S: np.ndarray) -> np.ndarray:
    """S_next[r] += M[r][c] * S[c] over the entries (out of place)."""
    r = (d.index // np.uint64(d.dim)).astype(np.int64)
    c = (d.index % np.uint64(d.dim)).astype(np.int64)
    out = np.zeros(d.dim, dtype=np.complex128)
    np.add.at(out, r, d.value * S[c])
    return out


# ------------------------------------------------------------------- DAS ---

def das_encode(M: np.ndarray) -> DAS:
    dim = M.shape[0]
    dist, val = [], []
    for r in range(dim):
        cols = [int(c) for c in np.nonzero(M[r])[0]]
        prev = -1
        for j, c in enumerate(cols):
            w = np.uint64(c - prev - 1)
            if j == len(cols) - 1:
                w |= LAST_FLAG
            dist.append(w)
            val.append(M[r, c])
            prev = c
    return DAS(dim, np.array(dist, dtype=np.uint64), np.array(val, dtype=np.complex128))


def das_rows(d: DAS):
    """Parse the entry stream into rows: a list (one per row) of
    (entry positions, columns).  A row ends at an entry with the flag."""
    rows, pos, cols = [], [], []
    prev = -1
    for p in range(d.nnz):
        w = d.dist[p]
        c = prev + int(w & DIST_MASK) + 1
        pos.append(p)
        cols.append(c)
        prev = c
        if w & LAST_FLAG:
            rows.append((pos, cols))
            pos, cols, prev = [], [], -1
    if pos:
        rows.append((pos, cols))
    return rows


def das_decode(d: DAS) -> np.ndarray:
    M = np.zeros((d.dim, d.dim), dtype=np.complex128)
    for r, (pos, cols) in enumerate(das_rows(d)):
        for p, c in zip(pos, cols):
            M[r, c] = d.value[p]
    return M


def das_mtp(A: DAS, B: DAS) -> DAS:
    """A (x) B with the paper's distance equation.  Row pairs (r_a, r_b) in
    result-row order; inside a row pair, A's entries outer and B's inner.
    For entries A_i of row r_a and B_i of row r_b:
      case1  (A_i and B_i both first of their rows):  A_i.dis * B.col + B_i.dis
      case2  (B_i first, A_i not first):              A_i.dis * B.col + B_i.dis + B_last_dis
      otherwise:                                      B_i.dis
    where B.col is B's column count and B_last_dis the zeros after the last
    non-zero of row r_b.  The flag is set when both are last in their rows."""
    rowsA, rowsB = das_rows(A), das_rows(B)
    dist, val = [], []
    for posA, colsA in rowsA:
        for posB, colsB in rowsB:
            b_last_dis = B.dim - 1 - colsB[-1]
            for ia, pa in enumerate(posA):
                a_dis = int(A.dist[pa] & DIST_MASK)
                a_last = ia == len(posA) - 1
                for ib, pb in enumerate(posB):
                    b_dis = int(B.dist[pb] & DIST_MASK)
                    b_last = ib == len(posB) - 1
                    if ia == 0 and ib == 0:
                        w = a_dis * B.dim + b_dis
                    elif ib == 0:
                        w = a_dis * B.dim + b_dis + b_last_dis
                    else:
                        w = b_dis
                    w = np.uint64(w)
                    if a_last and b_last:
                        w |= LAST_FLAG
                    dist.append(w)
                    val.append(A.value[pa] * B.value[pb])
    return DAS(A.dim * B.dim, np.array(dist, dtype=np.uint64), np.array(val, dtype=np.complex128))


def das_mvm(d: DAS, S: np.ndarray) -> np.ndarray:
    out = np.zeros(d.dim, dtype=np.complex128)
    for r, (pos, cols) in enumerate(das_rows(d)):
        for p, c in zip(pos, cols):
            out[r] += d.value[p] * S[c]
    return out


def das_to_dax(d: DAS) -> DAX:
    idx, val = [], []
    for r, (pos, cols) in enumerate(das_rows(d)):
        for p, c in zip(pos, cols):
            idx.append(r * d.dim + c)
            val.append(d.value[p])
    return DAX(d.dim, np.array(idx, dtype=np.uint64), np.array(val, dtype=np.complex128))


# ------------------------------------------------------------- layers -----

def layer_dax(factors) -> DAX:
    """Operation matrix of a layer of gates on consecutive qubit blocks,
    as the DAX MTP chain factors[0] (x) factors[1] (x) ... (first factor on
    the most significant qubits, Eq. 6 generalised to several gates)."""
    out = dax_encode(np.asarray(factors[0]))
    for f in factors[1:]:
        out = dax_mtp(out, dax_encode(np.asarray(f)))
    return out


def memory_model_bytes(nnz: int, n_amps: int) -> int:
    """Bytes of one compressed stage: 24 B per entry plus a 16 B complex128
    amplitude per state-vector element."""
    return ENTRY_BYTES * nnz + 16 * n_amps
