"""RH structure for H^{(x)n} and its MVM methods (Sec. III-B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

RH (Sec. III-B.1) stores one number, the common magnitude 1/sqrt(N) of
every element of H^{(x)n}; the sign of element (r, c) is parsed on demand.

Sign rule (Sec. III-B.2, Fig. 3): split the matrix into four quadrants;
only the lower-right one is negative; recurse into the quadrant holding
(r, c) and multiply the signs of all levels.

MVM methods, all out of place with S first scaled by the RH value
(Table II gives their sign-computation counts):

* non-optimised: a sign for every (r, c), 2^n * 2^n computations;
* quarter-based (Method 1): signs of the upper-left quarter only; the
  upper-right and lower-left quarters repeat them and the lower-right
  negates them, (2^{n-1})^2 computations;
* block-based (Method 2): each quarter row is cut into blocks of b; the
  first block is computed in full, every other block only at its first
  element, whose sign multiplies the first block's signs,
  2^{n-1} (2^{n-1}/b + b - 1) computations;
* logarithm-based (Method 3, Algorithm 1): per quarter row only the signs
  at columns 2^0, 2^1, ... are computed; any other column c takes
  sign[2^p] * sign[c - 2^p] with 2^p the largest power of two <= c.
  Reading: the paper's listing leaves p undefined; this reading is the
  only one that keeps the index inside the computed prefix.  Table II
  counts 2^{n-1} (n - 1) computations; the n = 5 example's "5 signs per
  row" also counts the trivial sign at column 0.

Every method returns (S_next, number of compute_sign calls).
"""
from __future__ import annotations

import math

import numpy as np


class RH:
    """H^{(x)n} as its single magnitude 1/sqrt(2^n)."""

    def __init__(self, n: int):
        self.n = n
        self.value = 1.0 / math.sqrt(float(1 << n))


def compute_sign(r: int, c: int, n: int) -> int:
    """Quadrant recursion of Fig. 3: O(n)."""
    s = 1
    size = 1 << n
    while size > 1:
        half = size >> 1
        if r >= half and c >= half:
            s = -s
        r %= half
        c %= half
        size = half
    return s


def mvm_nonopt(rh: RH, S: np.ndarray):
    N = 1 << rh.n
    Ss = rh.value * S
    out = np.zeros(N, dtype=np.complex128)
    count = 0
    for r in range(N):
        acc = 0j
        for c in range(N):
            s = compute_sign(r, c, rh.n)
            count += 1
            acc += s * Ss[c]
        out[r] = acc
    return out, count


def _accumulate_quarter(out, Ss, r, c, h, s):
    """Alg. 1 body: the four quarter updates of one upper-left sign."""
    out[r] += s * Ss[c]
    out[r] += s * Ss[c + h]
    out[r + h] += s * Ss[c]
    out[r + h] += -s * Ss[c + h]


def mvm_quarter(rh: RH, S: np.ndarray):
    N = 1 << rh.n
    h = N >> 1
    Ss = rh.value * S
    out = np.zeros(N, dtype=np.complex128)
    count = 0
    for r in range(h):
        for c in range(h):
            s = compute_sign(r, c, rh.n)
            count += 1
            _accumulate_quarter(out, Ss, r, c, h, s)
    return out, count


def mvm_block(rh: RH, S: np.ndarray, b: int | None = None):
    N = 1 << rh.n
    h = N >> 1
    if b is None:   # Theorem 3: b = sqrt(2^{n-1}) minimises the count
        b = 1 << ((rh.n - 1) // 2)
    assert b >= 1 and (b & (b - 1)) == 0 and h % b == 0
    Ss = rh.value * S
    out = np.zeros(N, dtype=np.complex128)
    count = 0
    for r in range(h):
        first = []
        for j in range(b):
            first.append(compute_sign(r, j, rh.n))
            count += 1
        for blk in range(h // b):
            if blk == 0:
                s0 = 1
            else:
                s0 = compute_sign(r, blk * b, rh.n)
                count += 1
            for j in range(b):
                _accumulate_quarter(out, Ss, r, blk * b + j, h, s0 * first[j])
    return out, count


def mvm_log(rh: RH, S: np.ndarray):
    N = 1 << rh.n
    h = N >> 1
    Ss = rh.value * S
    out = np.zeros(N, dtype=np.complex128)
    count = 0
    sign = [0] * h
    for r in range(h):
        for c in range(h):
            if c == 0:
                sign[c] = 1
            elif c & (c - 1) == 0:
                sign[c] = compute_sign(r, c, rh.n)
                count += 1
            else:
                p = 1 << (c.bit_length() - 1)
                sign[c] = sign[p] * sign[c - p]
            _accumulate_quarter(out, Ss, r, c, h, sign[c])
    return out, count


def sign_count_formula(method: str, n: int, b: int | None = None) -> int:
    """Table II."""
    N, h = 1 << n, 1 << (n - 1)
    if method == "nonopt":
        return N * N
    if method == "quarter":
        return h * h
    if method == "block":
        return h * (h // b + b - 1)
    if method == "log":
        return h * (n - 1)
    raise ValueError(method)
