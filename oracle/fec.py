"""Reed-Solomon erasure code for I-frame packets (Section 3.2: an I-frame is
cut into n data packets, r = n/2 parity packets are added, and any n of the
n + r packets rebuild the frame).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests are the only
callers; the CUDA path never imports it.

The paper uses an RS erasure code without fixing its matrix; the reading taken
is a systematic code over GF(2^8) with the field polynomial
x^8 + x^4 + x^3 + x^2 + 1 (0x11D): packet i < n is data packet i; parity
packet i (0 <= i < r) is, byte by byte, sum_j C[i][j] * data[j] with the Cauchy
matrix C[i][j] = 1 / (x_i + y_j), x_i = n + i, y_j = j (distinct field
elements, so every square submatrix of [I; C] is invertible and any n packets
determine the data).  Decoding solves the n x n system of the received rows.

Arithmetic here is by definition, with no tables: multiplication is the
carry-less product reduced modulo the field polynomial, inversion is by
exponentiation (a^254).  Pinned by tests against field axioms over all
elements, the systematic property, and reconstruction from every n-subset on
small codes.
"""
from __future__ import annotations

import itertools

import numpy as np

POLY = 0x11D


def gf_mul(a: int, b: int) -> int:
    """Carry-less product of a and b reduced modulo POLY."""
    r = 0
    a &= 0xFF
    b &= 0xFF
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a & 0x100:
            a ^= POLY
    return r


def gf_pow(a: int, e: int) -> int:
    r = 1
    for _ in range(e):
        r = gf_mul(r, a)
    return r


def gf_inv(a: int) -> int:
    if a == 0:
        raise ZeroDivisionError("0 has no inverse in GF(2^8)")
    return gf_pow(a, 254)  # a^255 = 1 for a != 0


def cauchy(n: int, r: int) -> list[list[int]]:
    if n < 1 or r < 0 or n + r > 256:
        raise ValueError("need 1 <= n and n + r <= 256")
    return [[gf_inv((n + i) ^ j) for j in range(n)] for i in range(r)]


def generator(n: int, r: int) -> list[list[int]]:
    """The (n + r) x n systematic generator [I; C]."""
    ident = [[1 if i == j else 0 for j in range(n)] for i in range(n)]
    return ident + cauchy(n, r)


def encode(data: np.ndarray, r: int) -> np.ndarray:
    """data [n][S] uint8 -> parity [r][S] uint8."""
    data = np.asarray(data, dtype=np.uint8)
    n, S = data.shape
    C = cauchy(n, r)
    out = np.zeros((r, S), np.uint8)
    for i in range(r):
        for s in range(S):
            acc = 0
            for j in range(n):
                acc ^= gf_mul(C[i][j], int(data[j, s]))
            out[i, s] = acc
    return out


def invert(m: list[list[int]]) -> list[list[int]]:
    """Gauss-Jordan inverse over GF(2^8)."""
    k = len(m)
    a = [row[:] + [1 if i == j else 0 for j in range(k)] for i, row in enumerate(m)]
    for col in range(k):
        piv = next((rr for rr in range(col, k) if a[rr][col]), None)
        if piv is None:
            raise ValueError("singular")
        a[col], a[piv] = a[piv], a[col]
        inv = gf_inv(a[col][col])
        a[col] = [gf_mul(inv, v) for v in a[col]]
        for rr in range(k):
            if rr != col and a[rr][col]:
                f = a[rr][col]
                a[rr] = [x ^ gf_mul(f, y) for x, y in zip(a[rr], a[col])]
    return [row[k:] for row in a]


def decode(n: int, r: int, present: list[int], received: np.ndarray) -> np.ndarray:
    """received [n][S]: the packets whose indices (into data 0..n-1, parity
    n..n+r-1) are `present`, in that order -> data [n][S]."""
    received = np.asarray(received, dtype=np.uint8)
    if len(present) != n or len(set(present)) != n:
        raise ValueError("need n distinct packets")
    G = generator(n, r)
    inv = invert([G[p] for p in present])
    S = received.shape[1]
    out = np.zeros((n, S), np.uint8)
    for i in range(n):
        for s in range(S):
            acc = 0
            for j in range(n):
                acc ^= gf_mul(inv[i][j], int(received[j, s]))
            out[i, s] = acc
    return out


def all_subsets(n: int, r: int):
    return itertools.combinations(range(n + r), n)
