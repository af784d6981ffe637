"""Pins of the GF(2^8) Reed-Solomon oracle (oracle/fec.py)."""
import numpy as np
import pytest

from oracle import fec as F


def test_field_axioms_over_all_elements():
    el = range(256)
    for a in el:
        assert F.gf_mul(a, 1) == a and F.gf_mul(a, 0) == 0
        if a:
            assert F.gf_mul(a, F.gf_inv(a)) == 1
    rng = np.random.default_rng(0)
    for a, b, c in rng.integers(0, 256, (3000, 3)):
        a, b, c = int(a), int(b), int(c)
        assert F.gf_mul(a, b) == F.gf_mul(b, a)
        assert F.gf_mul(F.gf_mul(a, b), c) == F.gf_mul(a, F.gf_mul(b, c))
        assert F.gf_mul(a, b ^ c) == F.gf_mul(a, b) ^ F.gf_mul(a, c)


def test_field_polynomial_and_generator_element():
    # x^8 = x^4 + x^3 + x^2 + 1 in this field; x (= 2) generates the 255 non-zero elements
    assert F.gf_mul(0x80, 2) == 0x1D
    seen, v = set(), 1
    for _ in range(255):
        seen.add(v)
        v = F.gf_mul(v, 2)
    assert len(seen) == 255 and v == 1


def test_systematic_and_any_n_of_n_plus_r_rebuild():
    rng = np.random.default_rng(1)
    for n, r in ((2, 1), (4, 2), (6, 3)):
        data = rng.integers(0, 256, (n, 5), dtype=np.uint8)
        parity = F.encode(data, r)
        shards = np.concatenate([data, parity])
        assert np.array_equal(shards[:n], data)
        for present in F.all_subsets(n, r):
            got = F.decode(n, r, list(present), shards[list(present)])
            assert np.array_equal(got, data), (n, r, present)


def test_parity_is_linear_and_single_parity_of_ones():
    rng = np.random.default_rng(2)
    a = rng.integers(0, 256, (5, 7), dtype=np.uint8)
    b = rng.integers(0, 256, (5, 7), dtype=np.uint8)
    assert np.array_equal(F.encode(a ^ b, 3), F.encode(a, 3) ^ F.encode(b, 3))
    # data = unit vector e_j: parity column = the Cauchy column j
    e = np.zeros((5, 1), np.uint8)
    e[2, 0] = 1
    assert [int(v) for v in F.encode(e, 3)[:, 0]] == [F.cauchy(5, 3)[i][2] for i in range(3)]


def test_too_few_packets_rejected():
    with pytest.raises(ValueError):
        F.decode(3, 2, [0, 1], np.zeros((2, 4), np.uint8))
