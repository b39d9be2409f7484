"""Pins of the multi-word-mask oracle (oracle/wide.py): identical to the 64-bit
C oracle where both apply, and the canonical anticommutators above qubit 64."""
import numpy as np

import oracle
from oracle import wide
import workloads as w


def _as_list(S):
    return [(int(x), int(z), complex(c)) for x, z, c in zip(S.x, S.z, S.c)]


def _same(a, b):
    assert len(a) == len(b)
    for (xa, za, ca), (xb, zb, cb) in zip(a, b):
        assert xa == xb and za == zb and ca.real == cb.real and ca.imag == cb.imag


def _monomials(n, k, seed):
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(k):
        nf = int(rng.integers(1, 5))
        f = [(int(rng.integers(0, n)), int(rng.integers(0, 2))) for _ in range(nf)]
        terms.append((complex(rng.normal(), rng.normal()), f))
    return terms


def test_fermion_sums_equal_the_64_bit_oracle():
    for n, seed in [(8, 1), (40, 2), (64, 3)]:
        terms = _monomials(n, 60, seed)
        _same(wide.fermion_sum(n, terms), _as_list(oracle.fermion_sum(n, terms)))


def test_products_equal_the_64_bit_oracle():
    for n, seed in [(10, 4), (64, 5)]:
        xa, za, ga, ra, ia = w.random_pauli_terms(n, 40, seed)
        xb, zb, gb, rb, ib = w.random_pauli_terms(n, 30, seed + 1)
        A = oracle.build_sum(n, xa, za, ga, ra, ia)
        B = oracle.build_sum(n, xb, zb, gb, rb, ib)
        _same(wide.product(n, _as_list(A), _as_list(B)), _as_list(oracle.sum_product(A, B)))


def test_anticommutators_above_64_qubits():
    n = 150
    for P, Q in [(70, 70), (64, 149), (10, 100), (130, 129)]:
        a = wide.fermion_sum(n, [(1.0, [(P, 0)])])
        ad = wide.fermion_sum(n, [(1.0, [(Q, 1)])])
        ac = wide.add(wide.product(n, a, ad), wide.product(n, ad, a))
        if P == Q:
            assert ac == [(0, 0, 1 + 0j)]
        else:
            assert ac == []
        aa = wide.add(wide.product(n, a, a), [])
        assert aa == []  # a_P a_P = 0
