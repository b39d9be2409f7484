"""Device operator product and linear combination (pauli_sum_product /
pauli_sum_add) against the oracle's letter-by-letter product, bit for bit:
masks, coefficients and the canonical order."""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _same(dev, ref):
    x, z, c = dev.export()
    assert np.array_equal(x, ref.x) and np.array_equal(z, ref.z)
    assert np.array_equal(c.real, ref.c.real) and np.array_equal(c.imag, ref.c.imag)


@pytest.mark.parametrize("n,ma,mb,seed", [(5, 40, 30, 1), (12, 300, 200, 2), (40, 500, 400, 3), (64, 600, 500, 4)])
def test_product_of_random_sums_bit_exact(ps, n, ma, mb, seed):
    xa, za, ga, ra, ia = w.random_pauli_terms(n, ma, seed)
    xb, zb, gb, rb, ib = w.random_pauli_terms(n, mb, seed + 100)
    A = ps.PauliSum.from_terms(n, xa, za, ra, ia, gamma=ga)
    B = ps.PauliSum.from_terms(n, xb, zb, rb, ib, gamma=gb)
    Ao = oracle.build_sum(n, xa, za, ga, ra, ia)
    Bo = oracle.build_sum(n, xb, zb, gb, rb, ib)
    _same(A @ B, oracle.sum_product(Ao, Bo))
    _same(B @ A, oracle.sum_product(Bo, Ao))
    _same(A.add(B, -1.0), oracle.sum_add(Ao, Bo, -1.0))


def test_molecular_products_and_commutators(ps):
    """H^2 of the 12-qubit molecule, and [H, N_alpha] = 0 to rounding."""
    h, g = w.MOL12.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    Ho = oracle.jw_hamiltonian(6, h, g, eps_drop=1e-12)
    _same(H @ H, oracle.sum_product(Ho, Ho))
    na_terms = [(1.0, [(p, 1), (p, 0)]) for p in range(6)]
    N = ps.PauliSum.jw_fermion(12, na_terms)
    No = oracle.fermion_sum(12, na_terms)
    C = H.commutator(N)
    Co = oracle.sum_add(oracle.sum_product(Ho, No), oracle.sum_product(No, Ho), -1.0)
    _same(C, Co)
    # [H, N_alpha] = 0: what survives is the rounding of the two products
    _, _, cc = C.export()
    assert np.abs(cc).max(initial=0.0) <= 1e-13 * np.abs(Ho.c).max()
    # anticommutator of ladder operators on the device: {a_p, a_q^dagger} = delta_pq I
    for p, q in [(0, 0), (1, 4), (3, 3)]:
        ap = ps.PauliSum.jw_fermion(12, [(1.0, [(p, 0)])])
        aq = ps.PauliSum.jw_fermion(12, [(1.0, [(q, 1)])])
        ac = (ap @ aq).add(aq @ ap, 1.0)
        x, z, c = ac.export()
        if p == q:
            assert ac.m == 1 and x[0] == 0 and z[0] == 0 and c[0] == 1.0
        else:
            assert ac.m == 0


def test_product_limits(ps):
    A = ps.PauliSum.from_terms(3, [1], [0], [1.0])
    B = ps.PauliSum.from_terms(4, [1], [0], [1.0])
    with pytest.raises(ps.PauliError) as e:
        A @ B
    assert e.value.code == ps.EINVAL
