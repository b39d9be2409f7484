"""Pins of the oracle's Pauli algebra (Sec. 2.2-2.3) against matrices and the paper's rules."""
import numpy as np
import pytest

import oracle
from oracle import dense
import workloads as w

LETTER_NAMES = "IXYZ"


def test_letter_product_table_matches_2x2_matrices():
    """sigma_u sigma_v = i^k sigma_w for all 16 ordered pairs (textbook table)."""
    for u in range(4):
        for v in range(4):
            wl, k = oracle.letter_mul(u, v)
            lhs = dense.SIGMA[u] @ dense.SIGMA[v]
            rhs = (1j ** k) * dense.SIGMA[wl]
            assert np.array_equal(lhs, rhs), (LETTER_NAMES[u], LETTER_NAMES[v])


def test_named_products():
    """XY = iZ, YZ = iX, ZX = iY, YX = -iZ and P^2 = I."""
    X, Y, Z, I = oracle.X, oracle.Y, oracle.Z, oracle.I
    assert oracle.letter_mul(X, Y) == (Z, 1)
    assert oracle.letter_mul(Y, Z) == (X, 1)
    assert oracle.letter_mul(Z, X) == (Y, 1)
    assert oracle.letter_mul(Y, X) == (Z, 3)
    for p in (I, X, Y, Z):
        assert oracle.letter_mul(p, p) == (I, 0)


def test_single_qubit_encoding_bit_pairs():
    """eq. single_pauli_mapping: I=(0,0), X=(1,0), Y=(1,1), Z=(0,1) (one-qubit strings)."""
    pairs = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}
    for (a1, b1) in pairs:
        for (a2, b2) in pairs:
            x, z, k = oracle.string_mul(1, a1, b1, a2, b2)
            lhs = dense.SIGMA["IXYZ".index(pairs[(a1, b1)])] @ dense.SIGMA["IXYZ".index(pairs[(a2, b2)])]
            rhs = (1j ** k) * dense.SIGMA["IXYZ".index(pairs[(x, z)])]
            assert np.array_equal(lhs, rhs)


def test_string_product_matches_kronecker():
    rng = np.random.default_rng(7)
    n = 5
    for _ in range(60):
        xa, za, xb, zb = (int(v) for v in rng.integers(0, 1 << n, 4))
        x, z, k = oracle.string_mul(n, xa, za, xb, zb)
        lhs = (dense.letter_string(n, xa, za) @ dense.letter_string(n, xb, zb)).toarray()
        rhs = (1j ** k) * dense.letter_string(n, x, z).toarray()
        assert np.allclose(lhs, rhs, atol=0, rtol=0)


def test_letter_product_agrees_with_symplectic_phase_rule():
    """eq. pauli_prod_x/z/phase: (X^xa Z^za)(X^xb Z^zb) = (-1)^popc(za & xb) X^(xa^xb) Z^(za^zb).

    The oracle multiplies letter strings with the textbook table; a letter string
    is i^#Y X^x Z^z, so the two phases must satisfy
    k + #Y(c) - #Y(a) - #Y(b) = 2 popc(za & xb)  (mod 4)."""
    rng = np.random.default_rng(8)
    n = 64
    ny = lambda x, z: bin(x & z).count("1")
    for _ in range(2000):
        xa, za, xb, zb = (int(v) for v in w.random_masks(rng, n, 4))
        x, z, k = oracle.string_mul(n, xa, za, xb, zb)
        assert x == xa ^ xb and z == za ^ zb
        assert (k + ny(x, z) - ny(xa, za) - ny(xb, zb)) % 4 == (2 * bin(za & xb).count("1")) % 4


def test_to_xz_matches_dense_matrices():
    """A letter-form term i^gamma c * letters equals C * X^x Z^z with C from to_xz."""
    rng = np.random.default_rng(9)
    n = 4
    x, z, gamma, cre, cim = w.random_pauli_terms(n, 40, 9)
    C = oracle.to_xz(n, x, z, gamma, cre, cim, letter_form=True)
    for j in range(len(x)):
        lhs = (1j ** int(gamma[j])) * complex(cre[j], cim[j]) * dense.letter_string(n, int(x[j]), int(z[j])).toarray()
        rhs = C[j] * dense.xz_string(n, int(x[j]), int(z[j])).toarray()
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-15)
    Cx = oracle.to_xz(n, x, z, gamma, cre, cim, letter_form=False)
    assert np.array_equal(Cx, (1j ** gamma.astype(int)) * (cre + 1j * cim))


def test_operator_product_matches_dense():
    """eq. pauli_operator_multiplication: canonical(A B) == A_dense @ B_dense."""
    n = 4
    for seed in range(4):
        x, z, gamma, cre, cim = w.random_pauli_terms(n, 12, seed)
        A = oracle.build_sum(n, x, z, gamma, cre, cim)
        x, z, gamma, cre, cim = w.random_pauli_terms(n, 9, 100 + seed)
        B = oracle.build_sum(n, x, z, gamma, cre, cim)
        AB = oracle.sum_product(A, B)
        lhs = dense.pauli_sum_matrix(n, AB.x, AB.z, AB.c)
        rhs = dense.pauli_sum_matrix(n, A.x, A.z, A.c) @ dense.pauli_sum_matrix(n, B.x, B.z, B.c)
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)


def _dict_merge(x, z, c, eps):
    """Brute-force canonical form: dictionary accumulation in input order."""
    acc = {}
    for xi, zi, ci in zip(x.tolist(), z.tolist(), c.tolist()):
        key = (xi, zi)
        if key in acc:
            acc[key] = complex(acc[key].real + ci.real, acc[key].imag + ci.imag)
        else:
            acc[key] = complex(ci)
    keys = sorted(k for k, v in acc.items() if v.real * v.real + v.imag * v.imag > eps * eps)
    return keys, [acc[k] for k in keys]


@pytest.mark.parametrize("n,m,eps", [(3, 50, 0.0), (10, 400, 0.0), (64, 300, 0.5), (24, 1000, 1e-3)])
def test_canonical_reduction_bit_exact_vs_dictionary(n, m, eps):
    x, z, gamma, cre, cim = w.random_pauli_terms(n, m, 1000 + n, dup_frac=0.6)
    c = cre + 1j * cim
    S = oracle.canonical(n, x, z, c, eps)
    keys, vals = _dict_merge(x, z, c, eps)
    assert [(int(a), int(b)) for a, b in zip(S.x, S.z)] == keys
    assert np.array_equal(S.c, np.array(vals, dtype=np.complex128).reshape(-1))


def test_canonical_edge_cases():
    n = 4
    e = oracle.canonical(n, np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0, complex))
    assert e.m == 0
    # exact cancellation is dropped even at eps = 0
    x = np.array([3, 3, 1], np.uint64)
    z = np.array([1, 1, 0], np.uint64)
    c = np.array([0.25, -0.25, 2.0 + 1j])
    S = oracle.canonical(n, x, z, c)
    assert S.m == 1 and int(S.x[0]) == 1 and S.c[0] == 2.0 + 1j
