"""Dense / sparse matrix checkers built from first principles (numpy, scipy).

TEST INFRASTRUCTURE ONLY.  These build operators from 2x2 Pauli matrices and
Kronecker products (the definition of a Pauli string, eq. pauli_group, with
qubit 0 the rightmost Kronecker factor, i.e. the least significant bit of the
basis index) and fermionic ladder operators from their action on occupation
number states.  They pin the oracle; they use none of its arithmetic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA = {
    0: np.array([[1, 0], [0, 1]], dtype=np.complex128),
    1: np.array([[0, 1], [1, 0]], dtype=np.complex128),
    2: np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    3: np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def letter(a: int, b: int) -> int:
    """Letter of the bit pair (a, b): I=(0,0), X=(1,0), Y=(1,1), Z=(0,1)."""
    return {(0, 0): 0, (1, 0): 1, (1, 1): 2, (0, 1): 3}[(a, b)]


def _kron_all(factors):
    """factors[q] acts on qubit q; returns kron(f[n-1], ..., f[0]) as CSR."""
    m = sp.csr_matrix(np.ones((1, 1), dtype=np.complex128))
    for f in reversed(factors):
        m = sp.kron(m, sp.csr_matrix(f), format="csr")
    return m


def letter_string(n: int, x: int, z: int):
    """Sparse matrix of the letter string with masks (x, z)."""
    return _kron_all([SIGMA[letter((x >> q) & 1, (z >> q) & 1)] for q in range(n)])


def xz_string(n: int, x: int, z: int):
    """Sparse matrix of X^x Z^z = kron_q (X^{x_q} Z^{z_q})."""
    fs = []
    for q in range(n):
        m = np.eye(2, dtype=np.complex128)
        if (x >> q) & 1:
            m = m @ SIGMA[1]
        if (z >> q) & 1:
            m = m @ SIGMA[3]
        fs.append(m)
    return _kron_all(fs)


def pauli_sum_matrix(n: int, x, z, c, sparse: bool = False):
    """sum_k c_k X^{x_k} Z^{z_k}."""
    rows, cols, vals = [], [], []
    for xk, zk, ck in zip(np.asarray(x, dtype=np.uint64), np.asarray(z, dtype=np.uint64), np.asarray(c)):
        m = xz_string(n, int(xk), int(zk)).tocoo()
        rows.append(m.row)
        cols.append(m.col)
        vals.append(complex(ck) * m.data)
    dim = 1 << n
    if rows:
        H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim))
    else:
        H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    return H if sparse else H.toarray()


def sector_matrix(n: int, x, z, c, configs) -> np.ndarray:
    """Dense H restricted to the rows and columns of the given configurations."""
    idx = np.asarray(configs, dtype=np.int64)
    return pauli_sum_matrix(n, x, z, c, sparse=True)[idx][:, idx].toarray()


def propagate(Hs: np.ndarray, psi: np.ndarray, t: float) -> np.ndarray:
    """exp(-i t H) psi for a Hermitian dense matrix by its eigen-decomposition (numpy eigh)."""
    lam, V = np.linalg.eigh(Hs)
    return V @ (np.exp(-1j * t * lam) * (V.conj().T @ psi))


def annihilator(n_modes: int, P: int):
    """a_P on occupation-number states |b>, bit Q of b = occupation of mode Q:
    a_P |b> = (-1)^(sum_{Q<P} b_Q) |b - e_P> if b_P = 1, else 0  (sparse CSR)."""
    dim = 1 << n_modes
    rows, cols, vals = [], [], []
    for b in range(dim):
        if (b >> P) & 1:
            sign = -1.0 if bin(b & ((1 << P) - 1)).count("1") % 2 else 1.0
            rows.append(b ^ (1 << P))
            cols.append(b)
            vals.append(sign)
    return sp.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(dim, dim))


def fermionic_hamiltonian(norb: int, h, g, e_nn: float = 0.0, sparse: bool = False):
    """H = sum_{sigma,pq} h_pq a+_{p s} a_{q s}
         + 1/2 sum_{sigma,tau,pqrs} (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s} + e_nn,
    spin orbital P = p (alpha) or norb + p (beta), built from ladder matrices."""
    n = 2 * norb
    a = [annihilator(n, P) for P in range(n)]
    ad = [m.conj().T.tocsr() for m in a]
    dim = 1 << n
    H = e_nn * sp.identity(dim, dtype=np.complex128, format="csr")
    for s in range(2):
        for p in range(norb):
            for q in range(norb):
                H = H + h[p, q] * (ad[s * norb + p] @ a[s * norb + q])
    for s in range(2):
        for t in range(2):
            for p in range(norb):
                for q in range(norb):
                    for r in range(norb):
                        for u in range(norb):
                            v = g[p, q, r, u]
                            if v == 0.0:
                                continue
                            P, Q, R, U = s * norb + p, s * norb + q, t * norb + r, t * norb + u
                            H = H + 0.5 * v * (ad[P] @ ad[R] @ a[U] @ a[Q])
    return H.tocsr() if sparse else H.toarray()
