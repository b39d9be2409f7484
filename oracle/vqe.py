"""Oracle of the variational pieces: product-ansatz state, energy and gradient.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs).

The ansatz of Sec. 3.2 is a product of exponentials of single-group
generators, psi(theta) = U_{K-1} ... U_0 |ref>, U_k = exp(-i theta_k G_k),
each factor applied with the oracle's own rotation (``oracle.rotate``).

``gradient`` is the plain definition
    dE/dtheta_k = 2 Re <H psi | d_k psi>,
    d_k psi = U_{K-1} ... U_{k+1} (-i G_k) U_k ... U_0 |ref>,
with every d_k psi built from scratch (O(K^2) rotations: small K only).
Pinned in tests/test_oracle_vqe.py against central finite differences of
``energy``, against the variational bound E(theta) >= lowest eigenvalue of
the dense sector matrix, and against the 2 pi periodicity of a generator with
spectrum {-1, 0, 1}.

``pool_gradients`` is the operator-selection quantity of ADAPT-VQE (Sec. 3.3):
for each pool operator A_k (anti-Hermitian; here A_k = -i G_k for the
Hermitian generator G_k) the commutator expectation
    g_k = <psi|[H, A_k]|psi> = <psi| H A_k psi> - <psi| A_k H psi>,
with both products formed by the oracle's apply.  Pinned in
tests/test_oracle_vqe.py by central finite differences of
<psi|exp(i t G_k) H exp(-i t G_k)|psi> (oracle rotations), whose derivative at
t = 0 it is, and by a generator that commutes with H (zero gradient).
"""
from __future__ import annotations

import numpy as np

from . import apply, expect, rotate


def state(sector, gens, theta, ref_index: int) -> np.ndarray:
    psi = np.zeros(sector.dim, np.complex128)
    psi[ref_index] = 1.0
    for G, t in zip(gens, theta):
        psi = rotate(sector, G, float(t), psi)
    return psi


def energy(sector, H, gens, theta, ref_index: int) -> float:
    e, _ = expect(sector, H, state(sector, gens, theta, ref_index))
    return e.real


def gradient(sector, H, gens, theta, ref_index: int) -> np.ndarray:
    psi = state(sector, gens, theta, ref_index)
    hpsi = apply(sector, H, psi)
    K = len(gens)
    g = np.zeros(K)
    for k in range(K):
        v = np.zeros(sector.dim, np.complex128)
        v[ref_index] = 1.0
        for j in range(k + 1):
            v = rotate(sector, gens[j], float(theta[j]), v)
        v = -1j * apply(sector, gens[k], v)
        for j in range(k + 1, K):
            v = rotate(sector, gens[j], float(theta[j]), v)
        g[k] = 2.0 * np.vdot(hpsi, v).real
    return g


def pool_gradients(sector, H, gens, psi) -> np.ndarray:
    """<psi|[H, A_k]|psi> for A_k = -i G_k, every generator of the pool."""
    psi = np.asarray(psi, dtype=np.complex128)
    hpsi = apply(sector, H, psi)
    out = np.zeros(len(gens))
    for k, G in enumerate(gens):
        a_psi = -1j * apply(sector, G, psi)          # A psi
        h_a_psi = apply(sector, H, a_psi)            # H A psi
        a_h_psi = -1j * apply(sector, G, hpsi)       # A H psi
        c = np.vdot(psi, h_a_psi) - np.vdot(psi, a_h_psi)
        out[k] = c.real  # [H, A] is Hermitian for an anti-Hermitian A: c is real up to rounding
    return out
