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
