"""Pins of the exact propagation oracle exp(-i t H) psi (dense eigh) used by the Krylov tests."""
import numpy as np
import scipy.linalg as sla

import oracle
from oracle import dense
import workloads as w


def _xxz(n):
    x, z, cre, cim = w.xxz_terms(n, 1)
    return oracle.build_sum(n, x, z, None, cre, cim)


def test_propagate_matches_pade_expm():
    """eigh-based exp(-itH) agrees with scipy's Pade expm (a different algorithm)."""
    n = 6
    H = _xxz(n)
    Hd = dense.pauli_sum_matrix(n, H.x, H.z, H.c)
    psi = w.random_state(1 << n, 3)
    for t in (0.05, 0.7):
        assert np.allclose(dense.propagate(Hd, psi, t), sla.expm(-1j * t * Hd) @ psi, atol=1e-12)


def test_propagation_conserves_norm_energy_and_sz():
    n = 10
    H = _xxz(n)
    Hd = dense.pauli_sum_matrix(n, H.x, H.z, H.c)
    neel = w.neel_config(n)
    psi = np.zeros(1 << n, complex)
    psi[neel] = 1.0
    E0 = np.vdot(psi, Hd @ psi).real
    out = dense.propagate(Hd, psi, 1.0)
    assert abs(np.linalg.norm(out) - 1.0) < 1e-12
    assert abs(np.vdot(out, Hd @ out).real - E0) < 1e-11
    # H conserves Sz: the Neel state never leaves the Sz = 0 configurations
    pop = np.array([bin(b).count("1") for b in range(1 << n)])
    assert np.abs(out[pop != n // 2]).max() < 1e-13
    # and the Sz = 0 block of H propagates it identically
    s = oracle.Sector(n, oracle.BLOCKS, n // 2, [(k, n // 2 - k) for k in range(n // 2 + 1)])
    cfg = s.configs().astype(np.int64)
    Hs = dense.sector_matrix(n, H.x, H.z, H.c, cfg)
    ps0 = np.zeros(s.dim, complex)
    ps0[s.index(neel)[0]] = 1.0
    assert np.allclose(dense.propagate(Hs, ps0, 1.0), out[cfg], atol=1e-12)
