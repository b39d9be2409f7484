"""Shared fixtures.  GPU tests are marked ``gpu``; everything else runs on CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def mol12():
    """12-qubit molecule (6 orbitals, seed 0) as an oracle Pauli sum + integrals."""
    import oracle
    import workloads as w
    h, g = w.MOL12.integrals()
    H = oracle.jw_hamiltonian(6, h, g, eps_drop=1e-12)
    return h, g, H


@pytest.fixture(scope="session")
def mol12_dense(mol12):
    from oracle import dense
    _, _, H = mol12
    return dense.pauli_sum_matrix(12, H.x, H.z, H.c, sparse=True)
