"""GPU Krylov (Lanczos) propagation vs exact exp(-i t H) psi (dense eigh oracle), and
vs the free-fermion closed form of an XX chain at a size beyond dense propagation.

For m = 20 and dt = 0.05 the Krylov truncation error per step is far below
rounding (||H|| dt < 1), so the FP64 path must match the exact propagation to
1e-10 after 10 steps and the FP32-storage path to 1e-5 (relative 2-norm)."""
import numpy as np
import pytest

import oracle
from oracle import dense
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _xxz(ps, n):
    x, z, cre, cim = w.xxz_terms(n, 1)
    return ps.PauliSum.from_terms(n, x, z, cre, cim), oracle.build_sum(n, x, z, None, cre, cim)


def _run(ps, H, S, psi0, dt, nsteps, dtype, graph, m=20):
    import torch
    k = ps.Krylov(H, S, m=m, dtype=dtype)
    x = torch.from_numpy(psi0).to("cuda", dtype)
    k.step(x, dt, nsteps=nsteps, graph=graph)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128), k


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_krylov_full_space_xxz_neel(ps, graph, prec):
    import torch
    n = 12
    H, Ho = _xxz(ps, n)
    S = ps.Sector.full(n)
    psi0 = np.zeros(1 << n, complex)
    psi0[w.neel_config(n)] = 1.0
    dt, nsteps = 0.05, 10
    dtype = torch.complex128 if prec == "c128" else torch.complex64
    out, k = _run(ps, H, S, psi0, dt, nsteps, dtype, graph)
    Hd = dense.pauli_sum_matrix(n, Ho.x, Ho.z, Ho.c)
    ref = dense.propagate(Hd, psi0, dt * nsteps)
    tol = 1e-10 if prec == "c128" else 1e-5
    assert np.linalg.norm(out - ref) <= tol
    a, b = k.scalars()
    assert abs(b[0] - 1.0) < 1e-5 and np.all(np.isfinite(a))


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_krylov_sz0_blocks_match_exact_and_full_space(ps, prec):
    import torch
    n = 14
    H, Ho = _xxz(ps, n)
    blocks = [(k, 7 - k) for k in range(8)]
    S = ps.Sector(n, ps.BLOCKS, 7, blocks)
    So = oracle.Sector(n, oracle.BLOCKS, 7, blocks)
    neel = w.neel_config(n)
    psi0 = np.zeros(S.dim, complex)
    psi0[So.index(neel)[0]] = 1.0
    dtype = torch.complex128 if prec == "c128" else torch.complex64
    out, _ = _run(ps, H, S, psi0, 0.05, 8, dtype, True)
    Hs = dense.sector_matrix(n, Ho.x, Ho.z, Ho.c, So.configs())
    ref = dense.propagate(Hs, psi0, 0.4)
    tol = 1e-10 if prec == "c128" else 1e-5
    assert np.linalg.norm(out - ref) <= tol
    # the same evolution in the full 2^14 space stays in Sz = 0 and agrees
    F = ps.Sector.full(n)
    pf = np.zeros(1 << n, complex)
    pf[neel] = 1.0
    outf, _ = _run(ps, H, F, pf, 0.05, 8, dtype, True)
    assert np.linalg.norm(outf[So.configs().astype(np.int64)] - out) <= tol
    assert abs(np.linalg.norm(outf) - 1.0) <= tol


def test_krylov_molecular_random_state(ps):
    import torch
    norb = 5
    h, g = w.molecular_integrals(norb, 4)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, 2, 3)
    So = oracle.Sector.molecular(norb, 2, 3)
    psi0 = w.random_state(S.dim, 8)
    out, _ = _run(ps, H, S, psi0, 0.02, 5, torch.complex128, True, m=16)
    Hs = dense.sector_matrix(2 * norb, R.x, R.z, R.c, So.configs())
    assert np.linalg.norm(out - dense.propagate(Hs, psi0, 0.1)) <= 1e-10


def test_krylov_30_sites_full_space_agrees_with_sz0(ps):
    """The 30-site chain at full size: the Neel state lies in Sz = 0 and H keeps Sz,
    so 3 graph-replayed steps in the full 2^30 space (complex64, 21 Krylov vectors
    of 8.6 GB) and in the Sz = 0 block sector (D = 155,117,520) must give the same
    amplitudes on Sz = 0 and nothing outside it; norm and energy are conserved.
    (The exact propagator is out of reach at this size; this is the pin.)"""
    import torch
    n = w.XXZ_SITES
    x, z, cre, cim = w.xxz_terms(n, w.XXZ_SEED)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim)
    Sf = ps.Sector.full(n, 10)
    nl = 12
    Sz = ps.Sector(n, ps.BLOCKS, nl, [(k, n // 2 - k) for k in range(0, min(nl, n // 2) + 1)])
    neel = w.neel_config(n)
    dt, nsteps = 0.05, 3
    res = {}
    for name, S in (("sz0", Sz), ("full", Sf)):
        psi = torch.zeros(S.dim, dtype=torch.complex64, device="cuda")
        psi[S.rank(torch.tensor([neel], dtype=torch.int64, device="cuda"))[0].item()] = 1.0
        e0 = ps.expect(H, S, psi)[0].item()
        k = ps.Krylov(H, S, m=20, dtype=torch.complex64)
        k.step(psi, dt, nsteps=nsteps, graph=True)
        r = ps.expect(H, S, psi).cpu().numpy()
        assert abs(r[3] - 1.0) < 1e-5          # norm
        assert abs(r[0] - e0) < 1e-4 * max(1.0, abs(e0))  # energy
        res[name] = psi
        del k
        torch.cuda.empty_cache()
    # Sz = 0 amplitudes of the full-space result, in the block sector's order
    cfg = Sz.unrank(torch.arange(Sz.dim, dtype=torch.int64, device="cuda"))
    full_on_sz0 = res["full"][cfg]
    a, b = full_on_sz0, res["sz0"]
    assert (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item() < 2e-5
    # and the full-space vector carries no weight outside Sz = 0
    outside = 1.0 - torch.linalg.vector_norm(full_on_sz0).item() ** 2
    assert abs(outside) < 1e-5


def _xx_chain(n, seed):
    """Open XX chain with fields, H = sum_i J_i (X_i X_i+1 + Y_i Y_i+1) + sum_i h_i Z_i
    (letter form), and its single-particle matrix: with n_i the bit of qubit i,
    Z_i = 1 - 2 n_i and the bond term hops a particle with amplitude 2 J_i."""
    rng = np.random.default_rng(seed)
    J, h = 0.5 * rng.normal(size=n - 1), 0.5 * rng.normal(size=n)
    xs, zs, cs = [], [], []
    for i in range(n - 1):
        b = (1 << i) | (1 << (i + 1))
        xs += [b, b]; zs += [0, b]; cs += [J[i], J[i]]
    for i in range(n):
        xs.append(0); zs.append(1 << i); cs.append(h[i])
    c = np.array(cs)
    T = np.diag(-2.0 * h) + np.diag(2.0 * J, 1) + np.diag(2.0 * J, -1)
    return np.array(xs, np.uint64), np.array(zs, np.uint64), c, np.zeros_like(c), T


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_krylov_xx_chain_densities_follow_free_fermions(ps, prec):
    """24-site open XX chain with fields from the Neel state in the 12|12 Sz = 0 blocks
    (D = 2,704,156), 20 graph-replayed steps of dt = 0.05.  The model is free fermions,
    so the site densities are <n_i(t)> = sum over occupied j of |U_ij(t)|^2 with
    U = exp(-i T t): a closed form at a size that no dense propagation reaches."""
    import torch
    n, n_lo, dt, nsteps = 24, 12, 0.05, 20
    x, z, cre, cim, T = _xx_chain(n, 23)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim)
    S = ps.Sector(n, ps.BLOCKS, n_lo, [(k, n // 2 - k) for k in range(n // 2 + 1)])
    assert S.dim == 2704156
    neel = w.neel_config(n)
    dtype = torch.complex128 if prec == "c128" else torch.complex64
    psi = torch.zeros(S.dim, dtype=dtype, device="cuda")
    psi[S.rank(torch.tensor([neel], dtype=torch.int64, device="cuda"))[0].item()] = 1.0
    k = ps.Krylov(H, S, m=20, dtype=dtype)
    k.step(psi, dt, nsteps=nsteps, graph=True)
    torch.cuda.synchronize()
    prob = psi.abs().double() ** 2
    cfg = S.unrank(torch.arange(S.dim, device="cuda"))
    got = np.array([float((prob * ((cfg >> i) & 1)).sum()) for i in range(n)])
    e, V = np.linalg.eigh(T)
    U = (V * np.exp(-1j * e * dt * nsteps)) @ V.T
    occ = [j for j in range(n) if (neel >> j) & 1]
    ref = (np.abs(U[:, occ]) ** 2).sum(axis=1)
    assert abs(got.sum() - n // 2) <= (1e-9 if prec == "c128" else 1e-4)
    assert np.abs(got - ref).max() <= (1e-9 if prec == "c128" else 2e-5)
