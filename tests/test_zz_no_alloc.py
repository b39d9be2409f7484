"""pauli_expect_noalloc: the expectation value for callers that cannot have device
memory allocated for them (a framework pool that owns the whole GPU, latency-
critical loops where cudaMalloc/cudaFree would synchronise the device).

It is called here through the C ABI and must give the same result as
pauli_expect, call after call, although its partial sums live in one static
device array shared by every call.  Collected last so that a failure here stops
a run only after every other test has run."""
import ctypes as C

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _noalloc(ps, H, S, psi, result, hpsi=None):
    import torch
    rc = ps.lib().pauli_expect_noalloc(H._h, S._h, C.c_void_p(psi.data_ptr()), ps._dtype_code(psi),
                                       C.c_void_p(result.data_ptr()),
                                       None if hpsi is None else C.c_void_p(hpsi.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("wl", ["mol12", "mol24"])
def test_noalloc_matches_expect_twice(ps, dt, wl):
    import torch
    mol = w.MOL12 if wl == "mol12" else w.MOL24
    h, g = mol.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(mol.norb, mol.n_alpha, mol.n_beta)
    ps.prepare(H, S)
    tdt = torch.complex128 if dt == "c128" else torch.complex64
    psi = torch.from_numpy(w.random_state(S.dim, mol.psi_seed)).to("cuda", tdt)
    phi = torch.from_numpy(w.random_state(S.dim, mol.psi_seed + 100)).to("cuda", tdt)
    ref_psi = ps.expect(H, S, psi).cpu().numpy()
    ref_phi_h = torch.empty_like(phi)
    ref_phi = ps.expect(H, S, phi, hpsi_out=ref_phi_h).cpu().numpy()
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    hp = torch.empty_like(phi)
    # the tolerances of the other GPU tests: energies 1e-12 (FP64) / 1e-6 Ha (FP32
    # group sums), ||H psi||-relative 1e-12 / 1e-5 (pauli_expect may add its
    # partial sums in another order)
    e_tol = 1e-12 if dt == "c128" else 1e-6
    v_tol = 1e-12 if dt == "c128" else 1e-5
    # two calls in a row on different states: the second must not see the first's scratch
    for x, ref, want_h in ((psi, ref_psi, False), (phi, ref_phi, True)):
        res.fill_(float("nan"))
        rc = _noalloc(ps, H, S, x, res, hp if want_h else None)
        assert rc == 0, ps.lib().pauli_last_error()
        torch.cuda.synchronize()
        got = res.cpu().numpy()
        assert abs(complex(got[0], got[1]) - complex(ref[0], ref[1])) <= e_tol
        assert abs(got[2] - ref[2]) <= v_tol * ref[2]
        assert abs(got[3] - ref[3]) <= 1e-12
    a = hp.cpu().numpy().astype(np.complex128)
    b = ref_phi_h.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(a - b) <= v_tol * np.linalg.norm(b)


def test_noalloc_rejections(ps):
    import torch
    h, g = w.MOL12.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(6, 3, 3)
    psi = torch.zeros(S.dim, dtype=torch.complex128, device="cuda")
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    # no plan for this split yet: the call would have to allocate one
    assert _noalloc(ps, H, S, psi, res) == ps.EINVAL
    assert "pauli_prepare" in ps.lib().pauli_last_error().decode()
    # a launch larger than the static scratch is refused before anything runs
    x, z, cre, cim = w.xxz_terms(30, 1)
    Hx = ps.PauliSum.from_terms(30, x, z, cre, cim)
    Sx = ps.Sector.full(30)
    ps.prepare(Hx, Sx)
    small = torch.zeros(16, dtype=torch.complex64, device="cuda")
    rc = ps.lib().pauli_expect_noalloc(Hx._h, Sx._h, C.c_void_p(small.data_ptr()), ps.C64,
                                       C.c_void_p(res.data_ptr()), None,
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == ps.EUNSUPPORTED
    assert "static scratch" in ps.lib().pauli_last_error().decode()


def test_noalloc_full_space_passes(ps):
    """A 22-site chain in the full space runs in passes over local bit sets,
    which accumulate H psi in a vector.  Without hpsi_out the call is refused
    (the passes would need a vector the library would have to allocate) until
    an ordinary pauli_expect has made the operator's own one; with hpsi_out, or
    after that, it matches pauli_expect, and free device memory does not move
    across the no-allocation calls."""
    import torch
    n = 22
    x, z, cre, cim = w.xxz_terms(n, 1)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim)
    S = ps.Sector.full(n)
    ps.prepare(H, S)
    assert ps.launch_config(H, S)["direct"] == 2
    psi = torch.from_numpy(w.random_state(S.dim, 22)).to("cuda", torch.complex64)
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    hp = torch.empty_like(psi)
    assert _noalloc(ps, H, S, psi, res) == ps.EUNSUPPORTED
    assert "hpsi_out" in ps.lib().pauli_last_error().decode()
    # the first successful call on a device looks up the static array (which may
    # load the library's module onto the device); memory is compared after it
    rc = _noalloc(ps, H, S, psi, res, hp)
    assert rc == 0, ps.lib().pauli_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc = _noalloc(ps, H, S, psi, res, hp)
        assert rc == 0, ps.lib().pauli_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = res.cpu().numpy()
    ref_h = torch.empty_like(psi)
    ref = ps.expect(H, S, psi, hpsi_out=ref_h).cpu().numpy()
    assert abs(complex(got[0], got[1]) - complex(ref[0], ref[1])) <= 1e-6 * max(1.0, abs(ref[0]))
    assert abs(got[2] - ref[2]) <= 1e-5 * ref[2]
    a = hp.cpu().numpy().astype(np.complex128)
    b = ref_h.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    # an ordinary expectation without an output vector makes the operator's scratch;
    # from then on the no-allocation call works without hpsi_out too
    ref2 = ps.expect(H, S, psi).cpu().numpy()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        res.fill_(float("nan"))
        rc = _noalloc(ps, H, S, psi, res)
        assert rc == 0, ps.lib().pauli_last_error()
        torch.cuda.synchronize()
        got = res.cpu().numpy()
        assert abs(complex(got[0], got[1]) - complex(ref2[0], ref2[1])) <= 1e-6 * max(1.0, abs(ref2[0]))
    assert torch.cuda.mem_get_info()[0] == free1
