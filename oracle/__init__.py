"""Python face of the CPU oracle (``oracle.c``) plus dense numpy checkers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` import this package.  It
shares no code with ``paper_2606_28952_gb300`` (the CUDA path) and imports
nothing from it.

Parity status of each oracle function (what pins it, see tests/test_oracle_*.py):
  letter_mul, string_mul   2x2 / Kronecker matrix products (numpy)
  to_xz                    dense matrices of letter strings vs X^x Z^z
  jw_raw / jw_hamiltonian  anticommutators {a_p, a_q^dagger} = delta_pq,
                           Hermiticity, number conservation, dense matrix of
                           the fermionic Hamiltonian built from Kronecker
                           products, Hartree-Fock closed form
  canonical                brute-force dictionary merge on small inputs
  sector_*                 eq. fcidim and the Det column of Table 2
  apply / apply_rows       dense Kronecker-built H on <= 12 qubits
  expect                   Hartree-Fock closed form, dense H
  rotate                   scipy.linalg.expm on <= 10 qubits, closed forms
  hf_energy                determinant energy from the dense H
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, FP64, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


_lib_lock = threading.Lock()


def lib():
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(build())
        L.orc_letter_mul.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.orc_letter_mul.restype = C.c_int
        L.orc_string_mul.argtypes = [C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_int)]
        L.orc_to_xz.argtypes = [C.c_int, C.c_int64, _u64p, _u64p, C.c_void_p, _f64p, _f64p, C.c_int,
                                _f64p, _f64p]
        L.orc_jw_raw.argtypes = [C.c_int, _f64p, _f64p, C.c_double, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
        L.orc_jw_raw.restype = C.c_int64
        L.orc_canonical.argtypes = [C.c_int64, _u64p, _u64p, _f64p, _f64p, C.c_double, _u64p, _u64p,
                                    _f64p, _f64p]
        L.orc_canonical.restype = C.c_int64
        L.orc_sector_new.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _i32p, _i32p]
        L.orc_sector_new.restype = C.c_void_p
        L.orc_sector_new_irrep.argtypes = [C.c_int, C.c_int, C.c_int, _i32p, _i32p, _i32p, _i32p, _i32p]
        L.orc_sector_new_irrep.restype = C.c_void_p
        L.orc_sector_free.argtypes = [C.c_void_p]
        L.orc_sector_dim.argtypes = [C.c_void_p]
        L.orc_sector_dim.restype = C.c_int64
        L.orc_sector_configs.argtypes = [C.c_void_p, _u64p]
        L.orc_sector_rank_many.argtypes = [C.c_void_p, C.c_int64, _u64p, _i64p]
        L.orc_apply.argtypes = [C.c_void_p, C.c_int64, _u64p, _u64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_apply_rows.argtypes = [C.c_void_p, C.c_int64, _u64p, _u64p, _f64p, _f64p, _f64p,
                                     C.c_int64, _i64p, _f64p]
        L.orc_expect.argtypes = [C.c_void_p, C.c_int64, _u64p, _u64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_leaks.argtypes = [C.c_void_p, C.c_int64, _u64p, _u64p, _f64p, _f64p]
        L.orc_leaks.restype = C.c_int
        L.orc_rotate.argtypes = [C.c_void_p, C.c_int64, _u64p, _u64p, _f64p, _f64p, C.c_double,
                                 _f64p]
        L.orc_jw_ladder.argtypes = [C.c_int, C.c_int, _u64p, _u64p, _f64p, _f64p]
        L.orc_sum_product.argtypes = [C.c_int, C.c_int64, _u64p, _u64p, _f64p, _f64p, C.c_int64, _u64p,
                                      _u64p, _f64p, _f64p, _u64p, _u64p, _f64p, _f64p]
        L.orc_count_strings.argtypes = [C.c_int, C.c_int]
        L.orc_count_strings.restype = C.c_int64
        L.orc_fermion_raw.argtypes = [C.c_int, C.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_fermion_raw.restype = C.c_int64
        L.orc_hf_energy.argtypes = [C.c_int, _f64p, _f64p, C.c_int, C.c_int, C.c_double]
        L.orc_hf_energy.restype = C.c_double
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# letters and strings
# ---------------------------------------------------------------------------
I, X, Y, Z = 0, 1, 2, 3


def letter_mul(u: int, v: int) -> tuple[int, int]:
    """sigma_u sigma_v = i^k sigma_w; returns (w, k)."""
    k = C.c_int()
    w = lib().orc_letter_mul(u, v, C.byref(k))
    return w, k.value


def string_mul(n: int, xa: int, za: int, xb: int, zb: int) -> tuple[int, int, int]:
    """Product of two letter strings; returns (x, z, k) with phase i^k."""
    x, z, k = C.c_uint64(), C.c_uint64(), C.c_int()
    lib().orc_string_mul(n, xa, za, xb, zb, C.byref(x), C.byref(z), C.byref(k))
    return x.value, z.value, k.value


@dataclass
class PauliSum:
    """Sum_j C_j X^{x_j} Z^{z_j} (symplectic form) on n qubits."""
    n: int
    x: np.ndarray  # uint64
    z: np.ndarray  # uint64
    c: np.ndarray  # complex128, XZ-form coefficients

    @property
    def m(self) -> int:
        return len(self.x)

    def arrays(self):
        return (np.ascontiguousarray(self.x, dtype=np.uint64), np.ascontiguousarray(self.z, dtype=np.uint64),
                np.ascontiguousarray(self.c.real, dtype=np.float64),
                np.ascontiguousarray(self.c.imag, dtype=np.float64))


def to_xz(n, x, z, gamma, cre, cim, letter_form: bool) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    m = len(x)
    ore = np.zeros(m)
    oim = np.zeros(m)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.uint8)
    lib().orc_to_xz(n, m, x, z, None if g is None else g.ctypes.data, np.ascontiguousarray(cre, dtype=np.float64),
                    np.ascontiguousarray(cim, dtype=np.float64), int(letter_form), ore, oim)
    return ore + 1j * oim


def canonical(n, x, z, c, eps: float = 0.0) -> PauliSum:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.asarray(c, dtype=np.complex128)
    m = len(x)
    ox = np.zeros(max(m, 1), np.uint64)
    oz = np.zeros(max(m, 1), np.uint64)
    ore = np.zeros(max(m, 1))
    oim = np.zeros(max(m, 1))
    k = lib().orc_canonical(m, x, z, np.ascontiguousarray(c.real), np.ascontiguousarray(c.imag), eps,
                            ox, oz, ore, oim)
    return PauliSum(n, ox[:k].copy(), oz[:k].copy(), ore[:k] + 1j * oim[:k])


def build_sum(n, x, z, gamma, cre, cim, eps=0.0, letter_form=True) -> PauliSum:
    """Input arrays -> canonical Pauli sum (XZ form), the contract of pauli_sum_build."""
    c = to_xz(n, x, z, gamma, cre, cim, letter_form)
    return canonical(n, x, z, c, eps)


def jw_raw(norb: int, h: np.ndarray, g: np.ndarray, eps: float = 0.0):
    L = lib()
    h = np.ascontiguousarray(h, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    m = L.orc_jw_raw(norb, h, g, eps, None, None, None, None)
    x = np.zeros(m, np.uint64)
    z = np.zeros(m, np.uint64)
    re = np.zeros(m)
    im = np.zeros(m)
    L.orc_jw_raw(norb, h, g, eps, x.ctypes.data, z.ctypes.data, re.ctypes.data, im.ctypes.data)
    return x, z, re + 1j * im


def jw_hamiltonian(norb: int, h, g, eps_int: float = 0.0, e_nn: float = 0.0, eps_drop: float = 0.0) -> PauliSum:
    """Qubit Hamiltonian of Algorithm 1; a nonzero e_nn is the first raw entry (identity)."""
    x, z, c = jw_raw(norb, h, g, eps_int)
    if e_nn != 0.0:
        x = np.concatenate([np.zeros(1, np.uint64), x])
        z = np.concatenate([np.zeros(1, np.uint64), z])
        c = np.concatenate([np.array([e_nn + 0j]), c])
    return canonical(2 * norb, x, z, c, eps_drop)


def ladder(n: int, P: int, dagger: bool) -> PauliSum:
    """a_P (or a_P^dagger) as a two-term Pauli sum in XZ form (Jordan-Wigner)."""
    x = np.zeros(2, np.uint64)
    z = np.zeros(2, np.uint64)
    re = np.zeros(2)
    im = np.zeros(2)
    lib().orc_jw_ladder(P, int(dagger), x, z, re, im)
    return PauliSum(n, x, z, re + 1j * im)


def fermion_sum(n: int, terms, eps: float = 0.0) -> PauliSum:
    """Canonical Pauli sum of sum_t c_t prod_j f_{t,j}; terms = [(c, [(mode, dagger), ...]), ...]."""
    nf = np.array([len(f) for _, f in terms], np.int32)
    modes = np.array([m for _, f in terms for m, _ in f] or [0], np.int32)
    dag = np.array([int(d) for _, f in terms for _, d in f] or [0], np.int32)
    cre = np.array([complex(c).real for c, _ in terms], np.float64)
    cim = np.array([complex(c).imag for c, _ in terms], np.float64)
    L = lib()
    m = L.orc_fermion_raw(n, len(terms), nf, modes, dag, cre, cim, None, None, None, None)
    x = np.zeros(max(m, 1), np.uint64)
    z = np.zeros(max(m, 1), np.uint64)
    re = np.zeros(max(m, 1))
    im = np.zeros(max(m, 1))
    L.orc_fermion_raw(n, len(terms), nf, modes, dag, cre, cim, x.ctypes.data, z.ctypes.data, re.ctypes.data,
                      im.ctypes.data)
    return canonical(n, x[:m], z[:m], re[:m] + 1j * im[:m], eps)


def sum_product(A: PauliSum, B: PauliSum, eps: float = 0.0) -> PauliSum:
    """Canonical form of the operator product A B."""
    xa, za, ra, ia = A.arrays()
    xb, zb, rb, ib = B.arrays()
    m = A.m * B.m
    ox = np.zeros(max(m, 1), np.uint64)
    oz = np.zeros(max(m, 1), np.uint64)
    ore = np.zeros(max(m, 1))
    oim = np.zeros(max(m, 1))
    lib().orc_sum_product(A.n, A.m, xa, za, ra, ia, B.m, xb, zb, rb, ib, ox, oz, ore, oim)
    return canonical(A.n, ox[:m], oz[:m], ore[:m] + 1j * oim[:m], eps)


def sum_add(A: PauliSum, B: PauliSum, b_scale: complex = 1.0, eps: float = 0.0) -> PauliSum:
    """Canonical form of A + b_scale * B (A's entries first in raw order)."""
    return canonical(A.n, np.concatenate([A.x, B.x]), np.concatenate([A.z, B.z]),
                     np.concatenate([A.c, b_scale * B.c]), eps)


# ---------------------------------------------------------------------------
# sectors
# ---------------------------------------------------------------------------
FULL, BLOCKS = 0, 1


class Sector:
    """Full space (kind=FULL) or a union of product blocks (k_lo, k_hi)."""

    def __init__(self, n: int, kind: int = FULL, n_lo: int = 0, blocks=()):
        self.n, self.kind, self.n_lo = n, kind, n_lo
        self.blocks = [tuple(b) for b in blocks]
        klo = np.array([b[0] for b in self.blocks] or [0], dtype=np.int32)
        khi = np.array([b[1] for b in self.blocks] or [0], dtype=np.int32)
        self._h = lib().orc_sector_new(n, kind, n_lo, len(self.blocks), klo, khi)

    @classmethod
    def irrep_blocks(cls, n: int, n_lo: int, blocks, qubit_irrep):
        """Point-group blocks (k_lo, irrep_lo, k_hi, irrep_hi); qubit_irrep[q] in 0..7."""
        self = cls.__new__(cls)
        self.n, self.kind, self.n_lo = n, BLOCKS, n_lo
        self.blocks = [tuple(b) for b in blocks]
        arr = lambda i: np.array([b[i] for b in self.blocks] or [0], dtype=np.int32)
        qi = np.ascontiguousarray(np.asarray(qubit_irrep, dtype=np.int32))
        self._h = lib().orc_sector_new_irrep(n, n_lo, len(self.blocks), arr(0), arr(2), arr(1), arr(3), qi)
        return self

    @classmethod
    def full(cls, n):
        return cls(n, FULL)

    @classmethod
    def molecular(cls, norb, na, nb):
        return cls(2 * norb, BLOCKS, norb, [(na, nb)])

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_sector_free(self._h)
            self._h = None

    @property
    def dim(self) -> int:
        return lib().orc_sector_dim(self._h)

    def configs(self) -> np.ndarray:
        out = np.zeros(max(self.dim, 1), np.uint64)
        lib().orc_sector_configs(self._h, out)
        return out[: self.dim]

    def index(self, b) -> np.ndarray:
        b = np.ascontiguousarray(np.atleast_1d(b), dtype=np.uint64)
        out = np.zeros(len(b), np.int64)
        lib().orc_sector_rank_many(self._h, len(b), b, out)
        return out


def count_strings(bits: int, k: int) -> int:
    """Number of bits-bit strings with k ones (Pascal's rule)."""
    return lib().orc_count_strings(bits, k)


def _interleave(psi):
    return np.ascontiguousarray(np.asarray(psi, dtype=np.complex128).view(np.float64))


def apply(sector: Sector, H: PauliSum, psi: np.ndarray) -> np.ndarray:
    x, z, cre, cim = H.arrays()
    out = np.zeros(2 * sector.dim)
    lib().orc_apply(sector._h, H.m, x, z, cre, cim, _interleave(psi), out)
    return out.view(np.complex128)


def apply_rows(sector: Sector, H: PauliSum, psi: np.ndarray, rows) -> np.ndarray:
    x, z, cre, cim = H.arrays()
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(2 * len(rows))
    lib().orc_apply_rows(sector._h, H.m, x, z, cre, cim, _interleave(psi), len(rows), rows, out)
    return out.view(np.complex128)


def expect(sector: Sector, H: PauliSum, psi: np.ndarray) -> tuple[complex, float]:
    x, z, cre, cim = H.arrays()
    res = np.zeros(3)
    lib().orc_expect(sector._h, H.m, x, z, cre, cim, _interleave(psi), res)
    return complex(res[0], res[1]), float(res[2])


def leaks(sector: Sector, G: PauliSum) -> bool:
    x, z, cre, cim = G.arrays()
    return bool(lib().orc_leaks(sector._h, G.m, x, z, cre, cim))


def rotate(sector: Sector, G: PauliSum, theta: float, psi: np.ndarray) -> np.ndarray:
    x, z, cre, cim = G.arrays()
    v = _interleave(psi).copy()
    lib().orc_rotate(sector._h, G.m, x, z, cre, cim, float(theta), v)
    return v.view(np.complex128)


def hf_energy(norb, h, g, na, nb, e_nn=0.0) -> float:
    return lib().orc_hf_energy(norb, np.ascontiguousarray(h, dtype=np.float64),
                               np.ascontiguousarray(g, dtype=np.float64), na, nb, e_nn)


def hf_config(norb: int, na: int, nb: int) -> int:
    """Determinant with the lowest na alpha and nb beta orbitals occupied (blocked order)."""
    return ((1 << na) - 1) | (((1 << nb) - 1) << norb)
