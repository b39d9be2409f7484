"""paulisim -- GB300 (sm_103a) Pauli-algebra operator-state library, Python binding.

This module only marshals arguments: every step (Jordan-Wigner expansion,
canonical reduction, grouping, sector ranking, apply / expect / rotate) runs
in the CUDA kernels of ``libpaulisim.so`` behind the C ABI of
``include/paulisim.h``.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpaulisim.so")

C64, C128 = 0, 1
LETTER, XZ = 0, 1
FULL, BLOCKS = 0, 1

OK, EINVAL, ENOMEM, ECUDA, ESECTOR, ENOTHERMITIAN, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "PAULI_OK", -1: "PAULI_EINVAL", -2: "PAULI_ENOMEM", -3: "PAULI_ECUDA", -4: "PAULI_ESECTOR",
                -5: "PAULI_ENOTHERMITIAN", -6: "PAULI_ETIMEOUT", -7: "PAULI_EUNSUPPORTED"}


class PauliError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_vp, _i64, _i32, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double

# name -> (restype, argtypes); mirrors include/paulisim.h
SIGNATURES = {
    "pauli_last_error": (C.c_char_p, []),
    "pauli_version": (_i32, []),
    "pauli_set_allocator": (_i32, [_vp, _vp, _vp]),
    "pauli_sum_build": (_i32, [_i32, _i64, _vp, _vp, _vp, _vp, _vp, _i32, _dbl, _vp]),
    "pauli_jw_molecular": (_i32, [_i32, _vp, _vp, _dbl, _dbl, _dbl, _vp]),
    "pauli_jw_molecular_raw": (_i32, [_i32, _vp, _vp, _dbl, _dbl, _vp, _vp, _vp, _vp, _vp]),
    "pauli_jw_fermion": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _dbl, _vp]),
    "pauli_sum_product": (_i32, [_vp, _vp, _dbl, _vp]),
    "pauli_sum_add": (_i32, [_vp, _vp, _dbl, _dbl, _dbl, _vp]),
    "pauli_sum_info": (_i32, [_vp, _vp, _vp, _vp]),
    "pauli_wsum_jw_fermion": (_i32, [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _dbl, _vp]),
    "pauli_wsum_jw_molecular": (_i32, [_i32, _vp, _vp, _dbl, _dbl, _dbl, _vp]),
    "pauli_wsum_product": (_i32, [_vp, _vp, _dbl, _vp]),
    "pauli_wsum_info": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "pauli_wsum_export": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "pauli_wsum_groups": (_i32, [_vp, _vp]),
    "pauli_wsum_destroy": (_i32, [_vp]),
    "pauli_sum_export": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "pauli_sum_groups": (_i32, [_vp, _vp, _vp]),
    "pauli_sum_destroy": (_i32, [_vp]),
    "pauli_sector_create": (_i32, [_i32, _i32, _i32, _i32, _vp, _vp, _vp]),
    "pauli_sector_create_irrep": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pauli_sector_dim": (_i32, [_vp, _vp]),
    "pauli_sector_rank": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "pauli_sector_unrank": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "pauli_sector_destroy": (_i32, [_vp]),
    "pauli_prepare": (_i32, [_vp, _vp]),
    "pauli_apply": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "pauli_expect": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "pauli_expect_noalloc": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "pauli_expect_rows": (_i32, [_vp, _vp, _vp, _i32, _vp, _i64, _vp, _vp, _vp]),
    "pauli_rotate": (_i32, [_vp, _vp, _dbl, _vp, _i32, _vp]),
    "pauli_rotate_seq": (_i32, [_vp, _vp, _i32, _vp, _vp, _i32, _vp]),
    "pauli_rotate_adjoint": (_i32, [_vp, _vp, _dbl, _vp, _vp, _i32, _vp, _vp]),
    "pauli_vdot": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    "pauli_mlp_create": (_i32, [_i32, _i32, _i32, _i32, _vp]),
    "pauli_mlp_num_params": (_i32, [_vp, _vp]),
    "pauli_mlp_set_params": (_i32, [_vp, _vp]),
    "pauli_mlp_get_params": (_i32, [_vp, _vp]),
    "pauli_mlp_forward": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "pauli_mlp_backward": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "pauli_mlp_adam_step": (_i32, [_vp, C.c_float, _i32, _vp]),
    "pauli_mlp_train": (_i32, [_vp, _i32, _vp, _vp, _i32, C.c_float, _i32, _vp, _vp]),
    "pauli_mlp_destroy": (_i32, [_vp]),
    "pauli_status": (_i32, [_vp, _vp, _vp]),
    "pauli_tune": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp]),
    "pauli_set_launch_config": (_i32, [_vp, _vp, _i32, _vp]),
    "pauli_get_launch_config": (_i32, [_vp, _vp, _i32, _vp]),
    "pauli_tune_save": (_i32, [_vp, _vp, C.c_char_p]),
    "pauli_svd_ranks": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "pauli_tune_load": (_i32, [_vp, _vp, C.c_char_p, _vp]),
    "pauli_batch_create": (_i32, [_i32, _vp, _vp, _i32, _vp]),
    "pauli_batch_apply": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "pauli_batch_tune": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "pauli_batch_set_launch_config": (_i32, [_vp, _vp]),
    "pauli_batch_get_launch_config": (_i32, [_vp, _vp]),
    "pauli_batch_destroy": (_i32, [_vp]),
    "pauli_rotseq_create": (_i32, [_vp, _i32, _vp, _vp]),
    "pauli_rotseq_apply": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "pauli_rotseq_info": (_i32, [_vp, _i32, _vp, _vp]),
    "pauli_rotseq_destroy": (_i32, [_vp]),
    "pauli_pool_create": (_i32, [_vp, _i32, _vp, _vp]),
    "pauli_pool_size": (_i32, [_vp, _vp]),
    "pauli_pool_gradients": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "pauli_pool_destroy": (_i32, [_vp]),
    "pauli_krylov_create": (_i32, [_vp, _vp, _i32, _i32, _vp]),
    "pauli_krylov_step": (_i32, [_vp, _vp, _dbl, _i32, _i32, _vp]),
    "pauli_krylov_scalars": (_i32, [_vp, _vp, _vp, _vp]),
    "pauli_krylov_destroy": (_i32, [_vp]),
}


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise PauliError(rc, lib().pauli_last_error().decode())


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"state vectors must be complex64 or complex128, got {t.dtype}")


def _check_state(t, dim: int, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != dim:
        raise ValueError(f"{name} has {t.numel()} elements, the sector has {dim}")


# ---------------------------------------------------------------------------
# Pauli sums
# ---------------------------------------------------------------------------
class PauliSum:
    """Canonical Pauli sum on the device (opaque handle of the C library)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    # -- construction -------------------------------------------------------
    @classmethod
    def from_terms(cls, n: int, x, z, c_re, c_im=None, gamma=None, form: int = LETTER, eps_drop: float = 0.0):
        x = np.ascontiguousarray(x, dtype=np.uint64)
        z = np.ascontiguousarray(z, dtype=np.uint64)
        c_re = np.ascontiguousarray(c_re, dtype=np.float64)
        c_im = np.zeros_like(c_re) if c_im is None else np.ascontiguousarray(c_im, dtype=np.float64)
        g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.uint8)
        out = C.c_void_p()
        _check(lib().pauli_sum_build(n, len(x), _np_ptr(x), _np_ptr(z), None if g is None else _np_ptr(g),
                                     _np_ptr(c_re), _np_ptr(c_im), form, eps_drop, C.byref(out)))
        return cls(out.value)

    @classmethod
    def jw_molecular(cls, h, g, e_nn: float = 0.0, eps_int: float = 0.0, eps_drop: float = 0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        norb = h.shape[0]
        out = C.c_void_p()
        _check(lib().pauli_jw_molecular(norb, _np_ptr(h), _np_ptr(g), e_nn, eps_int, eps_drop, C.byref(out)))
        return cls(out.value)

    @classmethod
    def jw_fermion(cls, n: int, terms, eps_drop: float = 0.0):
        """terms = [(coefficient, [(mode, dagger), ...]), ...] (left-to-right products)."""
        nf = np.array([len(f) for _, f in terms], np.int32)
        modes = np.array([m for _, f in terms for m, _ in f] or [0], np.int32)
        dag = np.array([int(d) for _, f in terms for _, d in f] or [0], np.int32)
        cre = np.array([complex(c).real for c, _ in terms] or [0.0], np.float64)
        cim = np.array([complex(c).imag for c, _ in terms] or [0.0], np.float64)
        out = C.c_void_p()
        _check(lib().pauli_jw_fermion(n, len(terms), _np_ptr(nf), _np_ptr(modes), _np_ptr(dag), _np_ptr(cre),
                                      _np_ptr(cim), eps_drop, C.byref(out)))
        return cls(out.value)

    # -- algebra --------------------------------------------------------------
    def __matmul__(self, other: "PauliSum") -> "PauliSum":
        """Canonical operator product self @ other (pauli_sum_product)."""
        return self.product(other)

    def product(self, other: "PauliSum", eps_drop: float = 0.0) -> "PauliSum":
        out = C.c_void_p()
        _check(lib().pauli_sum_product(self._h, other._h, eps_drop, C.byref(out)))
        return PauliSum(out.value)

    def add(self, other: "PauliSum", beta: complex = 1.0, eps_drop: float = 0.0) -> "PauliSum":
        """Canonical self + beta * other (pauli_sum_add)."""
        out = C.c_void_p()
        b = complex(beta)
        _check(lib().pauli_sum_add(self._h, other._h, b.real, b.imag, eps_drop, C.byref(out)))
        return PauliSum(out.value)

    def commutator(self, other: "PauliSum", eps_drop: float = 0.0) -> "PauliSum":
        """[self, other] = self other - other self, canonical."""
        return self.product(other).add(other.product(self), -1.0, eps_drop)

    # -- properties ---------------------------------------------------------
    def info(self):
        n, m, g = C.c_int(), C.c_int64(), C.c_int64()
        _check(lib().pauli_sum_info(self._h, C.byref(n), C.byref(m), C.byref(g)))
        return n.value, m.value, g.value

    @property
    def n(self) -> int:
        return self.info()[0]

    @property
    def m(self) -> int:
        return self.info()[1]

    @property
    def n_groups(self) -> int:
        return self.info()[2]

    def export(self):
        """Canonical (x, z, C) with XZ-form coefficients, as numpy arrays."""
        _, m, _ = self.info()
        x = np.zeros(max(m, 1), np.uint64)
        z = np.zeros(max(m, 1), np.uint64)
        re = np.zeros(max(m, 1))
        im = np.zeros(max(m, 1))
        _check(lib().pauli_sum_export(self._h, _np_ptr(x), _np_ptr(z), _np_ptr(re), _np_ptr(im)))
        return x[:m], z[:m], re[:m] + 1j * im[:m]

    def groups(self):
        _, _, g = self.info()
        gx = np.zeros(max(g, 1), np.uint64)
        gs = np.zeros(g + 1, np.int64)
        _check(lib().pauli_sum_groups(self._h, _np_ptr(gx), _np_ptr(gs)))
        return gx[:g], gs

    def status(self, stream=None) -> int:
        code = C.c_int()
        _check(lib().pauli_status(self._h, _stream_ptr(stream), C.byref(code)))
        return code.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_sum_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WidePauliSum:
    """Canonical Pauli sum with multi-word masks (up to 256 qubits): the
    operator algebra of large Jordan-Wigner builds (pauli_wsum_*).  export()
    gives the masks as Python integers."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @classmethod
    def jw_fermion(cls, n: int, terms, eps_drop: float = 0.0):
        nf = np.array([len(f) for _, f in terms], np.int32)
        modes = np.array([m for _, f in terms for m, _ in f] or [0], np.int32)
        dag = np.array([int(d) for _, f in terms for _, d in f] or [0], np.int32)
        cre = np.array([complex(c).real for c, _ in terms] or [0.0], np.float64)
        cim = np.array([complex(c).imag for c, _ in terms] or [0.0], np.float64)
        out = C.c_void_p()
        _check(lib().pauli_wsum_jw_fermion(n, len(terms), _np_ptr(nf), _np_ptr(modes), _np_ptr(dag), _np_ptr(cre),
                                           _np_ptr(cim), eps_drop, C.byref(out)))
        return cls(out.value)

    @classmethod
    def jw_molecular(cls, h, g, e_nn: float = 0.0, eps_int: float = 0.0, eps_drop: float = 0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = C.c_void_p()
        _check(lib().pauli_wsum_jw_molecular(h.shape[0], _np_ptr(h), _np_ptr(g), e_nn, eps_int, eps_drop,
                                             C.byref(out)))
        return cls(out.value)

    def __matmul__(self, other: "WidePauliSum") -> "WidePauliSum":
        out = C.c_void_p()
        _check(lib().pauli_wsum_product(self._h, other._h, 0.0, C.byref(out)))
        return WidePauliSum(out.value)

    def info(self):
        n, wds, m, g = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        _check(lib().pauli_wsum_info(self._h, C.byref(n), C.byref(wds), C.byref(m), C.byref(g)))
        return n.value, wds.value, m.value, g.value

    @property
    def m(self) -> int:
        return self.info()[2]

    def export(self):
        """(x, z, C): lists of Python-int masks and a complex128 array (XZ form)."""
        n, W, m, _ = self.info()
        xw = np.zeros(max(m * W, 1), np.uint64)
        zw = np.zeros(max(m * W, 1), np.uint64)
        re = np.zeros(max(m, 1))
        im = np.zeros(max(m, 1))
        _check(lib().pauli_wsum_export(self._h, _np_ptr(xw), _np_ptr(zw), _np_ptr(re), _np_ptr(im)))
        def words(a, t):
            return sum(int(a[t * W + k]) << (64 * k) for k in range(W))
        return [words(xw, t) for t in range(m)], [words(zw, t) for t in range(m)], re[:m] + 1j * im[:m]

    def groups(self):
        _, _, _, g = self.info()
        gs = np.zeros(g + 1, np.int64)
        _check(lib().pauli_wsum_groups(self._h, _np_ptr(gs)))
        return gs

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_wsum_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def jw_molecular_raw(h, g, e_nn: float = 0.0, eps_int: float = 0.0):
    """Raw (pre-reduction) Jordan-Wigner entries (x, z, C) as numpy arrays."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    norb = h.shape[0]
    cnt = C.c_int64(0)
    _check(lib().pauli_jw_molecular_raw(norb, _np_ptr(h), _np_ptr(g), e_nn, eps_int, C.byref(cnt), None, None,
                                        None, None))
    n = cnt.value
    x = np.zeros(max(n, 1), np.uint64)
    z = np.zeros(max(n, 1), np.uint64)
    re = np.zeros(max(n, 1))
    im = np.zeros(max(n, 1))
    _check(lib().pauli_jw_molecular_raw(norb, _np_ptr(h), _np_ptr(g), e_nn, eps_int, C.byref(cnt), _np_ptr(x),
                                        _np_ptr(z), _np_ptr(re), _np_ptr(im)))
    return x[:n], z[:n], re[:n] + 1j * im[:n]


# ---------------------------------------------------------------------------
# sectors
# ---------------------------------------------------------------------------
class Sector:
    def __init__(self, n: int, kind: int = FULL, n_lo: int = 0, blocks: Sequence = ()):
        blocks = [tuple(b) for b in blocks]
        klo = np.array([b[0] for b in blocks] or [0], np.int32)
        khi = np.array([b[1] for b in blocks] or [0], np.int32)
        out = C.c_void_p()
        _check(lib().pauli_sector_create(n, kind, n_lo, len(blocks), _np_ptr(klo), _np_ptr(khi), C.byref(out)))
        self._h = out
        self.n, self.kind, self.n_lo, self.blocks = n, kind, n_lo, blocks
        d = C.c_int64()
        _check(lib().pauli_sector_dim(self._h, C.byref(d)))
        self.dim = d.value

    @classmethod
    def irrep_blocks(cls, n: int, n_lo: int, blocks, qubit_irrep):
        """Point-group blocks (k_lo, irrep_lo, k_hi, irrep_hi) with per-qubit irrep
        labels 0..7 (pauli_sector_create_irrep)."""
        self = cls.__new__(cls)
        blocks = [tuple(int(v) for v in b) for b in blocks]
        arr = lambda i: np.array([b[i] for b in blocks] or [0], np.int32)
        qi = np.ascontiguousarray(np.asarray(qubit_irrep, dtype=np.int32))
        if qi.size != n:
            raise ValueError("qubit_irrep needs one label per qubit")
        out = C.c_void_p()
        _check(lib().pauli_sector_create_irrep(n, n_lo, len(blocks), _np_ptr(arr(0)), _np_ptr(arr(1)), _np_ptr(arr(2)),
                                               _np_ptr(arr(3)), _np_ptr(qi), C.byref(out)))
        self._h = out
        self.n, self.kind, self.n_lo, self.blocks = n, BLOCKS, n_lo, blocks
        d = C.c_int64()
        _check(lib().pauli_sector_dim(self._h, C.byref(d)))
        self.dim = d.value
        return self

    @classmethod
    def full(cls, n: int, n_lo: int = 0):
        return cls(n, FULL, n_lo)

    @classmethod
    def molecular(cls, norb: int, na: int, nb: int):
        return cls(2 * norb, BLOCKS, norb, [(na, nb)])

    def rank(self, configs, stream=None):
        """configs: CUDA int64 tensor of bit patterns -> int64 indices (-1 outside)."""
        import torch
        configs = configs.contiguous()
        idx = torch.empty(configs.shape, dtype=torch.int64, device=configs.device)
        _check(lib().pauli_sector_rank(self._h, C.c_void_p(configs.data_ptr()), configs.numel(),
                                       C.c_void_p(idx.data_ptr()), _stream_ptr(stream)))
        return idx

    def unrank(self, idx, stream=None):
        import torch
        idx = idx.contiguous()
        cfg = torch.empty(idx.shape, dtype=torch.int64, device=idx.device)
        _check(lib().pauli_sector_unrank(self._h, C.c_void_p(idx.data_ptr()), idx.numel(),
                                         C.c_void_p(cfg.data_ptr()), _stream_ptr(stream)))
        return cfg

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_sector_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# operator-state products
# ---------------------------------------------------------------------------
def prepare(H: PauliSum, s: Sector):
    _check(lib().pauli_prepare(H._h, s._h))


def apply(H: PauliSum, s: Sector, psi_in, psi_out=None, stream=None):
    """psi_out = P_S H P_S psi_in on the device; returns psi_out."""
    import torch
    _check_state(psi_in, s.dim, "psi_in")
    if psi_out is None:
        psi_out = torch.empty_like(psi_in)
    _check_state(psi_out, s.dim, "psi_out")
    if psi_out.dtype != psi_in.dtype:
        raise TypeError("psi_in and psi_out must have the same dtype")
    _check(lib().pauli_apply(H._h, s._h, C.c_void_p(psi_in.data_ptr()), C.c_void_p(psi_out.data_ptr()),
                             _dtype_code(psi_in), _stream_ptr(stream)))
    return psi_out


def expect(H: PauliSum, s: Sector, psi, hpsi_out=None, result=None, stream=None):
    """Device tensor [Re E, Im E, ||H psi||^2, <psi|psi>] (float64); optionally stores H psi."""
    import torch
    _check_state(psi, s.dim, "psi")
    if result is None:
        result = torch.empty(4, dtype=torch.float64, device=psi.device)
    hp = None
    if hpsi_out is not None:
        _check_state(hpsi_out, s.dim, "hpsi_out")
        hp = C.c_void_p(hpsi_out.data_ptr())
    _check(lib().pauli_expect(H._h, s._h, C.c_void_p(psi.data_ptr()), _dtype_code(psi),
                              C.c_void_p(result.data_ptr()), hp, _stream_ptr(stream)))
    return result


def expect_rows(H: PauliSum, s: Sector, psi, rows, hpsi_out=None, result=None, stream=None):
    """Rows of H psi at the sector indices ``rows`` (device int64 tensor, distinct)
    written into ``hpsi_out`` (a full-length state; other entries untouched), and
    [Re, Im sum conj(psi_r) (H psi)_r, sum |(H psi)_r|^2, sum |psi_r|^2] over the
    rows (device float64[4], returned).  <psi|H|psi> when psi vanishes off the rows."""
    import torch
    _check_state(psi, s.dim, "psi")
    if not (isinstance(rows, torch.Tensor) and rows.dtype == torch.int64 and rows.is_cuda and rows.is_contiguous()
            and rows.dim() == 1):
        raise TypeError("rows: a contiguous 1-D int64 CUDA tensor")
    if result is None:
        result = torch.empty(4, dtype=torch.float64, device=psi.device)
    hp = None
    if hpsi_out is not None:
        _check_state(hpsi_out, s.dim, "hpsi_out")
        hp = C.c_void_p(hpsi_out.data_ptr())
    _check(lib().pauli_expect_rows(H._h, s._h, C.c_void_p(psi.data_ptr()), _dtype_code(psi),
                                   C.c_void_p(rows.data_ptr()), rows.numel(), hp, C.c_void_p(result.data_ptr()),
                                   _stream_ptr(stream)))
    return result


def expect_noalloc(H: PauliSum, s: Sector, psi, result, hpsi_out=None, stream=None):
    """pauli_expect with its scratch in a static device array: allocates nothing.

    For callers that cannot have device memory allocated for them.  Needs
    prepare(H, s) beforehand and a caller-provided ``result`` (float64[4] on the
    device); calls that overlap on the GPU race on the shared scratch."""
    _check_state(psi, s.dim, "psi")
    hp = None
    if hpsi_out is not None:
        _check_state(hpsi_out, s.dim, "hpsi_out")
        hp = C.c_void_p(hpsi_out.data_ptr())
    _check(lib().pauli_expect_noalloc(H._h, s._h, C.c_void_p(psi.data_ptr()), _dtype_code(psi),
                                      C.c_void_p(result.data_ptr()), hp, _stream_ptr(stream)))
    return result


class LaunchConfig(C.Structure):
    _fields_ = [("cols_per_thread", C.c_int), ("staged_rows", C.c_int), ("row_split", C.c_int),
                ("direct", C.c_int), ("ranked", C.c_int), ("ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def tune(H: PauliSum, s: Sector, dtype=None, reps: int = 5, cache: str | None = None, stream=None) -> dict:
    """Pick the fastest launch shape for (H, s, dtype) by timing the candidates
    (pauli_tune), or install it from a cache file of earlier results
    (pauli_tune_load / pauli_tune_save)."""
    import torch
    code = C64 if dtype in (None, torch.complex64) else C128
    if cache:
        prepare(H, s)
        found = C.c_int(0)
        _check(lib().pauli_tune_load(H._h, s._h, os.fsencode(cache), C.byref(found)))
        if found.value:
            out = launch_config(H, s, torch.complex64 if code == C64 else torch.complex128)
            if out["ms"] > 0:
                return dict(out, cached=True)
    cfg = LaunchConfig()
    _check(lib().pauli_tune(H._h, s._h, code, reps, C.byref(cfg), _stream_ptr(stream)))
    if cache:
        _check(lib().pauli_tune_save(H._h, s._h, os.fsencode(cache)))
    return dict(cfg.as_dict(), cached=False)


def svd_ranks(H: PauliSum, s: Sector, max_rank: int = 65):
    """(hist, batches): hist[R] = number of X-mask groups whose coefficient matrix
    has SVD rank R (pauli_svd_ranks), and the gather's on-the-fly batch count."""
    hist = np.zeros(max_rank, np.int32)
    nb = C.c_int(0)
    _check(lib().pauli_svd_ranks(H._h, s._h, _np_ptr(hist), max_rank, C.byref(nb)))
    return hist, nb.value


def set_launch_config(H: PauliSum, s: Sector, dtype, cfg: "LaunchConfig"):
    """Install a launch shape for (H, s, dtype) (pauli_set_launch_config)."""
    import torch
    code = C64 if dtype in (None, torch.complex64) else C128
    _check(lib().pauli_set_launch_config(H._h, s._h, code, C.byref(cfg)))


def launch_config(H: PauliSum, s: Sector, dtype=None) -> dict:
    import torch
    code = C64 if dtype in (None, torch.complex64) else C128
    cfg = LaunchConfig()
    _check(lib().pauli_get_launch_config(H._h, s._h, code, C.byref(cfg)))
    return cfg.as_dict()


class Batch:
    """Many (H_b, sector_b) pairs applied in one persistent launch."""

    def __init__(self, Hs, sectors, dtype=None):
        import torch
        self.code = C64 if dtype in (None, torch.complex64) else C128
        self.Hs, self.sectors = list(Hs), list(sectors)
        n = len(self.Hs)
        harr = (C.c_void_p * n)(*[h._h.value for h in self.Hs])
        sarr = (C.c_void_p * n)(*[s._h.value for s in self.sectors])
        out = C.c_void_p()
        _check(lib().pauli_batch_create(n, harr, sarr, self.code, C.byref(out)))
        self._h = out

    def _ptrs(self, tensors, name, allow_none=False):
        n = len(self.Hs)
        if tensors is None:
            return None
        vals = []
        for t, s in zip(tensors, self.sectors):
            if t is None and allow_none:
                vals.append(None)
                continue
            _check_state(t, s.dim, name)
            if _dtype_code(t) != self.code:
                raise TypeError(f"{name}: dtype does not match the batch")
            vals.append(t.data_ptr())
        return (C.c_void_p * n)(*vals)

    def apply(self, psis, outs=None, results=None, stream=None):
        """outs[b] = H_b psis[b]; results (device float64 [n, 4]) = per-state expectation data."""
        import torch
        if results is None:
            results = torch.empty((len(self.Hs), 4), dtype=torch.float64, device=psis[0].device)
        _check(lib().pauli_batch_apply(self._h, self._ptrs(psis, "psi_in"), self._ptrs(outs, "psi_out", True),
                                       C.c_void_p(results.data_ptr()), _stream_ptr(stream)))
        return results

    def tune(self, psis, outs=None, reps: int = 3, stream=None):
        cfg = LaunchConfig()
        _check(lib().pauli_batch_tune(self._h, self._ptrs(psis, "psi_in"), self._ptrs(outs, "psi_out", True), reps,
                                      C.byref(cfg), _stream_ptr(stream)))
        return cfg.as_dict()

    def set_launch_config(self, cfg: "LaunchConfig"):
        _check(lib().pauli_batch_set_launch_config(self._h, C.byref(cfg)))

    def launch_config(self) -> dict:
        cfg = LaunchConfig()
        _check(lib().pauli_batch_get_launch_config(self._h, C.byref(cfg)))
        return cfg.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Krylov:
    """m-vector Lanczos propagator psi <- exp(-i dt H) psi (device scalars, optional CUDA graph)."""

    def __init__(self, H: PauliSum, s: Sector, m: int = 20, dtype=None):
        import torch
        code = C64 if dtype in (None, torch.complex64) else C128
        out = C.c_void_p()
        _check(lib().pauli_krylov_create(H._h, s._h, m, code, C.byref(out)))
        self._h, self.H, self.s, self.m, self.code = out, H, s, m, code

    def step(self, psi, dt: float, nsteps: int = 1, graph: bool = True, stream=None):
        _check_state(psi, self.s.dim, "psi")
        if _dtype_code(psi) != self.code:
            raise TypeError("psi dtype does not match the propagator")
        _check(lib().pauli_krylov_step(self._h, C.c_void_p(psi.data_ptr()), float(dt), int(nsteps), int(graph),
                                       _stream_ptr(stream)))
        return psi

    def scalars(self, stream=None):
        a = np.zeros(self.m)
        b = np.zeros(self.m + 1)
        _check(lib().pauli_krylov_scalars(self._h, _np_ptr(a), _np_ptr(b), _stream_ptr(stream)))
        return a, b

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_krylov_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RotSeq:
    """A fixed product of single-group rotations applied tile by tile
    (pauli_rotseq_*): apply(thetas, psi) = rotate_seq(gens, s, thetas, psi)."""

    def __init__(self, generators, s: Sector):
        self.s = s
        self.gens = list(generators)  # kept alive with the handle
        self.K = len(self.gens)
        arr = (C.c_void_p * self.K)(*[G._h.value for G in self.gens])
        out = C.c_void_p()
        _check(lib().pauli_rotseq_create(arr, self.K, s._h, C.byref(out)))
        self._h = out

    def apply(self, thetas, psi, stream=None):
        _check_state(psi, self.s.dim, "psi")
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1))
        if th.size != self.K:
            raise ValueError(f"expected {self.K} angles, got {th.size}")
        _check(lib().pauli_rotseq_apply(self._h, _np_ptr(th), C.c_void_p(psi.data_ptr()), _dtype_code(psi),
                                        _stream_ptr(stream)))
        return psi

    def info(self, dtype=None):
        import torch
        code = C64 if dtype in (None, torch.complex64) else C128
        nl, nf = C.c_int(), C.c_int()
        _check(lib().pauli_rotseq_info(self._h, code, C.byref(nl), C.byref(nf)))
        return {"launches": nl.value, "fused": nf.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_rotseq_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """Operator pool of ADAPT-VQE: K single-X-group Hermitian generators on one
    sector; gradients() gives dE/dtheta_k = 2 Im <H psi|G_k psi> for all k in
    one pass (pauli_pool_gradients)."""

    def __init__(self, generators, s: Sector):
        self.s = s
        self.K = len(generators)
        arr = (C.c_void_p * self.K)(*[G._h.value for G in generators])
        out = C.c_void_p()
        _check(lib().pauli_pool_create(arr, self.K, s._h, C.byref(out)))
        self._h = out

    def gradients(self, psi, hpsi, out=None, stream=None):
        import torch
        _check_state(psi, self.s.dim, "psi")
        _check_state(hpsi, self.s.dim, "hpsi")
        if psi.dtype != hpsi.dtype:
            raise TypeError("psi and hpsi must have the same dtype")
        if out is None:
            out = torch.empty(self.K, dtype=torch.float64, device=psi.device)
        _check(lib().pauli_pool_gradients(self._h, C.c_void_p(psi.data_ptr()), C.c_void_p(hpsi.data_ptr()),
                                          _dtype_code(psi), C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_pool_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rotate(G: PauliSum, s: Sector, theta: float, psi, stream=None):
    """psi <- exp(-i theta G) psi in place (G: one Hermitian X-group)."""
    _check_state(psi, s.dim, "psi")
    _check(lib().pauli_rotate(G._h, s._h, float(theta), C.c_void_p(psi.data_ptr()), _dtype_code(psi),
                              _stream_ptr(stream)))
    return psi


def rotate_seq(Gs, s: Sector, thetas, psi, stream=None):
    """psi <- prod_j exp(-i thetas[j] Gs[j]) psi in place, G_0 applied first."""
    _check_state(psi, s.dim, "psi")
    k = len(Gs)
    if len(thetas) != k:
        raise ValueError("Gs and thetas differ in length")
    hs = (C.c_void_p * max(k, 1))(*[G._h.value for G in Gs])
    th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1))
    _check(lib().pauli_rotate_seq(hs, _np_ptr(th), k, s._h, C.c_void_p(psi.data_ptr()), _dtype_code(psi),
                                  _stream_ptr(stream)))
    return psi


def rotate_adjoint(G: PauliSum, s: Sector, theta: float, phi, lam, out, stream=None):
    """out[0:2] <- (Re, Im) <lam|G|phi> (device float64), then phi, lam <-
    exp(-i theta G) phi, lam in place."""
    _check_state(phi, s.dim, "phi")
    _check_state(lam, s.dim, "lam")
    _check(lib().pauli_rotate_adjoint(G._h, s._h, float(theta), C.c_void_p(phi.data_ptr()),
                                      C.c_void_p(lam.data_ptr()), _dtype_code(phi), C.c_void_p(out.data_ptr()),
                                      _stream_ptr(stream)))
    return out


def vdot(x, y, out=None, stream=None):
    """<x|y> accumulated in FP64 on the device.  With out (a float64 device
    tensor of 2) the result stays on the device; otherwise a Python complex."""
    import torch
    if x.dtype != y.dtype or x.numel() != y.numel():
        raise TypeError("x and y must have the same dtype and size")
    for v, nm in ((x, "x"), (y, "y")):
        if not v.is_cuda or not v.is_contiguous() or v.data_ptr() % 16:
            raise ValueError(f"{nm} must be a contiguous 16-byte aligned CUDA tensor")
    res = out if out is not None else torch.empty(2, dtype=torch.float64, device=x.device)
    if res.dtype != torch.float64 or res.numel() < 2 or not res.is_cuda:
        raise ValueError("out must be a float64 CUDA tensor of 2 elements")
    _check(lib().pauli_vdot(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), int(x.numel()), _dtype_code(x),
                            C.c_void_p(res.data_ptr()), _stream_ptr(stream)))
    if out is not None:
        return out
    r = res.cpu()
    return complex(float(r[0]), float(r[1]))


class MLP:
    """Geometry -> ansatz-amplitude network of the learned warm start
    (two tanh hidden layers; BF16 tensor-core products, FP32 master weights,
    Adam).  Parameters are one FP32 vector: W1[in][hid], b1, W2[hid][hid], b2,
    W3[hid][out], b3."""

    def __init__(self, in_dim: int, hidden: int, out_dim: int, max_batch: int):
        out = C.c_void_p()
        _check(lib().pauli_mlp_create(int(in_dim), int(hidden), int(out_dim), int(max_batch), C.byref(out)))
        self._h = out
        self.in_dim, self.hidden, self.out_dim, self.max_batch = in_dim, hidden, out_dim, max_batch
        n = C.c_int64()
        _check(lib().pauli_mlp_num_params(self._h, C.byref(n)))
        self.num_params = n.value

    def shapes(self):
        i, h, o = self.in_dim, self.hidden, self.out_dim
        return [("W1", (i, h)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)), ("W3", (h, o)), ("b3", (o,))]

    def set_params(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if p.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {p.size}")
        _check(lib().pauli_mlp_set_params(self._h, _np_ptr(p)))

    def get_params(self):
        p = np.zeros(self.num_params, dtype=np.float32)
        _check(lib().pauli_mlp_get_params(self._h, _np_ptr(p)))
        return p

    def _check_batch(self, x, width, nm):
        import torch
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.dim() != 2 or x.shape[1] != width:
            raise ValueError(f"{nm} must be a contiguous float32 CUDA tensor of shape (batch, {width})")
        if not 1 <= x.shape[0] <= self.max_batch:
            raise ValueError("batch size out of range")

    def forward(self, x, stream=None):
        import torch
        self._check_batch(x, self.in_dim, "x")
        y = torch.empty(x.shape[0], self.out_dim, dtype=torch.float32, device=x.device)
        _check(lib().pauli_mlp_forward(self._h, int(x.shape[0]), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                       _stream_ptr(stream)))
        return y

    def backward(self, x, target, want_grads: bool = False, stream=None):
        """Loss 1/(2B) sum (y - target)^2 as a float64 device tensor (and the
        gradient vector when want_grads)."""
        import torch
        self._check_batch(x, self.in_dim, "x")
        self._check_batch(target, self.out_dim, "target")
        if target.shape[0] != x.shape[0]:
            raise ValueError("x and target differ in batch size")
        loss = torch.empty(1, dtype=torch.float64, device=x.device)
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device) if want_grads else None
        _check(lib().pauli_mlp_backward(self._h, int(x.shape[0]), C.c_void_p(x.data_ptr()),
                                        C.c_void_p(target.data_ptr()), C.c_void_p(g.data_ptr() if g is not None else 0),
                                        C.c_void_p(loss.data_ptr()), _stream_ptr(stream)))
        return (loss, g) if want_grads else loss

    def train(self, x, target, steps: int, lr: float, t0: int, stream=None):
        """steps Adam steps (t = t0+1 ..) on (x, target) in one library call;
        returns the last step's loss as a float64 device tensor."""
        import torch
        self._check_batch(x, self.in_dim, "x")
        self._check_batch(target, self.out_dim, "target")
        if target.shape[0] != x.shape[0]:
            raise ValueError("x and target differ in batch size")
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device=x.device)
        _check(lib().pauli_mlp_train(self._h, int(x.shape[0]), C.c_void_p(x.data_ptr()),
                                     C.c_void_p(target.data_ptr()), int(steps), C.c_float(lr), int(t0),
                                     C.c_void_p(loss.data_ptr()), _stream_ptr(stream)))
        return loss

    def adam_step(self, lr: float, t: int, stream=None):
        _check(lib().pauli_mlp_adam_step(self._h, C.c_float(lr), int(t), _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            if _lib is not None:
                lib().pauli_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
