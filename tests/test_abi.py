"""The C-ABI library builds, loads without a GPU and exports every symbol of include/paulisim.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "paulisim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pauli_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_28952_gb300 import build_lib
    return build_lib.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pauli_sum_build", "pauli_apply", "pauli_expect", "pauli_rotate", "pauli_jw_molecular",
                     "pauli_sector_create", "pauli_sector_rank", "pauli_status"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    import paper_2606_28952_gb300 as ps
    assert set(_declared_functions()) == set(ps.SIGNATURES)
    L = ps.lib()
    assert L.pauli_version() >= 10000
    assert L.pauli_last_error() == b""


def test_calls_fail_loudly_without_a_gpu(libpath):
    """No CPU fallback: without a usable GPU a build call returns an error status."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2606_28952_gb300 as ps
    with pytest.raises(ps.PauliError):
        ps.PauliSum.from_terms(2, [1], [0], [1.0])


def test_invalid_arguments_rejected_on_host(libpath):
    """Host-side validation runs before any device work."""
    import paper_2606_28952_gb300 as ps
    with pytest.raises(ps.PauliError) as e:
        ps.PauliSum.from_terms(3, [8], [0], [1.0])  # bit 3 set on a 3-qubit string
    assert e.value.code == ps.EINVAL
    with pytest.raises(ps.PauliError) as e:
        ps.PauliSum.from_terms(3, [1], [0], [float("nan")])
    assert e.value.code == ps.EINVAL
    with pytest.raises(ps.PauliError) as e:
        ps.Sector(12, ps.BLOCKS, 6, [(3, 3), (2, 3)])  # repeated k_hi
    assert e.value.code == ps.EINVAL
