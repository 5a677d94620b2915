"""The C-ABI library builds, loads and exports every symbol include/kry.h declares (no GPU).

Only calls that fail argument validation before touching CUDA are made here.
"""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "kry.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kry_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_02770_gb300 import build
    path = build.build()
    import paper_1704_02770_gb300 as k
    return k.load(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 12
    import paper_1704_02770_gb300 as k
    for n in names:
        assert hasattr(lib, n), n
        assert n in k.SIGNATURES, f"binding lacks {n}"


def test_binding_declares_nothing_extra():
    import paper_1704_02770_gb300 as k
    assert set(k.SIGNATURES) == set(declared_symbols())


def test_argument_validation_without_gpu(lib):
    import paper_1704_02770_gb300 as k
    h = ctypes.c_void_p()
    assert lib.kry_basis_create(0, 0, ctypes.byref(h)) == k.KRY_EINVAL
    assert b"1 <= L <= 64" in lib.kry_last_error()
    assert lib.kry_basis_create(65, 3, ctypes.byref(h)) == k.KRY_EINVAL
    assert lib.kry_basis_create_list(65, 3, ctypes.byref(h)) == k.KRY_EINVAL
    assert lib.kry_basis_create_list(40, 20, ctypes.byref(h)) == k.KRY_EINVAL   # D > 2^31 - 1
    assert b"exceeds" in lib.kry_last_error()
    assert lib.kry_basis_create(8, 9, ctypes.byref(h)) == k.KRY_EINVAL
    assert lib.kry_basis_dim(None) == -1
    assert lib.kry_hamiltonian_set(None, 1.0, 1.0, None, 1, 1, ctypes.byref(h)) == k.KRY_EINVAL
    assert lib.kry_apply(None, 0, None, None, None) == k.KRY_EINVAL
    t = (ctypes.c_double * 2)(0.0, 1.0)
    P = (ctypes.c_double * 2)()
    assert lib.kry_return_probability(None, 0, 3, t, 2, 30, 1e-10, P, None, None) == k.KRY_EINVAL
    C = (ctypes.c_double * 2)()
    assert lib.kry_autocorrelation(None, 0, 3, t, 2, 30, 1e-10, C, P, None, None) == k.KRY_EINVAL
    assert lib.kry_autocorrelation(None, 0, 3, t, 2, 30, 1e-10, None, P, None, None) == k.KRY_EINVAL
    assert b"C_out" in lib.kry_last_error()
    assert lib.kry_tridiag_expv(None, None, 0, 0.0, 0.0, None, None, None) == k.KRY_EINVAL
    assert lib.kry_workspace_size(None, 0, 30) == -1
    assert lib.kry_workspace_bytes(None, 0, 30, 40) == -1
    assert lib.kry_set_workspace(None, None, 0) == k.KRY_EINVAL
    assert lib.kry_basis_destroy(None) == k.KRY_OK
    assert lib.kry_hamiltonian_destroy(None) == k.KRY_OK


def test_sources_target_sm103a_only():
    from paper_1704_02770_gb300 import build
    f = build.flags()
    assert "arch=compute_103a,code=sm_103a" in f
    assert not any("sm_90" in x or "sm_100" in x for x in f)


def test_binding_refuses_tensors_the_kernels_would_overrun():
    """The binding hands the library only tensors of the element type and size it will read
    or write: a complex64 output for a complex128 input, int32 states or int64 ranks would
    send a kernel past the end of the buffer, so they are refused before any call."""
    import torch
    import paper_1704_02770_gb300 as k
    with pytest.raises(TypeError):
        k._dev_ptr(torch.zeros(4, dtype=torch.complex64), 4, torch.complex128)
    with pytest.raises(TypeError):
        k._dev_ptr(torch.zeros(4, dtype=torch.int32), dtype=torch.int64)
    with pytest.raises(TypeError):
        k._dev_ptr(torch.zeros(4, dtype=torch.int64), dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA"):        # the right type, but host memory
        k._dev_ptr(torch.zeros(4, dtype=torch.int64), dtype=torch.int64)
    with pytest.raises(TypeError):
        k._dtype_code(torch.zeros(4, dtype=torch.float64))
    # the checks run before the library is called: a stub Hamiltonian whose handle is unset
    H = object.__new__(k.Hamiltonian)
    H._h, H.K = None, 1
    H.basis = type("B", (), {"dim": 4})()
    with pytest.raises(ValueError, match="CUDA"):
        H.apply(torch.zeros(4, dtype=torch.complex128))
    with pytest.raises(TypeError):
        H.evolve(torch.zeros(4, dtype=torch.float32), [1.0])
