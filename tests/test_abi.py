"""The C-ABI library loads and exports every entry point of include/lbm.h, and its
host-side validation works without a GPU (no CUDA call is made for bad input)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def L():
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    lib = L.library()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers exactly the header
    assert sorted(s[0] for s in L.SIGNATURES) == names


def test_struct_layouts_match_header(L):
    import ctypes
    assert ctypes.sizeof(L.lbm_params) == 8 * 4 + 11 * 8
    assert ctypes.sizeof(L.lbm_diag) == 14 * 8 + 2 * 4 + 8
    assert ctypes.sizeof(L.lbm_monitor) == 3 * 8 + 2 * 4 + 8


def _valid():
    from paper_1902_08933_gb300 import lbm, workloads
    return lbm.make_params(workloads.static_droplet(n=16))


@pytest.mark.parametrize("field,value", [
    ("nx", 2), ("ny", 0), ("bc_y", 2), ("variant", 5), ("pressure_scheme", 3),
    ("surface_force", -1), ("viscosity_model", 2), ("nz", -1), ("rho_A", 0.0),
    ("rho_B", -1.0), ("nu_A", 0.0), ("W", 0.0), ("sigma", -1e-3), ("tau_h", 0.5),
    ("mobility", -0.1), ("gravity", float("nan")), ("force_x", float("inf"))])
def test_validation_rejects(L, field, value):
    p = _valid()
    assert L.lbm_validate_params(p) == L.LBM_OK
    setattr(p, field, value)
    assert L.lbm_validate_params(p) == L.LBM_EINVAL


def test_create_rejects_bad_input_without_touching_cuda(L):
    import ctypes
    lib = L.library()
    p = _valid()
    p.tau_h = 0.2
    out = ctypes.c_void_p(1234)
    arr = (L.lbm_params * 1)(p)
    assert lib.lbm_create(arr, 1, 0, None, ctypes.byref(out)) == L.LBM_EINVAL
    assert out.value is None
    good = (L.lbm_params * 1)(_valid())
    assert lib.lbm_create(good, 0, 0, None, ctypes.byref(out)) == L.LBM_EINVAL
    assert lib.lbm_create(good, 1, 7, None, ctypes.byref(out)) == L.LBM_EINVAL
    assert lib.lbm_create(good, 1, 0, None, None) == L.LBM_EINVAL
    # D3Q15 (nz >= 2): one lattice a context, and no FP16 storage forms
    p3 = _valid()
    p3.nz = 8
    assert L.lbm_validate_params(p3) == L.LBM_OK
    mixed = (L.lbm_params * 2)(_valid(), p3)
    assert lib.lbm_create(mixed, 2, 0, None, ctypes.byref(out)) == L.LBM_EINVAL
    only3 = (L.lbm_params * 1)(p3)
    for form in (L.LBM_F32_G16, L.LBM_F32_H16):
        assert lib.lbm_create(only3, 1, form, None, ctypes.byref(out)) == L.LBM_EINVAL
    # the single-phase model of Remark 3
    sp = L.lbm_sp_params(16, 16, 0, 0, 0.1, 0.0, 0.0, 0.0)
    spo = ctypes.c_void_p(1234)
    for field, value in (("nx", 2), ("bc_y", 5), ("model", 3), ("model", 2), ("nu", 0.0), ("xi", -1.0),
                         ("force_x", float("nan")), ("scheme", 2), ("reserved", 1),
                         ("drag_lin", 0.1), ("drag_quad", 0.1)):   # model 2 needs p0 > 0; drag the Remark 4 scheme
        bad = L.lbm_sp_params(16, 16, 0, 0, 0.1, 0.0, 0.0, 0.0)
        setattr(bad, field, value)
        assert lib.lbm_sp_create(ctypes.byref(bad), 0, None, ctypes.byref(spo)) == L.LBM_EINVAL
        assert spo.value is None
    for field, value in (("drag_lin", -1.0), ("drag_quad", float("inf")), ("model", 1)):
        bad = L.lbm_sp_params(16, 16, 0, 0, 0.1, 0.0, 0.0, 0.0, 1)   # Remark 4 scheme
        setattr(bad, field, value)
        assert lib.lbm_sp_create(ctypes.byref(bad), 0, None, ctypes.byref(spo)) == L.LBM_EINVAL
        assert spo.value is None
    assert lib.lbm_sp_create(ctypes.byref(sp), L.LBM_F32_C, None, ctypes.byref(spo)) == L.LBM_EINVAL
    assert lib.lbm_sp_step(None, 1) == L.LBM_EINVAL and lib.lbm_sp_init(None, None) == L.LBM_EINVAL
    lib.lbm_sp_destroy(None)
    big = _valid()
    big.nx, big.ny, big.nz = 2048, 2048, 512
    assert L.lbm_validate_params(big) == L.LBM_EINVAL     # 2^31 cells


def test_null_context_calls_are_errors(L):
    lib = L.library()
    assert lib.lbm_step(None, 1) == L.LBM_EINVAL
    assert lib.lbm_sync(None) == L.LBM_EINVAL
    assert lib.lbm_inject_wait_timeout(None, 16) == L.LBM_EINVAL
    assert lib.lbm_set_monitor(None, 1) == L.LBM_EINVAL
    assert lib.lbm_read_monitor(None, 0, None) == L.LBM_EINVAL
    assert lib.lbm_read_monitor_async(None, 0, None) == L.LBM_EINVAL
    assert lib.lbm_time(None, 0) == -1
    assert lib.lbm_launches_per_step(None) == 0
    lib.lbm_destroy(None)
