"""Host-side checks of the C ABI: the library loads, exports every function
include/lbm.h declares, and validates arguments without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1803_04937_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load(build_if_missing=True)


def test_every_declared_symbol_is_exported_and_bound(lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == _lib.exported_symbols()


def test_abi_version_and_velocity_set(lib):
    assert lib.lbm_abi_version() == 1
    c = (ctypes.c_int * 57)()
    w = (ctypes.c_double * 19)()
    o = (ctypes.c_int * 19)()
    assert lib.lbm_velocity_set(c, w, o) == 0
    vel = [tuple(c[3 * q:3 * q + 3]) for q in range(19)]
    assert len(set(vel)) == 19
    assert abs(sum(w) - 1.0) < 1e-15
    for q in range(19):
        assert vel[o[q]] == tuple(-a for a in vel[q])


def test_d3q27_velocity_set_and_handle(lib):
    c = (ctypes.c_int * 81)()
    w = (ctypes.c_double * 27)()
    o = (ctypes.c_int * 27)()
    assert lib.lbm_velocity_set_of(27, c, w, o) == 0
    vel = [tuple(c[3 * q:3 * q + 3]) for q in range(27)]
    assert len(set(vel)) == 27 and abs(sum(w) - 1.0) < 1e-15
    assert all(vel[o[q]] == tuple(-a for a in vel[q]) for q in range(27))
    assert lib.lbm_velocity_set_of(15, c, w, o) == _lib.LBM_EUNSUPPORTED
    h = ctypes.c_void_p()
    assert lib.lbm_create(8, 6, 4, 27, 0, 0, 0.8, 1, ctypes.byref(h)) == 0
    try:
        pdf = ctypes.c_size_t()
        assert lib.lbm_required_bytes(h, ctypes.byref(pdf), None, None) == 0
        assert pdf.value == 27 * 8 * 6 * 4 * 4
        assert lib.lbm_set_option(h, _lib.OPT_PATTERN, 1) == _lib.LBM_EUNSUPPORTED
    finally:
        lib.lbm_destroy(h)


def test_create_validates_arguments_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(0, 4, 4, 19, 1, 0, 0.8, 1, ctypes.byref(h)) == _lib.LBM_EINVAL
    assert lib.lbm_create(4, 4, 4, 15, 1, 0, 0.8, 1, ctypes.byref(h)) == _lib.LBM_EUNSUPPORTED
    assert lib.lbm_create(4, 4, 4, 19, 1, 0, 0.5, 1, ctypes.byref(h)) == _lib.LBM_EINVAL
    assert lib.lbm_create(4, 4, 4, 19, 1, 0, 0.8, 9, ctypes.byref(h)) == _lib.LBM_EINVAL
    assert lib.lbm_create(2048, 1024, 1024, 19, 1, 0, 0.8, 1, ctypes.byref(h)) == _lib.LBM_EUNSUPPORTED
    assert lib.lbm_create(8, 6, 4, 19, 1, 1, 0.8, 2, ctypes.byref(h)) == _lib.LBM_OK
    try:
        pdf = ctypes.c_size_t()
        ng = ctypes.c_int()
        sb = ctypes.c_size_t()
        assert lib.lbm_required_bytes(h, ctypes.byref(pdf), ctypes.byref(ng), ctypes.byref(sb)) == 0
        assert pdf.value == 19 * 8 * 6 * 4 * 2 and ng.value == 2 and sb.value % 256 == 0 and sb.value > 0
        assert lib.lbm_set_option(h, _lib.OPT_PATTERN, 1) == 0
        assert lib.lbm_required_bytes(h, None, ctypes.byref(ng), None) == 0 and ng.value == 1
        assert lib.lbm_set_option(h, 999, 1.0) == _lib.LBM_EINVAL
        assert b"unknown option" in lib.lbm_last_error(h)
        assert lib.lbm_set_option(h, _lib.OPT_WALLS_Y, 0.5) == _lib.LBM_EINVAL
        assert lib.lbm_set_option(h, _lib.OPT_BLOCK_X, 48) == _lib.LBM_EINVAL
        v = ctypes.c_double()
        assert lib.lbm_set_option(h, _lib.OPT_TRT_MAGIC, 0.25) == 0
        assert lib.lbm_get_option(h, _lib.OPT_TRT_MAGIC, ctypes.byref(v)) == 0 and v.value == 0.25
        # calls that need device memory fail cleanly before any CUDA call
        assert lib.lbm_step(h, 1) == _lib.LBM_ESTATE
        assert lib.lbm_init(h, None, None, 0) == _lib.LBM_ESTATE
        out = (ctypes.c_double * 8)()
        assert lib.lbm_reduce(h, out) == _lib.LBM_ESTATE
        # misaligned device pointers are rejected on the host
        assert lib.lbm_bind(h, ctypes.c_void_p(0x1001), None, None, None) == _lib.LBM_EINVAL
        # tau gradient helper (host only): SRT d omega / d tau = -1/tau^2
        assert lib.lbm_set_option(h, _lib.OPT_COLLISION, 0) == 0
        g = (ctypes.c_double * 2)(1.0, 1.0)
        d = ctypes.c_double()
        assert lib.lbm_adjoint_tau_gradient(h, g, ctypes.byref(d)) == 0
        assert abs(d.value - 2 * (-1 / 0.8 ** 2)) < 1e-14
    finally:
        assert lib.lbm_destroy(h) == 0


def test_mrt_options_and_refusals_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(8, 6, 4, 27, 1, _lib.MRT, 0.8, 1, ctypes.byref(h)) == _lib.LBM_EUNSUPPORTED
    assert lib.lbm_create(8, 6, 4, 27, 1, _lib.TRT, 0.8, 1, ctypes.byref(h)) == _lib.LBM_OK
    try:
        assert lib.lbm_set_option(h, _lib.OPT_COLLISION, _lib.MRT) == _lib.LBM_EUNSUPPORTED
    finally:
        lib.lbm_destroy(h)
    assert lib.lbm_create(8, 6, 4, 19, 1, _lib.MRT, 0.8, 1, ctypes.byref(h)) == _lib.LBM_OK
    try:
        v = ctypes.c_double()
        for key in (_lib.OPT_MRT_OMEGA_BULK, _lib.OPT_MRT_OMEGA_4):
            assert lib.lbm_get_option(h, key, ctypes.byref(v)) == 0 and v.value == 1.0
            assert lib.lbm_set_option(h, key, 0.0) == _lib.LBM_EINVAL
            assert lib.lbm_set_option(h, key, 2.0) == _lib.LBM_EINVAL
            assert lib.lbm_set_option(h, key, 1.3) == 0
            assert lib.lbm_get_option(h, key, ctypes.byref(v)) == 0 and v.value == 1.3
        assert lib.lbm_get_option(h, _lib.OPT_COLLISION, ctypes.byref(v)) == 0 and v.value == _lib.MRT
        g = (ctypes.c_double * 2)(1.0, 1.0)
        d = ctypes.c_double()
        assert lib.lbm_adjoint_tau_gradient(h, g, ctypes.byref(d)) == _lib.LBM_EUNSUPPORTED
        assert b"SRT and TRT" in lib.lbm_last_error(h)
    finally:
        lib.lbm_destroy(h)


def test_graph_and_block_options_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_create(64, 8, 4, 19, 1, 0, 0.8, 2, ctypes.byref(h)) == _lib.LBM_OK
    try:
        v = ctypes.c_double()
        assert lib.lbm_get_option(h, _lib.OPT_GRAPHS, ctypes.byref(v)) == 0 and v.value == 1.0
        assert lib.lbm_set_option(h, _lib.OPT_GRAPHS, 0.5) == _lib.LBM_EINVAL
        assert lib.lbm_set_option(h, _lib.OPT_GRAPHS, 0.0) == 0
        assert lib.lbm_get_option(h, _lib.OPT_GRAPHS, ctypes.byref(v)) == 0 and v.value == 0.0
        # 16-bit storage defaults to four cells per thread
        assert lib.lbm_get_option(h, _lib.OPT_CELLS_X, ctypes.byref(v)) == 0 and v.value == 4.0
        assert lib.lbm_set_option(h, _lib.OPT_CELLS_X, 3.0) == _lib.LBM_EINVAL
        assert lib.lbm_set_option(h, _lib.OPT_TAU, 0.5) == _lib.LBM_EINVAL
        assert lib.lbm_set_option(h, _lib.OPT_TAU, float("nan")) == _lib.LBM_EINVAL
        assert lib.lbm_step(h, -1) in (_lib.LBM_EINVAL, _lib.LBM_ESTATE)
        # deferred adjoint sums: 0 or 1, default 0; nothing is pending on an unbound handle
        assert lib.lbm_get_option(h, _lib.OPT_ADJ_DEFER_SUM, ctypes.byref(v)) == 0 and v.value == 0.0
        assert lib.lbm_set_option(h, _lib.OPT_ADJ_DEFER_SUM, 2.0) == _lib.LBM_EINVAL
        assert lib.lbm_set_option(h, _lib.OPT_ADJ_DEFER_SUM, 1.0) == 0
        assert lib.lbm_get_option(h, _lib.OPT_ADJ_DEFER_SUM, ctypes.byref(v)) == 0 and v.value == 1.0
        assert lib.lbm_adjoint_flush(h) == _lib.LBM_ESTATE  # no bound memory
    finally:
        lib.lbm_destroy(h)
