"""lbm_reduce_noalloc: the FP64 reductions for callers that cannot allocate
device memory (a host application that gives the library a fixed budget of
buffers, or code that runs where cudaMalloc is not permitted).  It keeps its
scratch in a static device array of the library instead of the scratch buffer
lent through lbm_bind, and must give the same results as lbm_reduce.

This file is collected last on purpose: it runs after every other test."""
import ctypes

import pytest
import torch

from paper_1803_04937_gb300 import _lib
from tests._helpers import random_fields

pytestmark = pytest.mark.gpu

REL_TOL = {"f64": 1e-12, "f32": 1e-5}


def _call(fn, handle):
    out = (ctypes.c_double * _lib.RED_COUNT)()
    status = fn(handle, out)
    return status, list(out)


def _close(a, b, tol):
    return all(abs(x - y) <= tol * max(abs(x), abs(y), 1e-300) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_reduce_noalloc_matches_reduce_on_two_calls(precision, pattern):
    from paper_1803_04937_gb300.lbm import Simulation
    lib = _lib.load()
    shape = (9, 12, 41)
    rho, u = random_fields(shape, seed=31)
    sim = Simulation(41, 12, 9, collision="trt", tau=0.7, precision=precision, pattern=pattern,
                     force=(1e-4, 0.0, -2e-4), walls=(False, True, False))
    sim.init(rho.cuda(), u.cuda())
    sim.step(3)
    for _ in range(2):
        s_ref, ref = _call(lib.lbm_reduce, sim.handle)
        s_new, new = _call(lib.lbm_reduce_noalloc, sim.handle)
        assert s_ref == _lib.LBM_OK and s_new == _lib.LBM_OK
        assert _close(ref[:7], new[:7], REL_TOL[precision]), (ref, new)
        assert new[_lib.RED_NONFINITE] == 0
        sim.step(1)


def test_reduce_noalloc_works_without_a_scratch_buffer():
    """Bound with scratch = NULL, lbm_reduce refuses while lbm_reduce_noalloc
    still answers, twice in a row, with lbm_reduce's values."""
    from paper_1803_04937_gb300.lbm import Simulation
    lib = _lib.load()
    shape = (6, 7, 33)
    rho, u = random_fields(shape, seed=32)
    sim = Simulation(33, 7, 6, precision="f64")
    sim.init(rho.cuda(), u.cuda())
    sim.step(2)
    _, ref = _call(lib.lbm_reduce, sim.handle)
    stream = ctypes.c_void_p(sim.stream.cuda_stream)
    a, b = sim.grids
    _lib.check(lib.lbm_bind(sim.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), None, stream),
               sim.handle)
    s, _ = _call(lib.lbm_reduce, sim.handle)
    assert s == _lib.LBM_ESTATE
    for _ in range(2):
        s, new = _call(lib.lbm_reduce_noalloc, sim.handle)
        assert s == _lib.LBM_OK
        assert _close(ref[:7], new[:7], REL_TOL["f64"]), (ref, new)
    torch.cuda.synchronize()
