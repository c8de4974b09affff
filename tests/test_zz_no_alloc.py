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


_RESET_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1803_04937_gb300 import _lib
lib = _lib.load()
rt = ctypes.CDLL("libcudart.so.13")   # the runtime the library itself links
vp, sz = ctypes.c_void_p, ctypes.c_size_t
rt.cudaMalloc.argtypes = [ctypes.POINTER(vp), sz]
rt.cudaFree.argtypes = [vp]
rt.cudaMemcpy.argtypes = [vp, vp, sz, ctypes.c_int]
rt.cudaStreamCreate.argtypes = [ctypes.POINTER(vp)]
rt.cudaStreamDestroy.argtypes = [vp]

def ok(e, what):
    if e != 0:
        raise SystemExit("%s failed: %d" % (what, e))

nx, ny, nz = 33, 7, 6
rng = np.random.default_rng(33)
u = np.ascontiguousarray(rng.uniform(-0.05, 0.05, (3, nz, ny, nx)))
for rnd in range(2):
    ok(rt.cudaSetDevice(0), "cudaSetDevice")
    h = vp()
    _lib.check(lib.lbm_create(nx, ny, nz, 19, _lib.EQ_IMPROVED, _lib.TRT, 0.7, _lib.F64, ctypes.byref(h)))
    _lib.check(lib.lbm_set_option(h, _lib.OPT_FORCE_X, 1e-4), h)
    pdf, ng, scr = sz(), ctypes.c_int(), sz()
    _lib.check(lib.lbm_required_bytes(h, ctypes.byref(pdf), ctypes.byref(ng), ctypes.byref(scr)), h)
    bufs = {}
    for name, n in (("a", pdf.value), ("b", pdf.value), ("scratch", scr.value), ("u", u.nbytes)):
        p = vp()
        ok(rt.cudaMalloc(ctypes.byref(p), n), "cudaMalloc")
        bufs[name] = p
    ok(rt.cudaMemcpy(bufs["u"], u.ctypes.data, u.nbytes, 1), "cudaMemcpy")
    stream = vp()
    ok(rt.cudaStreamCreate(ctypes.byref(stream)), "cudaStreamCreate")
    _lib.check(lib.lbm_bind(h, bufs["a"], bufs["b"], bufs["scratch"], stream), h)
    _lib.check(lib.lbm_init(h, None, bufs["u"], _lib.DTYPE_F64), h)
    _lib.check(lib.lbm_step(h, 3), h)
    ref = (ctypes.c_double * _lib.RED_COUNT)()
    _lib.check(lib.lbm_reduce(h, ref), h)
    for _ in range(2):
        new = (ctypes.c_double * _lib.RED_COUNT)()
        _lib.check(lib.lbm_reduce_noalloc(h, new), h)
        for i in range(7):
            assert abs(ref[i] - new[i]) <= 1e-12 * max(abs(ref[i]), abs(new[i]), 1e-300), (rnd, i, ref[i], new[i])
    _lib.check(lib.lbm_destroy(h))
    ok(rt.cudaStreamDestroy(stream), "cudaStreamDestroy")
    for p in bufs.values():
        ok(rt.cudaFree(p), "cudaFree")
    if rnd == 0:
        ok(rt.cudaDeviceReset(), "cudaDeviceReset")
print("noalloc-after-reset ok")
"""


def test_reduce_noalloc_after_device_reset():
    """A caller that resets its device (cudaDeviceReset ends its context and
    every allocation in it) and then binds fresh buffers still gets
    lbm_reduce's values from lbm_reduce_noalloc: the static array's device
    address is looked up on each call, not kept from before the reset.  Runs in
    a child process that allocates with the CUDA runtime directly (no torch, so
    no allocator holds memory across the reset)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _RESET_CHILD, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "noalloc-after-reset ok" in r.stdout
