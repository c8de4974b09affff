"""lbm_init and lbm_moments on pinned host buffers: the kernels read and write
the host memory directly through its mapped device address.  The results are
bitwise those of the same calls on device buffers; pageable host memory is
refused before any launch."""
import ctypes

import pytest
import torch

from paper_1803_04937_gb300 import _lib
from tests._helpers import random_fields

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
def test_host_buffers_match_device_buffers(precision):
    from paper_1803_04937_gb300.lbm import Simulation
    shape = (5, 9, 37)
    rho, u = random_fields(shape, seed=41)
    dt = torch.float64 if precision == "f64" else torch.float32
    rho, u = rho.to(dt), u.to(dt)
    kw = dict(equilibrium="improved", collision="trt", tau=0.7, precision=precision, force=(1e-5, 0, 0))
    dev = Simulation(37, 9, 5, **kw)
    dev.init(rho.cuda(), u.cuda())
    dev.step(5)
    r_d, u_d = dev.moments(dt)
    host = Simulation(37, 9, 5, **kw)
    out = host.run_host(rho.pin_memory(), u.pin_memory(), 5)
    assert torch.equal(host.get_pdfs(), dev.get_pdfs())
    assert torch.equal(out[0], r_d.cpu()) and torch.equal(out[1], u_d.cpu())
    # rho = NULL (uniform 1) also works from host memory
    one = Simulation(37, 9, 5, **kw)
    one.run_host(None, u.pin_memory(), 2)
    ref = Simulation(37, 9, 5, **kw)
    ref.init(None, u.cuda())
    ref.step(2)
    assert torch.equal(one.get_pdfs(), ref.get_pdfs())


def test_pageable_host_buffers_are_refused():
    from paper_1803_04937_gb300.lbm import Simulation
    lib = _lib.load()
    sim = Simulation(8, 4, 4, precision="f32")
    u = torch.zeros((3, 4, 4, 8), dtype=torch.float32)  # pageable
    assert not u.is_pinned()
    s = lib.lbm_init(sim.handle, None, ctypes.c_void_p(u.data_ptr()), _lib.DTYPE_F32)
    assert s == _lib.LBM_EINVAL
    assert "pageable" in lib.lbm_last_error(sim.handle).decode()
    sim.init(None, u.cuda())
    s = lib.lbm_moments(sim.handle, None, ctypes.c_void_p(u.data_ptr()), _lib.DTYPE_F32)
    assert s == _lib.LBM_EINVAL
    with pytest.raises(ValueError):
        sim.run_host(None, u, 1)
    torch.cuda.synchronize()
