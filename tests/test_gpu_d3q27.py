"""The D3Q27 comparison lattice on the GPU (Sec. 2.3; standard equilibrium,
which the construction of Sec. 3.1 gives on D3Q27): parity with the FP64
oracle's D3Q27 step, the paper's duct result for D3Q27 (no transverse
currents, Sec. 5.1), and unsupported calls failing cleanly."""
import math

import numpy as np
import pytest
import torch

import oracle
from tests._helpers import gpu_pdfs_in_oracle_layout, oracle_config, random_fields, rel_maxnorm

pytestmark = pytest.mark.gpu

CASES = [
    dict(collision="srt", tau=0.8),
    dict(collision="trt", tau=0.6, force=(2e-4, -1e-4, 5e-5)),
    dict(collision="srt", tau=0.7, walls=(True, False, True), force=(1e-4, 0, 0)),
    dict(collision="trt", tau=0.9, walls=(True, True, True)),
    dict(collision="srt", tau=1.2, rho0_is_rho=True, force=(1e-4, 2e-4, 0)),
]


@pytest.mark.parametrize("precision,tol,pdf_tol", [("f64", 1e-12, 1e-13), ("f32", 1e-5, 1e-6)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_d3q27_step_matches_oracle(case, precision, tol, pdf_tol):
    from paper_1803_04937_gb300.lbm import Simulation
    kw = CASES[case]
    shape = (5, 9, 37)
    rho, u = random_fields(shape, seed=300 + case)
    sim = Simulation(37, 9, 5, precision=precision, stencil=27, equilibrium="standard", **kw)
    sim.init(rho.cuda(), u.cuda())
    sim.step(6)
    r_g, u_g = (t.cpu().numpy() for t in sim.moments())
    cfg = oracle_config(37, 9, 5, stencil=27, equilibrium="standard", **kw)
    f_o = oracle.step(cfg, oracle.init(cfg, rho.numpy(), u.numpy()), 6)
    r_o, u_o = oracle.moments(cfg, f_o)
    assert rel_maxnorm(u_g, u_o) < tol
    assert np.abs(r_g - r_o).max() < tol
    assert np.abs(gpu_pdfs_in_oracle_layout(sim) - f_o).max() < pdf_tol


@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("shape", [(3, 7, 4), (4, 9, 40), (3, 5, 388), (2, 3, 1040)])
def test_d3q27_four_cells_is_bitwise(shape, case, precision):
    """16-bit D3Q27 storage with nx % 4 == 0 runs four cells per thread; the
    results equal the one-cell kernel bit for bit (ragged warps, row ends,
    several blocks per row, walls on every axis)."""
    from paper_1803_04937_gb300.lbm import Simulation
    kw = CASES[case]
    rho, u = random_fields(shape, seed=43)
    nz, ny, nx = shape
    out = []
    for cells_x in (4, 1):
        sim = Simulation(nx, ny, nz, precision=precision, stencil=27, equilibrium="standard", cells_x=cells_x, **kw)
        sim.init(rho.cuda(), u.float().cuda())
        sim.step(5)
        out.append(sim.get_pdfs())
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
@pytest.mark.parametrize("walls", [(False, True, False), (False, False, True), (False, True, True), (True, False, False),
                                   (True, True, True)])
@pytest.mark.parametrize("shape", [(5, 7, 40), (1, 2, 388), (2, 1, 64), (2, 2, 8), (3, 2, 4), (6, 3, 1040)])
def test_d3q27_four_cell_split_rows_is_bitwise(shape, walls, precision):
    """On a walled lattice the four-cell D3Q27 step runs its interior rows
    through the periodic kernel (with walls on x, the kernel with the x-wall
    selects only) and the wall rows through the walled one (split_rows); the
    result is bitwise that of the one-cell kernel, also on lattices of one or
    two rows or planes (no interior)."""
    from paper_1803_04937_gb300.lbm import Simulation
    kw = dict(collision="trt", tau=0.6, walls=walls, force=(1e-4, -2e-4, 1e-4))
    rho, u = random_fields(shape, seed=47)
    nz, ny, nx = shape
    out = []
    for cells_x in (4, 1):
        sim = Simulation(nx, ny, nz, precision=precision, stencil=27, equilibrium="standard", cells_x=cells_x, **kw)
        sim.init(rho.cuda(), u.float().cuda())
        sim.step(5)
        out.append(sim.get_pdfs())
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("precision,tol", [("f16s", 2e-3), ("bf16s", 2e-2)])
def test_d3q27_16bit_storage_error(precision, tol):
    from paper_1803_04937_gb300.lbm import Simulation
    kw = CASES[1]
    shape = (6, 10, 64)
    rho, u = random_fields(shape, seed=17)
    sim = Simulation(64, 10, 6, precision=precision, stencil=27, equilibrium="standard", **kw)
    sim.init(rho.cuda(), u.float().cuda())
    sim.step(20)
    _, ug = sim.moments()
    cfg = oracle_config(64, 10, 6, stencil=27, equilibrium="standard", **kw)
    _, uo = oracle.run(cfg, rho.numpy(), u.numpy(), 20)
    err = rel_maxnorm(ug.cpu().numpy(), uo)
    print("D3Q27 %s: velocity error after 20 steps %.2e" % (precision, err))
    assert err < tol


def test_d3q27_duct_has_no_spurious_currents():
    from paper_1803_04937_gb300 import inputs
    from paper_1803_04937_gb300.lbm import Simulation
    D, tau = 24, 1.0
    nu = (tau - 0.5) / 3
    a = 10 * nu * nu / (0.2947 * D * (D / 2) ** 2)
    sim = Simulation(2, D, D, precision="f64", stencil=27, equilibrium="standard", tau=tau, force=(a, 0, 0),
                     walls=(False, True, True))
    rho, u = inputs.rest(2, D, D, device="cuda")
    sim.init(rho, u)
    sim.step(int(8 * D * D / (math.pi ** 2 * nu)) + 500)
    _, ug = sim.moments()
    ratio = float(ug[1:].abs().max() / ug[0].abs().max())
    print("duct D=%d D3Q27: max|u_yz|/max|u_x| = %.3e" % (D, ratio))
    assert ratio < 1e-13


def test_d3q27_uniform_flow_keeps_momentum_in_fp32():
    from paper_1803_04937_gb300.lbm import Simulation
    n = 16
    u = torch.zeros((3, n, n, n), dtype=torch.float64)
    u[0], u[1], u[2] = 0.1, -0.05, 0.02
    sim = Simulation(n, n, n, precision="f32", stencil=27, collision="srt", tau=0.55)
    sim.init(None, u.cuda())
    sim.step(2000)
    _, ug = sim.moments()
    err = float((ug.cpu() - u).abs().max() / 0.1)
    print("D3Q27 uniform flow FP32, 2000 steps: %.2e" % err)
    assert err < 2e-6


def test_d3q27_unsupported_calls_fail_cleanly():
    from paper_1803_04937_gb300 import _lib
    from paper_1803_04937_gb300.lbm import Simulation
    sim = Simulation(8, 8, 8, stencil=27)
    sim.init(None, torch.zeros((3, 8, 8, 8), dtype=torch.float64, device="cuda"))
    with pytest.raises(_lib.LBMError) as e:
        sim.reduce()
    assert e.value.status == _lib.LBM_EUNSUPPORTED
    with pytest.raises(_lib.LBMError):
        Simulation(8, 8, 8, stencil=27, pattern="aa")


def test_d3q27_channel_fp32_long_run():
    """D3Q27, FP32: the walled channel of the benchmark workload (walls at
    y = -1/2 and 255.5, TRT 3/16, tau = 0.6, body force for a centreline speed
    of 0.05) on a thin 8x256x4 lattice, 5000 steps from rest: every (x, z)
    column is bitwise equal and matches the FP64 oracle's D3Q27 1x256x1 column
    to 1e-5.  This flow changes slowly, so without the compensated momentum sum
    the FP32 rounding of u fed back through the relaxation every step would add
    up coherently."""
    from paper_1803_04937_gb300 import inputs
    from paper_1803_04937_gb300.lbm import Simulation
    nx, ny, nz, steps, tau = 8, 256, 4, 5000, 0.6
    nu = (tau - 0.5) / 3
    a = 8 * nu * 0.05 / ny ** 2
    kw = dict(equilibrium="standard", collision="trt", tau=tau, force=(a, 0, 0), walls=(False, True, False))
    sim = Simulation(nx, ny, nz, precision="f32", stencil=27, **kw)
    rho, u = inputs.rest(nx, ny, nz, device="cuda")
    sim.init(rho, u.float())
    sim.step(steps)
    _, ug = sim.moments(torch.float32)
    ref = ug[:, 0:1, :, 0:1]
    assert torch.equal(ug, ref.expand_as(ug)), "columns differ"
    prof = ref[:, 0, :, 0].double().cpu().numpy()
    sim.close()
    cfg = oracle_config(1, ny, 1, stencil=27, **kw)
    r1, u1 = inputs.rest(1, ny, 1)
    _, uo = oracle.run(cfg, r1.numpy(), u1.numpy(), steps)
    err = rel_maxnorm(prof[0], uo[0, 0, :, 0])
    print("D3Q27 channel FP32, 5000 steps: u_x profile max-norm rel err vs FP64 oracle %.3e" % err)
    assert err < 1e-5
