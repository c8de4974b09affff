"""The MRT collision (Sec. 3.2-3.3: monomial moments, Maxwellian equilibrium
moments) on the GPU: parity with the FP64 oracle element by element on small
seeded lattices with a ragged tail, 16-bit storage error, A/B vs AA bitwise,
the TRT limit, the shear-wave workload at 256^3 against an exact oracle column,
the duct flow's spurious currents, and the refusals of the adjoint and of
D3Q27."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1803_04937_gb300 import inputs
from tests._helpers import gpu_pdfs_in_oracle_layout, oracle_config, random_fields, rel_maxnorm

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
PDF_TOL = {"f64": 1e-13, "f32": 1e-6}

CASES = [
    dict(equilibrium="improved", collision="mrt", tau=0.8, omega_bulk=1.0, omega_4=1.0),
    dict(equilibrium="standard", collision="mrt", tau=0.6, omega_bulk=1.3, omega_4=0.8, force=(2e-4, -1e-4, 5e-5)),
    dict(equilibrium="improved", collision="mrt", tau=0.55, omega_bulk=1.5, omega_4=1.2, trt_magic=0.25,
         walls=(False, True, False), force=(1e-4, 0, 0)),
    dict(equilibrium="improved", collision="mrt", tau=0.9, omega_bulk=0.9, omega_4=1.6, walls=(True, True, True)),
    dict(equilibrium="standard", collision="mrt", tau=1.2, omega_bulk=1.1, omega_4=0.7, rho0_is_rho=True,
         walls=(True, False, False), force=(1e-4, 2e-4, 0)),
    dict(equilibrium="improved", collision="mrt", tau=0.7, omega_bulk=1.4, omega_4=0.9, rho0_is_rho=True,
         walls=(False, False, True), force=(0, -1e-4, 1e-4)),
]


def _sim(nx, ny, nz, **kw):
    from paper_1803_04937_gb300.lbm import Simulation
    return Simulation(nx, ny, nz, **kw)


def _run_gpu(shape, rho, u, steps, precision, pattern, case):
    nz, ny, nx = shape
    sim = _sim(nx, ny, nz, precision=precision, pattern=pattern, **case)
    sim.init(rho.cuda(), u.cuda())
    sim.step(steps)
    r, uu = sim.moments(torch.float64)
    return sim, r.cpu().numpy(), uu.cpu().numpy()


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("nx", [37, 130])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_mrt_step_matches_oracle(case, nx, pattern, precision):
    kw = CASES[case]
    shape = (5, 9, nx)
    rho, u = random_fields(shape, seed=300 + case)
    steps = 7 if pattern == "aa" else 6
    sim, r_g, u_g = _run_gpu(shape, rho, u, steps, precision, pattern, kw)
    cfg = oracle_config(shape[2], shape[1], shape[0], **kw)
    f_o = oracle.step(cfg, oracle.init(cfg, rho.numpy(), u.numpy()), steps)
    r_o, u_o = oracle.moments(cfg, f_o)
    assert rel_maxnorm(u_g, u_o) < TOL[precision]
    assert np.abs(r_g - r_o).max() < TOL[precision]
    assert np.abs(gpu_pdfs_in_oracle_layout(sim) - f_o).max() < PDF_TOL[precision]


@pytest.mark.parametrize("precision,tol", [("f16s", 2e-3), ("bf16s", 2e-2)])
@pytest.mark.parametrize("case", [0, 2])
def test_mrt_16bit_storage_error(case, precision, tol):
    kw = CASES[case]
    shape = (6, 10, 64)
    rho, u = random_fields(shape, seed=17)
    _, _, u_g = _run_gpu(shape, rho, u, 20, precision, "ab", kw)
    cfg = oracle_config(shape[2], shape[1], shape[0], **kw)
    _, u_o = oracle.run(cfg, rho.numpy(), u.numpy(), 20)
    err = rel_maxnorm(u_g, u_o)
    print("MRT %s case %d: velocity error after 20 steps %.2e" % (precision, case, err))
    assert err < tol


@pytest.mark.parametrize("precision", ["f32", "f16s", "f64"])
@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
def test_mrt_aa_equals_ab_bitwise(case, precision):
    """AA and A/B run the same MRT arithmetic per cell: identical bits, also
    with the walled AA odd step split into interior and wall rows (walls on y,
    on z, on x only, and on all axes)."""
    kw = CASES[case]
    shape = (6, 11, 45)
    rho, u = random_fields(shape, seed=5)
    for steps in (1, 4, 9):
        sa, _, _ = _run_gpu(shape, rho, u, steps, precision, "ab", kw)
        sb, _, _ = _run_gpu(shape, rho, u, steps, precision, "aa", kw)
        assert torch.equal(sa.get_pdfs(), sb.get_pdfs())


@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("case", [0, 2, 3, 4])
@pytest.mark.parametrize("shape", [(3, 7, 4), (4, 9, 40), (3, 8, 64), (2, 6, 256), (3, 5, 388), (2, 3, 600),
                                   (1, 2, 1000), (2, 3, 1040)])
def test_mrt_four_cells_is_bitwise(shape, case, pattern, precision):
    """16-bit storage with nx % 4 == 0 runs MRT in the four-cell kernels (A/B
    and AA); they equal the one-cell MRT kernel bit for bit (ragged warps,
    row-end and multi-block rows, blocks of 32 x 4, 64 x 2 and 128 x 1
    threads, walls on every axis)."""
    from paper_1803_04937_gb300.lbm import Simulation
    kw = CASES[case]
    rho, u = random_fields(shape, seed=41)
    nz, ny, nx = shape
    out = []
    for cells_x, pat in ((4, pattern), (1, "ab")):
        sim = Simulation(nx, ny, nz, precision=precision, pattern=pat, cells_x=cells_x, **kw)
        sim.init(rho.cuda(), u.float().cuda())
        sim.step(5)
        out.append(sim.get_pdfs())
    assert torch.equal(out[0], out[1])


def test_mrt_with_equal_even_rates_is_trt():
    """omega_bulk = omega_4 = 1/tau: the MRT kernel reproduces the TRT kernel
    to rounding."""
    tau = 0.7
    shape = (5, 8, 40)
    rho, u = random_fields(shape, seed=21)
    base = dict(equilibrium="improved", tau=tau, force=(1e-4, 0, -1e-4), walls=(False, True, False))
    sm, _, um = _run_gpu(shape, rho, u, 10, "f64", "ab", dict(base, collision="mrt", omega_bulk=1 / tau,
                                                                  omega_4=1 / tau))
    st, _, ut = _run_gpu(shape, rho, u, 10, "f64", "ab", dict(base, collision="trt"))
    assert np.abs(sm.get_pdfs().cpu().numpy() - st.get_pdfs().cpu().numpy()).max() < 1e-15
    assert rel_maxnorm(um, ut) < 1e-13


def test_mrt_shear_wave_256_fp32():
    """Periodic 256^3, FP32, u = (0.1, 0.01 sin(2 pi x/256), 0), tau = 0.8,
    omega_bulk = 1.2, omega_4 = 1.0, 1000 steps: every (y,z) column is bitwise
    equal and matches the FP64 oracle's 256x1x1 run (an exact sample) within
    the 1e-5 FP32 target."""
    n, steps = 256, 1000
    kw = dict(equilibrium="improved", collision="mrt", tau=0.8, omega_bulk=1.2, omega_4=1.0)
    rho, u = inputs.shear_wave(n, n, n, U=(0.1, 0, 0), amplitude=0.01, device="cuda")
    sim = _sim(n, n, n, precision="f32", **kw)
    sim.init(rho, u.float())
    del rho, u
    sim.step(steps)
    _, ug = sim.moments(torch.float32)
    col = ug[:, 0:1, 0:1, :]
    assert torch.equal(ug, col.expand_as(ug)), "columns differ"
    col = col[:, 0, 0, :].double().cpu().numpy()
    del ug
    sim.close()
    cfg = oracle_config(n, 1, 1, **kw)
    r1, u1 = inputs.shear_wave(n, 1, 1, U=(0.1, 0, 0), amplitude=0.01)
    _, uo = oracle.run(cfg, r1.numpy(), u1.numpy(), steps)
    err = rel_maxnorm(col, uo[:, 0, 0, :])
    print("MRT shear wave 256^3 FP32, 1000 steps: max-norm rel err vs FP64 oracle %.2e" % err)
    assert err < 1e-5


def _duct(D, tau, equilibrium, omega_bulk, omega_4, Re=10.0):
    nu = (tau - 0.5) / 3
    a = Re * nu * nu / (0.2947 * D * (D / 2) ** 2)
    nsteps = int(8 * D * D / (math.pi ** 2 * nu)) + 500
    sim = _sim(2, D, D, precision="f64", equilibrium=equilibrium, collision="mrt", tau=tau, force=(a, 0, 0),
               walls=(False, True, True), omega_bulk=omega_bulk, omega_4=omega_4)
    rho, u = inputs.rest(2, D, D, device="cuda")
    sim.init(rho, u)
    sim.step(nsteps)
    _, ug = sim.moments()
    return float(ug[1:].abs().max() / ug[0].abs().max())


def test_mrt_duct_spurious_currents():
    """Square duct (Sec. 5.1) with MRT at tau = 0.8, Re = 10.  With the
    Maxwellian moments (D3Q19-I) the transverse velocity stays at rounding level
    whenever the bulk rate equals omega+, for any fourth-order rate; a bulk rate
    different from omega+ lets the second-order moments' trace respond to the
    flow and brings small transverse currents that vanish under refinement
    faster than those of D3Q19-S."""
    tau = 0.8
    wp = 1 / tau
    rows = {}
    for D in (12, 24):
        rows[D] = dict(S=_duct(D, tau, "standard", wp, 1.0), I_eq=_duct(D, tau, "improved", wp, 1.0),
                       I_eq4=_duct(D, tau, "improved", wp, 1.6), I_bulk=_duct(D, tau, "improved", 1.0, 1.0))
        print("MRT duct D=%d: S %.3e  I(bulk=omega+, omega_4=1) %.3e  I(bulk=omega+, omega_4=1.6) %.3e  "
              "I(bulk=1) %.3e" % (D, rows[D]["S"], rows[D]["I_eq"], rows[D]["I_eq4"], rows[D]["I_bulk"]))
    for D in (12, 24):
        assert rows[D]["I_eq"] < 1e-13 and rows[D]["I_eq4"] < 1e-13
        assert rows[D]["S"] > 1e-6
        assert 1e-9 < rows[D]["I_bulk"] < rows[D]["S"]
    order_s = math.log2(rows[12]["S"] / rows[24]["S"])
    order_b = math.log2(rows[12]["I_bulk"] / rows[24]["I_bulk"])
    print("MRT duct convergence orders 12 -> 24: S %.2f, I(bulk=1) %.2f" % (order_s, order_b))
    assert order_b > order_s


def test_mrt_adjoint_is_refused():
    """The adjoint covers SRT and TRT; the backward pass of an MRT run fails loudly."""
    from paper_1803_04937_gb300 import _lib, adjoint
    n = 8
    rho = torch.ones(n, n, n, dtype=torch.float64, device="cuda")
    u0 = torch.zeros(3, n, n, n, dtype=torch.float64, device="cuda", requires_grad=True)
    _, u = adjoint.simulate(u0, 0.7, 2, n, n, n, rho=rho, collision="mrt", precision="f64")
    with pytest.raises(_lib.LBMError):
        u.sum().backward()
