"""The GPU adjoint (reverse-mode derivative of the D3Q19 step behind a
torch.autograd.Function with sqrt(T) checkpointing) against the FP64 CPU
oracle's adjoint and against central finite differences of the GPU forward."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1803_04937_gb300 import inputs
from tests._helpers import oracle_config, random_fields, rel_maxnorm

pytestmark = pytest.mark.gpu

CASES = [
    dict(equilibrium="improved", collision="srt", tau=0.7),
    dict(equilibrium="standard", collision="srt", tau=0.9, force=(1e-4, -5e-5, 0.0)),
    dict(equilibrium="improved", collision="trt", tau=0.62, force=(2e-4, 0.0, 1e-4), walls=(False, True, False)),
    dict(equilibrium="standard", collision="trt", tau=0.8, walls=(True, False, True)),
]


def _gpu_grad(shape, rho, u0, tgt, steps, precision, case, every=None):
    from paper_1803_04937_gb300 import adjoint
    nz, ny, nx = shape
    dt = torch.float64 if precision == "f64" else torch.float32
    u = u0.to("cuda", dt).clone().requires_grad_(True)
    tau = torch.tensor(case["tau"], dtype=torch.float64, requires_grad=True)
    kw = {k: v for k, v in case.items() if k != "tau"}
    r, uT = adjoint.simulate(u, tau, steps, nx, ny, nz, rho=rho.to("cuda", dt), precision=precision,
                             checkpoint_every=every, **kw)
    L = 0.5 * ((uT.double() - tgt.to("cuda")) ** 2).sum()
    L.backward()
    return L.item(), u.grad.double().cpu().numpy(), tau.grad.item()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-4)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_adjoint_matches_oracle_adjoint(case, precision, tol):
    kw = CASES[case]
    shape = (5, 7, 12)
    rho, u0 = random_fields(shape, seed=40 + case, amp=0.04)
    _, tgt = random_fields(shape, seed=80 + case, amp=0.04)
    steps = 10
    L, gu, gt = _gpu_grad(shape, rho, u0, tgt, steps, precision, kw, every=3)
    cfg = oracle_config(shape[2], shape[1], shape[0], **kw)
    Lo, guo, gto = oracle.gradient_velocity_l2(cfg, rho.numpy(), u0.numpy(), tgt.numpy(), steps)
    assert L == pytest.approx(Lo, rel=max(tol, 1e-12))
    assert rel_maxnorm(gu, guo) < tol
    assert gt == pytest.approx(gto, rel=tol)


def test_checkpoint_interval_does_not_change_the_gradient():
    kw = CASES[2]
    shape = (4, 6, 10)
    rho, u0 = random_fields(shape, seed=5, amp=0.04)
    _, tgt = random_fields(shape, seed=6, amp=0.04)
    ref = _gpu_grad(shape, rho, u0, tgt, 13, "f64", kw, every=1)
    for every in (2, 5, 13, 20):
        g = _gpu_grad(shape, rho, u0, tgt, 13, "f64", kw, every=every)
        assert np.array_equal(g[1], ref[1]) and g[2] == ref[2]


def test_adjoint_16cube_against_cpu_adjoint():
    """The 16^3 copy of the adjoint workload (same recipe, |n| <= 7 so 16^3
    resolves it), T = 400: GPU FP64 adjoint to 1e-10, FP32 adjoint to 1e-3."""
    n, steps = 16, 400
    rho, u0 = inputs.random_solenoidal(n, n, n, kmax=7, u_rms=0.02, seed=1)
    _, tgt = inputs.random_solenoidal(n, n, n, kmax=7, u_rms=0.02, seed=2)
    case = dict(equilibrium="improved", collision="srt", tau=0.7)
    cfg = oracle_config(n, n, n, **case)
    Lo, guo, gto = oracle.gradient_velocity_l2(cfg, rho.numpy(), u0.numpy(), tgt.numpy(), steps)
    for precision, tol in (("f64", 1e-10), ("f32", 1e-3)):
        L, gu, gt = _gpu_grad((n, n, n), rho, u0, tgt, steps, precision, case)
        assert rel_maxnorm(gu, guo) < tol, precision
        assert gt == pytest.approx(gto, rel=tol), precision


def test_adjoint_128cube_against_finite_differences():
    """Adjoint workload: periodic 128^3, tau = 0.7, D3Q19-I, SRT, T = 400 with
    sqrt(T) checkpoints, random solenoidal u0 (|n| <= 8, u_rms = 0.02, seed 1),
    target seed 2.  FP32 adjoint vs central differences of the FP64 GPU forward
    on 64 random components of u0 (seed 3) and on tau: <= 1e-3 relative."""
    from paper_1803_04937_gb300 import adjoint
    n, steps = 128, 400
    case = dict(equilibrium="improved", collision="srt", tau=0.7)
    rho, u0 = inputs.random_solenoidal(n, n, n, kmax=8, u_rms=0.02, seed=1, device="cuda")
    _, tgt = inputs.random_solenoidal(n, n, n, kmax=8, u_rms=0.02, seed=2, device="cuda")
    u = u0.float().clone().requires_grad_(True)
    tau = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    _, uT = adjoint.simulate(u, tau, steps, n, n, n, precision="f32", equilibrium="improved", collision="srt")
    L = 0.5 * ((uT.double() - tgt) ** 2).sum()
    L.backward()
    g = u.grad.double()

    def loss(uu, t):
        _, ue = adjoint.forward_only(uu, t, steps, n, n, n, precision="f64", equilibrium="improved",
                                     collision="srt")
        return float(0.5 * ((ue - tgt) ** 2).sum())

    rng = np.random.default_rng(3)
    idx = [tuple(int(rng.integers(0, s)) for s in (3, n, n, n)) for _ in range(64)]
    h = 1e-5
    fd, ad = [], []
    for i in idx:
        up = u0.clone()
        um = u0.clone()
        up[i] += h
        um[i] -= h
        fd.append((loss(up, 0.7) - loss(um, 0.7)) / (2 * h))
        ad.append(float(g[i]))
    fd, ad = np.array(fd), np.array(ad)
    err = np.abs(fd - ad).max() / np.abs(fd).max()
    print("dL/du0: 64-component max-norm relative error vs FD = %.3e" % err)
    assert err < 1e-3
    ht = 1e-6
    fdt = (loss(u0, 0.7 + ht) - loss(u0, 0.7 - ht)) / (2 * ht)
    print("dL/dtau: adjoint %.9e, FD %.9e" % (float(tau.grad), fdt))
    assert float(tau.grad) == pytest.approx(fdt, rel=1e-3)


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("shape,walls", [((33, 40, 130), (False, False, False)), ((130, 128, 64), (False, False, False)),
                                         ((9, 14, 40), (False, True, True))])
def test_deferred_adjoint_sums_are_bitwise_the_immediate_ones(shape, walls, precision):
    """LBM_OPT_ADJ_DEFER_SUM: each step's dL/domega partials summed by the next
    step's first block (256 threads) or by lbm_adjoint_flush give bitwise the
    sums of the one-block kernel (1024 threads) after every step, and the same
    lambdas; lbm_reduce flushes a pending sum first.  The lattices give 1320
    and 8320 block partials (one and two passes of the 1024-thread loop) and a
    walled one."""
    import ctypes

    from paper_1803_04937_gb300 import _lib
    from paper_1803_04937_gb300.lbm import Simulation
    nz, ny, nx = shape
    dt = torch.float64 if precision == "f64" else torch.float32
    rho, u = random_fields(shape, seed=61)
    gen = torch.Generator().manual_seed(62)
    lam0 = (torch.rand((19,) + tuple(shape), generator=gen, dtype=torch.float64) - 0.5).to("cuda", dt)
    steps = 5
    out = {}
    for defer in (0, 1):
        sim = Simulation(nx, ny, nz, precision=precision, equilibrium="improved", collision="trt", tau=0.6,
                         walls=walls, force=(1e-4, 0.0, -5e-5))
        sim.init(rho.cuda(), u.cuda())
        lib, h = sim._lib, sim.handle
        _lib.check(lib.lbm_set_option(h, _lib.OPT_ADJ_DEFER_SUM, float(defer)), h)
        lam = [lam0.clone(), torch.empty_like(lam0)]
        gws = [torch.zeros(2, dtype=torch.float64, device="cuda") for _ in range(steps)]
        state = ctypes.c_void_p(sim.grids[0].data_ptr())
        for i in range(steps):
            # every step adds to its own accumulator, so each step's sum is checked
            _lib.check(lib.lbm_adjoint_step(h, state, ctypes.c_void_p(lam[i % 2].data_ptr()),
                                            ctypes.c_void_p(lam[1 - i % 2].data_ptr()),
                                            ctypes.cast(ctypes.c_void_p(gws[i].data_ptr()),
                                                        ctypes.POINTER(ctypes.c_double))), h)
            if i == 2:
                sim.reduce()  # flushes the pending sum of step 2
                torch.cuda.synchronize()
                assert gws[2].abs().sum().item() > 0
        _lib.check(lib.lbm_adjoint_flush(h), h)
        torch.cuda.synchronize()
        out[defer] = (torch.stack(gws).cpu(), lam[steps % 2].cpu())
        sim.close()
    print("deferred adjoint sums %s %s: %s" % (precision, shape, out[1][0][:, 0].tolist()))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert (out[0][0] != 0).all()
