"""The D3Q19 workloads at their full sizes, checked against the FP64 oracle on
sampled outputs it can compute (a y,z- or x,z-invariant flow is one oracle
column) and against properties that hold at any size.  Each test prints the
measured errors."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1803_04937_gb300 import inputs
from tests._helpers import oracle_config, oracle_run_fp32_storage, rel_maxnorm

pytestmark = pytest.mark.gpu


def _sim(nx, ny, nz, **kw):
    from paper_1803_04937_gb300.lbm import Simulation
    return Simulation(nx, ny, nz, **kw)


# ------------------------------------------------------------------ Taylor-Green 32^3, FP64

@pytest.mark.parametrize("equilibrium", ["standard", "improved"])
def test_taylor_green_32_fp64(equilibrium):
    """Periodic 32^3, FP64, TGV u0 = 0.05, tau = 0.8, 100 steps: velocity field
    and energy series vs the oracle (<= 1e-12), decay rate vs 2 nu |k|^2."""
    n, steps = 32, 100
    rho, u = inputs.taylor_green(n, u0=0.05)
    kw = dict(equilibrium=equilibrium, collision="srt", tau=0.8)
    sim = _sim(n, n, n, precision="f64", **kw)
    sim.init(rho.cuda(), u.cuda())
    cfg = oracle_config(n, n, n, **kw)
    f = oracle.init(cfg, rho.numpy(), u.numpy())
    e_gpu, e_or = [sim.reduce()["energy"]], []
    e_or.append(0.5 * (oracle.moments(cfg, f)[1] ** 2).sum())
    for _ in range(steps // 10):
        sim.step(10)
        f = oracle.step(cfg, f, 10)
        e_gpu.append(sim.reduce()["energy"])
        e_or.append(0.5 * (oracle.moments(cfg, f)[1] ** 2).sum())
    _, ug = sim.moments()
    _, uo = oracle.moments(cfg, f)
    err = rel_maxnorm(ug.cpu().numpy(), uo)
    e_err = max(abs(a - b) / b for a, b in zip(e_gpu, e_or))
    nu, k2 = (0.8 - 0.5) / 3, 3 * (2 * math.pi / n) ** 2
    rate = -np.polyfit(np.arange(len(e_gpu)) * 10.0, np.log(e_gpu), 1)[0]
    print("TGV32 %s: |u-u_oracle|/|u| = %.2e, energy rel err = %.2e, decay rate %.6f vs 2 nu k^2 = %.6f (%.2f%%)"
          % (equilibrium, err, e_err, rate, 2 * nu * k2, 100 * (rate / (2 * nu * k2) - 1)))
    assert err < 1e-12 and e_err < 1e-12
    assert abs(rate / (2 * nu * k2) - 1) < 0.03


# ------------------------------------------------------------------ shear wave 256^3, FP32

def _shear_amp_phase(uy, n):
    k = 2 * math.pi / n
    c = (uy * np.exp(-1j * k * np.arange(n))).sum() * 2 / n
    return abs(c), np.angle(c)


# FP32 runs against the FP64 oracle: the equilibrium's first moment is exact in
# FP32, every population is updated with a single rounding at its own scale,
# and the momentum is summed with compensation so that rounding the velocity
# does not feed a momentum error back through the relaxation (lbm_device.cuh).
# What remains is the rounding of the stored populations: the shear waves stay
# within about 1.5e-6 of max|u| after 2000 steps and the channel (5000 steps
# from rest) within about 1e-6; both are asserted at the 1e-5 FP32 target.
FP32_LONG_TOL = 1e-5


@pytest.mark.parametrize("collision", ["srt", "trt"])
def test_shear_wave_256_fp32(collision):
    """Periodic 256^3, FP32, u = (U, 0.01 sin(2 pi x/256), 0), U in {0, 0.05, 0.1},
    tau in {0.55, 0.8}, 2000 steps, S and I: every (y,z) column is bitwise equal,
    the column matches the FP64 oracle's 256x1x1 run, and S and I agree to
    rounding (the flow is z-invariant with u_z = 0).  Prints the oracle error and
    the decay-rate and phase errors against nu k^2 and U."""
    n, steps = 256, 2000
    k = 2 * math.pi / n
    rows = []
    for U in (0.0, 0.05, 0.1):
        for tau in (0.55, 0.8):
            cols = {}
            for equilibrium in ("standard", "improved"):
                kw = dict(equilibrium=equilibrium, collision=collision, tau=tau)
                rho, u = inputs.shear_wave(n, n, n, U=(U, 0, 0), amplitude=0.01, device="cuda")
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
                r1, u1 = inputs.shear_wave(n, 1, 1, U=(U, 0, 0), amplitude=0.01)
                _, uo = oracle.run(cfg, r1.numpy(), u1.numpy(), steps)
                uo = uo[:, 0, 0, :]
                err = rel_maxnorm(col, uo)
                amp, ph = _shear_amp_phase(col[1], n)
                nu = (tau - 0.5) / 3
                rate_err = (math.log(0.01 / amp) / steps) / (nu * k * k) - 1
                # u_y = A sin(k (x - U t)): Fourier coefficient -i A exp(-i k U t)
                ph_err = (ph + math.pi / 2 + k * U * steps + math.pi) % (2 * math.pi) - math.pi
                cols[equilibrium] = col
                rows.append((U, tau, equilibrium, err, rate_err, ph_err))
            d = np.abs(cols["standard"] - cols["improved"]).max() / np.abs(cols["improved"]).max()
            rows.append((U, tau, "S-I", d, float("nan"), float("nan")))
    for U, tau, eq, err, re, pe in rows:
        print("shear256 %s U=%.2f tau=%.2f %-8s oracle err %.2e  decay-rate err %+.3e  phase err %+.3e rad"
              % (collision, U, tau, eq, err, re, pe))
    assert max(r[3] for r in rows) < FP32_LONG_TOL


@pytest.mark.parametrize("precision", ["f16s", "bf16s"])
def test_shear_wave_256_16bit(precision):
    """The shear-wave workload (periodic 256^3, 2000 steps, SRT, tau = 0.8) with
    16-bit shifted storage: velocity-field error against the FP64 oracle column,
    decay-rate and phase errors against nu k^2 and U (stated, as the FP32 test
    does), for U in {0, 0.1} and both equilibria.  Measured: the viscous change
    of the shifted populations per step (about 1e-7) is below their 16-bit
    spacing (about 1e-6 for FP16), so with round-to-nearest storage the wave does
    not decay at U = 0 (decay-rate error -100 %, u_y error 13 %); with U = 0.1
    FP16 stays within 2 % of the oracle in u and 10-16 % in u_y, BF16 loses the
    wave.  The test asserts the exact column structure, finiteness and the
    FP16/BF16 error levels measured, as a guard against regressions."""
    n, steps, tau = 256, 2000, 0.8
    k = 2 * math.pi / n
    nu = (tau - 0.5) / 3
    worst = 0.0
    for U in (0.0, 0.1):
        for equilibrium in ("standard", "improved"):
            kw = dict(equilibrium=equilibrium, collision="srt", tau=tau)
            rho, u = inputs.shear_wave(n, n, n, U=(U, 0, 0), amplitude=0.01, device="cuda")
            sim = _sim(n, n, n, precision=precision, **kw)
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
            r1, u1 = inputs.shear_wave(n, 1, 1, U=(U, 0, 0), amplitude=0.01)
            _, uo = oracle.run(cfg, r1.numpy(), u1.numpy(), steps)
            uo = uo[:, 0, 0, :]
            err = rel_maxnorm(col, uo)
            err_y = float(np.abs(col[1] - uo[1]).max() / np.abs(uo[1]).max())
            amp, ph = _shear_amp_phase(col[1], n)
            rate_err = (math.log(0.01 / amp) / steps) / (nu * k * k) - 1
            ph_err = (ph + math.pi / 2 + k * U * steps + math.pi) % (2 * math.pi) - math.pi
            amp_o, ph_o = _shear_amp_phase(uo[1], n)
            rate_err_o = (math.log(0.01 / amp_o) / steps) / (nu * k * k) - 1
            print("shear256 %s U=%.2f %-8s |u-u_oracle|/|u| %.2e, u_y alone %.2e; decay-rate err %+.3e "
                  "(oracle %+.3e), phase err %+.3e rad" % (precision, U, equilibrium, err, err_y, rate_err,
                                                           rate_err_o, ph_err))
            assert np.isfinite(col).all()
            worst = max(worst, err)
    assert worst < (0.15 if precision == "f16s" else 0.2)


# ------------------------------------------------------------------ channel 512x256x256

# Profile error of the 16-bit channel runs against the FP64 oracle after 5000
# steps, as measured (guards against regressions, not targets): FP16 storage
# cannot hold the per-step force increment of the shifted populations (about
# 3e-8 against an FP16 spacing of about 6e-8 at 1e-4), so the flow never
# starts (error 1.0); BF16 stagnates (about 0.82).
CHANNEL_16BIT_ERR = {"f16s": 1.0 + 1e-6, "bf16s": 0.85}


# Absolute slack beside half an ulp of the stored value in the sampled
# one-step comparison (the FP32 arithmetic of the collision).
ONE_STEP_SLACK = {"f32": 2e-8, "f16s": 1e-7, "bf16s": 1e-7}


@pytest.mark.parametrize("precision,pattern", [("f32", "ab"), ("f16s", "ab"), ("bf16s", "ab"), ("f32", "aa"),
                                               ("f16s", "aa")])
def test_channel_512x256x256_one_step_on_a_random_state(precision, pattern):
    """The walled channel's lattice and collision (512x256x256, walls at both y
    ends, TRT 3/16, tau = 0.6, body force) at full size, with the bench's
    kernels (interior rows through the periodic kernel, wall rows through the
    walled one): from a random state (seeded rho in 1 +- 0.02, u in +-0.05,
    three steps on), one GPU step of 256 sampled cells (random, on both walls,
    and on the periodic x and z ends) equals the FP64 oracle's step of each
    cell's neighbourhood (next to a wall: the two rows at the wall with walls in
    the patch) to within half an ulp of the stored value plus the FP32
    arithmetic, for both AA parities."""
    from tests._helpers import one_step_sampled_errors
    nx, ny, nz, tau = 512, 256, 256, 0.6
    a = 8 * (tau - 0.5) / 3 * 0.05 / ny ** 2
    kw = dict(equilibrium="improved", collision="trt", tau=tau, force=(a, 0, 0), walls=(False, True, False))
    sim = _sim(nx, ny, nz, precision=precision, pattern=pattern, **kw)
    gen = torch.Generator(device="cuda").manual_seed(91)
    rho = 1 + 0.02 * (2 * torch.rand((nz, ny, nx), generator=gen, device="cuda") - 1)
    u = 0.05 * (2 * torch.rand((3, nz, ny, nx), generator=gen, device="cuda") - 1)
    sim.init(rho, u)
    del rho, u
    sim.step(3)
    rng = np.random.default_rng(92)
    pts = [np.array([rng.integers(0, nz), rng.integers(0, ny), rng.integers(0, nx)]) for _ in range(160)]
    pts += [np.array([rng.integers(0, nz), yw, rng.integers(0, nx)]) for yw in (0, ny - 1) for _ in range(32)]
    pts += [np.array([rng.integers(0, nz), rng.integers(0, ny), xe]) for xe in (0, nx - 1) for _ in range(8)]
    pts += [np.array([ze, rng.integers(0, ny), rng.integers(0, nx)]) for ze in (0, nz - 1) for _ in range(8)]
    res = [one_step_sampled_errors(sim, pts, kw, precision, ONE_STEP_SLACK[precision]) for _ in range(2)]
    sim.close()
    worst, worst_abs = max(r[0] for r in res), max(r[1] for r in res)
    print("channel 512x256x256 %s %s, random state: one-step error on %d sampled cells, in units of (half an ulp "
          "of the storage + slack): max %.3f (largest absolute difference %.3e)"
          % (precision, pattern, len(pts), worst, worst_abs))
    assert worst <= 1.0 + 1e-9


@pytest.mark.parametrize("precision,pattern,collision,equilibrium,stencil", [
    ("f32", "ab", "srt", "improved", 19), ("f32", "ab", "trt", "standard", 19), ("f16s", "ab", "srt", "improved", 19),
    ("bf16s", "aa", "trt", "improved", 19), ("f32", "aa", "mrt", "improved", 19), ("f16s", "ab", "mrt", "standard", 19),
    ("f32", "ab", "trt", "standard", 27), ("f16s", "ab", "srt", "standard", 27)])
def test_periodic_256_one_step_on_a_random_state(precision, pattern, collision, equilibrium, stencil):
    """The benchmark's lattice (periodic 256^3) and launch configuration from a
    random state (seeded rho in 1 +- 0.02, u in +-0.05, three steps on): one
    GPU step of 192 sampled cells (random, and on the periodic faces and
    corners) equals the FP64 oracle's step of each cell's 3 x 3 x 3
    neighbourhood to within half an ulp of the stored value plus the FP32
    arithmetic, for SRT, TRT and MRT, both equilibria, A/B and both AA
    parities, and for the D3Q27 comparison lattice."""
    from tests._helpers import one_step_sampled_errors
    n, tau = 256, 0.8
    kw = dict(equilibrium=equilibrium, collision=collision, tau=tau)
    if collision == "mrt":
        kw.update(omega_bulk=1.3, omega_4=0.9)
    sim = _sim(n, n, n, precision=precision, pattern=pattern, stencil=stencil, **kw)
    gen = torch.Generator(device="cuda").manual_seed(93)
    rho = 1 + 0.02 * (2 * torch.rand((n, n, n), generator=gen, device="cuda") - 1)
    u = 0.05 * (2 * torch.rand((3, n, n, n), generator=gen, device="cuda") - 1)
    sim.init(rho, u)
    del rho, u
    sim.step(3)
    rng = np.random.default_rng(94)
    pts = [rng.integers(0, n, 3) for _ in range(176)]
    pts += [np.array([a, b, c]) for a in (0, n - 1) for b in (0, n - 1) for c in (0, n - 1)]
    pts += [np.array([rng.integers(0, n), rng.integers(0, n), xe]) for xe in (0, n - 1) for _ in range(4)]
    res = [one_step_sampled_errors(sim, pts, kw, precision, ONE_STEP_SLACK[precision]) for _ in range(2)]
    sim.close()
    worst, worst_abs = max(r[0] for r in res), max(r[1] for r in res)
    print("periodic 256^3 D3Q%d %s %s %s %s, random state: one-step error on %d sampled cells, in units of (half an "
          "ulp of the storage + slack): max %.3f (largest absolute difference %.3e)"
          % (stencil, precision, pattern, collision, equilibrium, len(pts), worst, worst_abs))
    assert worst <= 1.0 + 1e-9


@pytest.mark.parametrize("precision", ["f32", "f16s", "bf16s"])
def test_channel_512x256x256(precision):
    """Walls at y = -1/2 and 255.5, periodic x, z, body force a_x = 8 nu u_c / H^2
    (steady centreline 0.05), TRT 3/16, tau = 0.6, 5000 steps: every (x,z) column
    is bitwise equal, and the y profile is compared with the FP64 oracle's
    1x256x1 column.  FP32: <= 1e-5 against the oracle and <= 1e-5 against the
    oracle with FP32 storage (FP64 steps, populations rounded to float32 after
    each step), whose own distance to the oracle (the floor that FP32 storage
    sets) is printed.  16-bit storage: the measured profile errors
    (CHANNEL_16BIT_ERR) are asserted as upper bounds."""
    nx, ny, nz, steps, tau = 512, 256, 256, 5000, 0.6
    nu = (tau - 0.5) / 3
    a = 8 * nu * 0.05 / ny ** 2
    kw = dict(equilibrium="improved", collision="trt", tau=tau, force=(a, 0, 0), walls=(False, True, False))
    sim = _sim(nx, ny, nz, precision=precision, **kw)
    rho, u = inputs.rest(nx, ny, nz, device="cuda")
    sim.init(rho, u.float())
    del rho, u
    sim.step(steps)
    _, ug = sim.moments(torch.float32)
    ref = ug[:, 0:1, :, 0:1]
    assert torch.equal(ug, ref.expand_as(ug)), "columns differ"
    prof = ref[:, 0, :, 0].double().cpu().numpy()
    del ug
    sim.close()
    cfg = oracle_config(1, ny, 1, **kw)
    r1, u1 = inputs.rest(1, ny, 1)
    _, uo = oracle.run(cfg, r1.numpy(), u1.numpy(), steps)
    uo = uo[:, 0, :, 0]
    err = rel_maxnorm(prof[0], uo[0])
    print("channel %s: u_x profile max-norm rel err vs FP64 oracle after %d steps = %.3e (u_max %.3e)"
          % (precision, steps, err, uo[0].max()))
    if precision == "f32":
        _, ue = oracle_run_fp32_storage(cfg, r1.numpy(), u1.numpy(), steps)
        ue = ue[:, 0, :, 0]
        err_e = rel_maxnorm(prof[0], ue[0])
        print("channel f32: vs the oracle with FP32 storage %.3e; that emulation vs the oracle %.3e"
              % (err_e, rel_maxnorm(ue[0], uo[0])))
        assert err < FP32_LONG_TOL and err_e < FP32_LONG_TOL
        assert np.abs(prof[1:]).max() < 1e-9
    else:
        assert np.isfinite(prof).all()
        assert err <= CHANNEL_16BIT_ERR[precision]


def test_poiseuille_steady_profile_on_gpu():
    """TRT 3/16 with half-way bounce-back reaches the exact parabola (small H so
    the steady state is reached in a few thousand steps)."""
    nx, ny, nz, tau = 64, 16, 8, 0.8
    nu = (tau - 0.5) / 3
    a = 1e-6
    sim = _sim(nx, ny, nz, precision="f64", equilibrium="improved", collision="trt", tau=tau, force=(a, 0, 0),
               walls=(False, True, False))
    rho, u = inputs.rest(nx, ny, nz, device="cuda")
    sim.init(rho, u)
    sim.step(20000)
    _, ug = sim.moments()
    y = np.arange(ny)
    exact = a / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    err = np.abs(ug[0, 0, :, 0].cpu().numpy() - exact).max() / exact.max()
    print("Poiseuille H=16 TRT 3/16: max rel deviation from the parabola %.2e" % err)
    assert err < 1e-9


# ------------------------------------------------------------------ duct and cross shear (S vs I)

def test_cross_shear_spurious_velocity_s_vs_i():
    """x-invariant u = (U + A sin sin, 0, 0): D3Q19-I keeps u_y = u_z = 0 exactly,
    D3Q19-S develops transverse velocity (the paper's duct mechanism, Sec. 4)."""
    n = 64
    out = {}
    for equilibrium in ("standard", "improved"):
        # tau = 1: Lambda^2 = 1/4, away from 1/12 where the S error term vanishes
        sim = _sim(8, n, n, precision="f64", equilibrium=equilibrium, collision="srt", tau=1.0)
        rho, u = inputs.cross_shear(8, n, n, U=0.05, amplitude=0.02, device="cuda")
        sim.init(rho, u)
        sim.step(500)
        _, ug = sim.moments()
        out[equilibrium] = float(ug[1:].abs().max() / ug[0].abs().max())
    print("cross shear: max|u_yz|/max|u_x|  S = %.3e   I = %.3e" % (out["standard"], out["improved"]))
    assert out["improved"] < 1e-13
    assert out["standard"] > 1e-7


def test_duct_flow_spurious_currents():
    """Square duct (Sec. 5.1): periodic x, half-way bounce-back walls in y and z,
    body force in x.  max|u_yz| / max|u_x| is at rounding level for D3Q19-I and
    clearly non-zero for D3Q19-S."""
    D, tau = 24, 1.0  # Lambda^2 = 1/4, far from the optimum 1/12 (Sec. 5.1)
    a = 1e-5
    out = {}
    for equilibrium in ("standard", "improved"):
        sim = _sim(4, D, D, precision="f64", equilibrium=equilibrium, collision="srt", tau=tau,
                   force=(a, 0, 0), walls=(False, True, True))
        rho, u = inputs.rest(4, D, D, device="cuda")
        sim.init(rho, u)
        sim.step(6000)
        _, ug = sim.moments()
        out[equilibrium] = float(ug[1:].abs().max() / ug[0].abs().max())
    print("duct D=%d: max|u_yz|/max|u_x|  S = %.3e   I = %.3e" % (D, out["standard"], out["improved"]))
    assert out["improved"] < 1e-12
    assert out["standard"] > 1e-8


def _duct_ratio(D, tau, equilibrium, nsteps=None, Re=10.0):
    """Steady square duct at Re = u_max D / nu = 10: max|u_yz| / max|u_x|."""
    nu = (tau - 0.5) / 3
    # square duct: u_max ~ 0.2947 a (D/2)^2 / nu  ->  a for the requested Re
    a = Re * nu * nu / (0.2947 * D * (D / 2) ** 2)
    if nsteps is None:
        nsteps = int(8 * D * D / (math.pi ** 2 * nu)) + 500
    sim = _sim(2, D, D, precision="f64", equilibrium=equilibrium, collision="srt", tau=tau, force=(a, 0, 0),
               walls=(False, True, True))
    rho, u = inputs.rest(2, D, D, device="cuda")
    sim.init(rho, u)
    sim.step(nsteps)
    _, ug = sim.moments()
    return float(ug[1:].abs().max() / ug[0].abs().max())


def test_duct_lambda_dependence():
    """Sec. 5.1, Fig. 1 right: the D3Q19-S spurious currents depend on
    Lambda^2 = (1/omega - 1/2)^2; the analysis (Sec. 4) puts the leading error
    term's zero at Lambda^2 = 1/12.  Measured at Re = 10: the minimum over
    Lambda^2 moves towards 1/12 as D grows from 16 to 32 to 64 (higher-order
    terms shift it at small D), and D3Q19-I stays at rounding level for every
    Lambda."""
    lam2 = [0.01, 0.03, 0.05, 0.0667, 1 / 12, 0.1, 0.12, 0.16, 0.25]
    argmin = {}
    for D in (16, 32, 64):
        rs, ri = [], []
        for l2 in lam2:
            tau = 0.5 + math.sqrt(l2)
            rs.append(_duct_ratio(D, tau, "standard"))
            ri.append(_duct_ratio(D, tau, "improved"))
        for l2, a, b in zip(lam2, rs, ri):
            print("duct D=%d Lambda^2=%.4f: S %.3e  I %.3e" % (D, l2, a, b))
        assert max(ri) < 1e-13
        argmin[D] = lam2[int(np.argmin(rs))]
        if D == 32:
            k = lam2.index(1 / 12)
            assert rs[k] < 0.2 * rs[-1] and rs[k] < 0.35 * rs[0]
    print("duct: Lambda^2 of the smallest S current: D=16 %.4f, D=32 %.4f, D=64 %.4f (analysis: %.4f)"
          % (argmin[16], argmin[32], argmin[64], 1 / 12))
    assert argmin[16] <= argmin[32] <= argmin[64] <= 0.1
    assert argmin[32] >= 0.05
    assert argmin[64] == 1 / 12  # measured: the grid point of the analysis' optimum


def test_duct_convergence_orders():
    """Sec. 5.1, Fig. 2: at Lambda^2 = 4/25 the D3Q19-S spurious-current ratio
    converges at second order under diffusive scaling (fixed tau, Re = 10)."""
    tau = 0.5 + 0.4
    r = [_duct_ratio(D, tau, "standard") for D in (12, 24, 48, 96)]
    orders = [math.log2(r[i] / r[i + 1]) for i in range(3)]
    print("duct Lambda^2=4/25 S ratios %s, observed orders %s" % (r, orders))
    assert 1.6 < orders[-2] < 2.4 and 1.8 < orders[-1] < 2.2


def test_shear_wave_with_normal_velocity_profile():
    """Shear wave u_y(x) plus a normal velocity u_z(x) = 0.05 sin(2 pi x / n):
    (u_x, u_y) evolve as without u_z for D3Q19-I (its (c_x, c_y) projection is
    D2Q9 for any u_z; Eq. 22) and also for D3Q19-S: the u_z^2 terms by which S
    differs are even in c_x and c_y and carry no x-momentum flux, so a flow that
    varies along one axis only cannot feel them.  The S/I difference needs
    variation along two axes (the duct and cross-shear tests; the error term of
    Eq. 39 has derivatives along two axes)."""
    import math as _m
    from paper_1803_04937_gb300.lbm import Simulation
    n, steps = 128, 500
    out = {}
    for equilibrium in ("standard", "improved"):
        res = []
        for amp_z in (0.0, 0.05):
            rho, u = inputs.shear_wave(n, 4, 4, U=(0.05, 0.0, 0.0), amplitude=0.01, device="cuda")
            x = torch.arange(n, dtype=torch.float64, device="cuda")
            u[2] += amp_z * torch.sin(2 * _m.pi * x / n)
            sim = Simulation(n, 4, 4, precision="f64", equilibrium=equilibrium, collision="srt", tau=0.6)
            sim.init(rho, u)
            sim.step(steps)
            _, ug = sim.moments()
            res.append(ug[:2].cpu().numpy())
        out[equilibrium] = float(np.abs(res[1] - res[0]).max() / np.abs(res[0]).max())
    print("shear wave with u_z(x) vs u_z = 0: max rel change of (u_x, u_y)  S = %.3e   I = %.3e"
          % (out["standard"], out["improved"]))
    assert out["improved"] < 1e-12 and out["standard"] < 1e-12
