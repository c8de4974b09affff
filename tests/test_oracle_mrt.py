"""Pins of the oracle's MRT collision (Sec. 3.2-3.3: relaxation in the monomial
moment space against the Maxwellian's moments) against the TRT and SRT updates
it contains, Table 1's moments, the per-moment relaxation that defines it, the
Chapman-Enskog sound attenuation with a bulk viscosity, conservation, and the
Poiseuille closed form."""
import itertools
import json
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_moments.json")

# the eight moments Eq. 21 drops on D3Q19
DROPPED = {(1, 2, 2), (2, 1, 2), (2, 2, 1), (1, 1, 2), (1, 2, 1), (2, 1, 1), (1, 1, 1), (2, 2, 2)}


def _random_cell(cfg, seed, amp=2e-3):
    rng = np.random.default_rng(seed)
    rho = 1 + rng.uniform(-0.03, 0.03, cfg.shape)
    u = rng.uniform(-0.06, 0.06, (3,) + cfg.shape)
    f = oracle.init(cfg, rho, u)
    return f + rng.uniform(-amp, amp, f.shape)


@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
@pytest.mark.parametrize("rho0_is_rho", [False, True])
@pytest.mark.parametrize("stencil", [19, 27])
def test_mrt_with_equal_even_rates_is_trt_and_srt(eq, rho0_is_rho, stencil):
    tau = 0.7
    kw = dict(equilibrium=eq, tau=tau, accel=(3e-4, -2e-4, 1e-4), rho0_is_rho=rho0_is_rho, stencil=stencil,
              walls=(False, True, False))
    mrt = oracle.Config(5, 4, 3, collision=oracle.MRT, omega_bulk=1 / tau, omega_4=1 / tau, **kw)
    trt = oracle.Config(5, 4, 3, collision=oracle.TRT, **kw)
    f = _random_cell(mrt, 3)
    assert np.abs(oracle.step(mrt, f, 3) - oracle.step(trt, f, 3)).max() < 2e-15
    # magic (tau - 1/2)^2 makes omega- = omega+: SRT (Eq. 15)
    srt = oracle.Config(5, 4, 3, collision=oracle.SRT, **kw)
    mrt.trt_magic = (tau - 0.5) ** 2
    assert np.abs(oracle.step(mrt, f, 3) - oracle.step(srt, f, 3)).max() < 2e-15


def _table1_maxwellian(rho, rho0, u):
    """Maxwellian moment xi^e (second order in u) for every e in {0,1,2}^3, from
    the Table 1 fixture."""
    table = json.load(open(GOLDEN))
    out = {}
    for row in table["rows"]:
        for perm in itertools.permutations(range(3)):
            roles = dict(zip("ijk", perm))
            e = [0, 0, 0]
            for r, p in row["exponents"].items():
                e[roles[r]] = p
            val = 0.0
            for coef, dens, mono in row["Maxwellian"]:
                if sum(mono.values()) > 2:
                    continue
                t = float(Fr(coef)) * (rho if dens == "rho" else rho0)
                for role, p in mono.items():
                    t *= u[roles[role]] ** p
                val += t
            out[tuple(e)] = val
    assert len(out) == 27
    return out


@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
def test_mrt_relaxes_each_moment_at_its_rate(eq):
    """One cell with periodic wrap: streaming is the identity, so one step is
    one collision.  Every kept moment's distance from its equilibrium value
    shrinks by (1 - its rate), the force entering as (1 - rate/2) M F: odd
    orders at omega-, the deviatoric second-order block at omega+, its trace at
    omega_bulk, the fourth-order moments at omega_4.  Equilibrium moments: the
    Maxwellian column of Table 1 for D3Q19-I (Sec. 3.2), the moments of Eq. 14
    for D3Q19-S."""
    tau, magic, wb, w4 = 0.62, 0.25, 1.37, 0.83
    a = np.array([2e-4, -3e-4, 1.5e-4])
    cfg = oracle.Config(1, 1, 1, equilibrium=eq, collision=oracle.MRT, tau=tau, trt_magic=magic, accel=tuple(a),
                        omega_bulk=wb, omega_4=w4)
    wp = 1 / tau
    wm = 1 / (0.5 + magic / (tau - 0.5))
    c, w, _ = oracle.velocity_set()
    cf = c.astype(float)
    f = _random_cell(cfg, 8).reshape(19)
    fs = oracle.step(cfg, f.reshape(1, 1, 1, 19)).reshape(19)
    rho = f.sum()
    u = cf.T @ f + a / 2
    F = 3 * w * (cf @ a)
    if eq == oracle.IMPROVED:
        meq = _table1_maxwellian(rho, 1.0, u)
    else:
        feq = oracle.equilibrium(oracle.STANDARD, np.array([rho]), u.reshape(3, 1))[0]

    def mom(g, e):
        return float((g * np.prod(cf ** np.asarray(e), axis=1)).sum())

    def eqm(e):
        return meq[e] if eq == oracle.IMPROVED else mom(feq, e)

    kept = [e for e in itertools.product((0, 1, 2), repeat=3) if e not in DROPPED]
    assert len(kept) == 19
    diag = [e for e in kept if sorted(e) == [0, 0, 2]]
    n_diag = np.array([mom(f, e) - eqm(e) for e in diag])
    F_diag = np.array([mom(F, e) for e in diag])
    trace = n_diag.mean()
    for e in kept:
        order = sum(e)
        before, after, Fe = mom(f, e) - eqm(e), mom(fs, e) - eqm(e), mom(F, e)
        if order == 0:
            want = before
        elif order % 2 == 1:
            want = (1 - wm) * before + (1 - wm / 2) * Fe
        elif e in diag:
            i = diag.index(e)
            want = (1 - wp) * (before - trace) + (1 - wb) * trace + F_diag[i]
        elif order == 2:
            want = (1 - wp) * before + Fe
        else:
            want = (1 - w4) * before + Fe
        assert after == pytest.approx(want, abs=3e-16), e
    # the second-order and fourth-order moments of F vanish (F is odd in c)
    assert np.abs(F_diag).max() < 1e-18


def _sound_decay_rate(cfg, n, amp=1e-5, steps=2400):
    from scipy.optimize import curve_fit
    x = np.arange(n)
    k = 2 * np.pi / n
    rho = (1 + amp * np.cos(k * x)).reshape(1, 1, n)
    f = oracle.init(cfg, rho, np.zeros((3, 1, 1, n)))
    t, a = [], []
    for s in range(steps):
        if s % 4 == 0:
            r, _ = oracle.moments(cfg, f)
            t.append(s)
            a.append(2 * float((r[0, 0] - 1) @ np.cos(k * x)) / n)
        f = oracle.step(cfg, f)
    t, a = np.array(t, float), np.array(a) / amp

    def model(tt, A, G, W, P):
        return A * np.exp(-G * tt) * np.cos(W * tt + P)

    p, _ = curve_fit(model, t, a, p0=(1.0, 3e-4, k / math.sqrt(3), 0.0))
    return p[1], p[2]


@pytest.mark.parametrize("wb", [None, 0.7, 1.0, 1.5])
def test_mrt_sound_attenuation_follows_bulk_viscosity(wb):
    """Chapman-Enskog with the trace of the second-order moments relaxing at
    omega_bulk: shear viscosity nu = (tau - 1/2)/3, bulk viscosity
    zeta = (2/9)(1/omega_bulk - 1/2), and a standing sound wave of wave number
    k decays at (k^2/2)(4/3 nu + zeta) (nu k^2 when omega_bulk = omega+).
    (Not every pair of rates is stable: omega_bulk = 1.9 with omega_4 = 1 at
    tau = 0.6 has a growing mode of wave number 2 pi/3.)"""
    tau, n = 0.6, 48
    wb_ = 1 / tau if wb is None else wb
    cfg = oracle.Config(n, 1, 1, collision=oracle.MRT, tau=tau, omega_bulk=wb_, omega_4=1.0)
    G, W = _sound_decay_rate(cfg, n)
    k = 2 * np.pi / n
    nu = (tau - 0.5) / 3
    zeta = 2 / 9 * (1 / wb_ - 0.5)
    want = k * k / 2 * (4 / 3 * nu + zeta)
    assert G == pytest.approx(want, rel=0.02)
    assert W == pytest.approx(k / math.sqrt(3), rel=0.01)


@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
def test_mrt_conserves_mass_and_momentum(eq):
    a = (1e-3, -2e-3, 5e-4)
    cfg = oracle.Config(1, 1, 1, equilibrium=eq, collision=oracle.MRT, tau=0.57, trt_magic=0.1, accel=a,
                        omega_bulk=1.7, omega_4=0.6)
    c, _, _ = oracle.velocity_set()
    f = _random_cell(cfg, 4)
    f1 = oracle.step(cfg, f)
    assert f1.sum() == pytest.approx(f.sum(), abs=1e-15)
    assert np.allclose(c.T @ f1.reshape(19) - c.T @ f.reshape(19), a, atol=1e-16)


@pytest.mark.parametrize("wb,w4", [(1.0, 1.0), (1.6, 0.7)])
def test_mrt_poiseuille_exact_with_magic(wb, w4):
    """Channel between half-way bounce-back walls: with Lambda = 3/16 the
    steady profile is u = a/(2 nu) (y + 1/2)(H - 1/2 - y) to rounding for any
    bulk and fourth-order rates (a unidirectional steady flow has non-equilibrium
    only in the shear moment and the odd moments)."""
    H, a, tau = 12, 1e-5, 0.7
    nu = (tau - 0.5) / 3
    cfg = oracle.Config(1, H, 1, collision=oracle.MRT, tau=tau, accel=(a, 0, 0), walls=(False, True, False),
                        omega_bulk=wb, omega_4=w4)
    f = oracle.step(cfg, oracle.init(cfg, np.ones(cfg.shape), np.zeros((3,) + cfg.shape)), 20000)
    _, u = oracle.moments(cfg, f)
    y = np.arange(H)
    exact = a / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    assert np.abs(u[0, 0, :, 0] - exact).max() / exact.max() < 1e-9


def test_mrt_adjoint_is_refused():
    cfg = oracle.Config(2, 2, 2, collision=oracle.MRT)
    f = oracle.init(cfg, np.ones(cfg.shape), np.zeros((3,) + cfg.shape))
    with pytest.raises(ValueError):
        oracle.adjoint_step(cfg, f, f)


def _duct_ratio(D, eq, coll, tau, wb=1.0, w4=1.0, Re=10.0):
    nu = (tau - 0.5) / 3
    a = Re * nu * nu / (0.2947 * D * (D / 2) ** 2)
    cfg = oracle.Config(1, D, D, equilibrium=eq, collision=coll, tau=tau, accel=(a, 0, 0), walls=(False, True, True),
                        omega_bulk=wb, omega_4=w4)
    f = oracle.step(cfg, oracle.init(cfg, np.ones(cfg.shape), np.zeros((3,) + cfg.shape)),
                    int(8 * D * D / (math.pi ** 2 * nu)) + 500)
    _, u = oracle.moments(cfg, f)
    return np.abs(u[1:]).max() / np.abs(u[0]).max()


def test_mrt_duct_improved_keeps_no_transverse_currents_when_bulk_equals_shear():
    """Square duct (Sec. 5.1) at D = 12: with the Maxwellian moments the
    transverse velocity stays at rounding level for any fourth-order rate as
    long as the bulk rate equals omega+ (the paper's remark that changing only
    higher-order rates keeps the benefit, Sec. 3.3); a different bulk rate does
    not, and D3Q19-S has currents for any rates."""
    tau = 0.8
    wp = 1 / tau
    assert _duct_ratio(12, oracle.IMPROVED, oracle.MRT, tau, wp, 1.0) < 1e-13
    assert _duct_ratio(12, oracle.IMPROVED, oracle.MRT, tau, wp, 1.6) < 1e-13
    s = _duct_ratio(12, oracle.STANDARD, oracle.MRT, tau, wp, 1.0)
    b = _duct_ratio(12, oracle.IMPROVED, oracle.MRT, tau, 1.0, 1.0)
    assert s > 1e-5 and 1e-8 < b < s
