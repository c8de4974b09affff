"""Pins of the oracle's time step (Eq. 15-17, TRT, boundaries) against facts that
do not come from the oracle: conservation laws, fixed points, the symmetries of
the cubic lattice, an independently written textbook D2Q9 step, the closed-form
Poiseuille solution of half-way bounce-back, and the viscous decay rate
nu = c_s^2 (tau - 1/2) approached at second order in the grid spacing."""
import math

import numpy as np
import pytest

import oracle
from paper_1803_04937_gb300 import inputs


def _np(t):
    return t.numpy()


def _random_state(shape, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    rho = 1 + rng.uniform(-0.02, 0.02, (nz, ny, nx))
    u = rng.uniform(-amp, amp, (3, nz, ny, nx))
    return rho, u


# ------------------------------------------------------------------ conservation

@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
@pytest.mark.parametrize("coll", [oracle.SRT, oracle.TRT])
@pytest.mark.parametrize("rho0_is_rho", [False, True])
def test_single_cell_collision_conserves_mass_and_momentum(eq, coll, rho0_is_rho):
    """On a 1x1x1 periodic lattice streaming is the identity, so one step is one
    collision: sum f is unchanged and sum c f grows by exactly a (Eq. 15-17)."""
    a = (1e-3, -2e-3, 5e-4)
    cfg = oracle.Config(1, 1, 1, equilibrium=eq, collision=coll, tau=0.7, accel=a, rho0_is_rho=rho0_is_rho)
    c, _, _ = oracle.velocity_set()
    rng = np.random.default_rng(1)
    f = oracle.init(cfg, np.array([[[1.01]]]), np.array([0.05, -0.02, 0.03]).reshape(3, 1, 1, 1))
    f = f + rng.uniform(-1e-3, 1e-3, f.shape)  # non-equilibrium part
    f1 = oracle.step(cfg, f)
    assert f1.sum() == pytest.approx(f.sum(), abs=1e-15)
    j0 = c.T @ f.reshape(19)
    j1 = c.T @ f1.reshape(19)
    assert np.allclose(j1 - j0, a, atol=1e-16)
    # non-trivial: the populations did change
    assert np.abs(f1 - f).max() > 1e-5


def test_global_mass_and_momentum_over_a_run():
    cfg = oracle.Config(8, 6, 5, tau=0.8, accel=(1e-5, 0, 0))
    rho, u = _random_state(cfg.shape, 2)
    f = oracle.init(cfg, rho, u)
    c, _, _ = oracle.velocity_set()
    m0 = f.sum()
    j0 = (f.reshape(-1, 19) @ c).sum(axis=0)
    f = oracle.step(cfg, f, 50)
    assert abs(f.sum() - m0) / m0 < 1e-13
    j = (f.reshape(-1, 19) @ c).sum(axis=0)
    assert np.allclose(j - j0, 50 * cfg.ncell * np.array(cfg.accel), atol=1e-12)


# ------------------------------------------------------------------ fixed points

@pytest.mark.parametrize("walls", [(False, False, False), (True, True, False)])
def test_rest_state_is_a_fixed_point(walls):
    cfg = oracle.Config(5, 4, 3, collision=oracle.TRT, walls=walls)
    rho, u = _np(inputs.rest(5, 4, 3)[0]), _np(inputs.rest(5, 4, 3)[1])
    f0 = oracle.init(cfg, rho, u)
    f = oracle.step(cfg, f0, 10)
    assert np.abs(f - f0).max() < 1e-16


@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
def test_uniform_flow_is_a_fixed_point(eq):
    cfg = oracle.Config(5, 4, 3, equilibrium=eq)
    rho = np.ones(cfg.shape)
    u = np.zeros((3,) + cfg.shape)
    u[0], u[1], u[2] = 0.05, -0.03, 0.02
    f0 = oracle.init(cfg, rho, u)
    f = oracle.step(cfg, f0, 10)
    assert np.abs(f - f0).max() < 1e-15


# ------------------------------------------------------------------ symmetries

def _run(cfg, rho, u, n):
    return oracle.run(cfg, rho, u, n)


@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
@pytest.mark.parametrize("coll", [oracle.SRT, oracle.TRT])
def test_axis_permutation_equivariance(eq, coll):
    """The D3Q19 lattice is invariant under axis permutations: permuting the
    input (fields, walls, force) permutes the output."""
    base = oracle.Config(7, 5, 4, equilibrium=eq, collision=coll, tau=0.65,
                         accel=(2e-4, -1e-4, 3e-4), walls=(False, True, False))
    rho, u = _random_state(base.shape, 3)
    r0, u0 = _run(base, rho, u, 6)
    for perm in [(1, 2, 0), (2, 0, 1), (1, 0, 2), (0, 2, 1)]:
        # new axis i is old axis perm[i]; numpy axes are (z, y, x) = (2, 1, 0)
        n_old = (base.nx, base.ny, base.nz)
        n_new = [n_old[perm[i]] for i in range(3)]
        cfg = oracle.Config(*n_new, equilibrium=eq, collision=coll, tau=0.65,
                            accel=tuple(base.accel[perm[i]] for i in range(3)),
                            walls=tuple(base.walls[perm[i]] for i in range(3)))
        np_axes = tuple(2 - perm[2 - k] for k in range(3))
        rho_p = np.transpose(rho, np_axes)
        u_p = np.stack([np.transpose(u[perm[i]], np_axes) for i in range(3)])
        r1, u1 = _run(cfg, rho_p, u_p, 6)
        assert np.abs(r1 - np.transpose(r0, np_axes)).max() < 1e-14
        for i in range(3):
            assert np.abs(u1[i] - np.transpose(u0[perm[i]], np_axes)).max() < 1e-14


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reflection_equivariance(axis):
    cfg = oracle.Config(6, 5, 4, collision=oracle.TRT, tau=0.9, accel=(1e-4, 2e-4, -1e-4),
                        walls=(axis == 0, False, axis == 2))
    rho, u = _random_state(cfg.shape, 4)
    r0, u0 = _run(cfg, rho, u, 5)
    npax = 2 - axis
    acc = list(cfg.accel)
    acc[axis] = -acc[axis]
    cfg_m = oracle.Config(6, 5, 4, collision=oracle.TRT, tau=0.9, accel=tuple(acc), walls=cfg.walls)
    um = np.flip(u, axis=npax + 1).copy()
    um[axis] *= -1
    r1, u1 = _run(cfg_m, np.flip(rho, axis=npax).copy(), um, 5)
    u1f = np.flip(u1, axis=npax + 1).copy()
    u1f[axis] *= -1
    assert np.abs(np.flip(r1, axis=npax) - r0).max() < 1e-14
    assert np.abs(u1f - u0).max() < 1e-14


def test_periodic_translation_equivariance():
    cfg = oracle.Config(6, 5, 4, tau=0.7)
    rho, u = _random_state(cfg.shape, 5)
    r0, u0 = _run(cfg, rho, u, 4)
    sh = (1, -2, 3)
    r1, u1 = _run(cfg, np.roll(rho, sh, axis=(0, 1, 2)), np.roll(u, sh, axis=(1, 2, 3)), 4)
    assert np.array_equal(r1, np.roll(r0, sh, axis=(0, 1, 2)))
    assert np.array_equal(u1, np.roll(u0, sh, axis=(1, 2, 3)))


# ------------------------------------------------------------------ D2Q9 textbook

def _d2q9_run(rho, ux, uy, tau, magic, trt, accel, wall_y, nsteps):
    """Independent textbook D2Q9 (standard second-order equilibrium with rho0 = 1,
    Buick-Greated force, u = j + a/2), push streaming with np.roll and half-way
    bounce-back at the two y ends.  Arrays are [y, x]."""
    c = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]
    opp = [0, 2, 1, 4, 3, 6, 5, 8, 7]
    w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
    ax, ay = accel

    def feq(r, vx, vy):
        uu = vx * vx + vy * vy
        return [w[q] * r + w[q] * (3 * (c[q][0] * vx + c[q][1] * vy)
                                   + 4.5 * (c[q][0] * vx + c[q][1] * vy) ** 2 - 1.5 * uu) for q in range(9)]

    f = feq(rho, ux, uy)
    wp = 1 / tau
    wm = 1 / (0.5 + magic / (tau - 0.5)) if trt else wp
    for _ in range(nsteps):
        r = sum(f)
        vx = sum(c[q][0] * f[q] for q in range(9)) + ax / 2
        vy = sum(c[q][1] * f[q] for q in range(9)) + ay / 2
        fe = feq(r, vx, vy)
        fs = []
        for q in range(9):
            o = opp[q]
            F = 3 * w[q] * (c[q][0] * ax + c[q][1] * ay)
            sym = 0.5 * (f[q] + f[o]) - 0.5 * (fe[q] + fe[o])
            asym = 0.5 * (f[q] - f[o]) - 0.5 * (fe[q] - fe[o])
            fs.append(f[q] - wp * sym - wm * asym + (1 - wm / 2) * F)
        new = []
        for q in range(9):
            g = np.roll(fs[q], (c[q][1], c[q][0]), axis=(0, 1))
            if wall_y and c[q][1] == 1:
                g[0, :] = fs[opp[q]][0, :]
            if wall_y and c[q][1] == -1:
                g[-1, :] = fs[opp[q]][-1, :]
            new.append(g)
        f = new
    r = sum(f)
    vx = sum(c[q][0] * f[q] for q in range(9)) + ax / 2
    vy = sum(c[q][1] * f[q] for q in range(9)) + ay / 2
    return r, vx, vy


@pytest.mark.parametrize("coll", [oracle.SRT, oracle.TRT])
@pytest.mark.parametrize("wall_y", [False, True])
def test_improved_equilibrium_projects_onto_textbook_d2q9(coll, wall_y):
    """For a z-invariant state, D3Q19-I summed over c_z is exactly a D2Q9 fluid
    with the standard equilibrium, for any u_z (a consequence of Eq. 22)."""
    nx, ny = 9, 7
    accel = (3e-4, -1e-4)
    cfg = oracle.Config(nx, ny, 1, equilibrium=oracle.IMPROVED, collision=coll, tau=0.7,
                        accel=(accel[0], accel[1], 0.0), walls=(False, wall_y, False))
    rho, u = _random_state(cfg.shape, 6)
    u[2] = np.random.default_rng(7).uniform(-0.05, 0.05, u[2].shape)  # arbitrary u_z
    r3, u3 = _run(cfg, rho, u, 12)
    r2, vx, vy = _d2q9_run(rho[0], u[0, 0], u[1, 0], 0.7, 3 / 16, coll == oracle.TRT, accel, wall_y, 12)
    assert np.abs(r3[0] - r2).max() < 1e-14
    assert np.abs(u3[0, 0] - vx).max() < 1e-14
    assert np.abs(u3[1, 0] - vy).max() < 1e-14


def test_standard_equals_improved_for_planar_flow_without_uz():
    """z-invariant flows with u_z = 0 evolve identically under D3Q19-S and
    D3Q19-I (both reduce to D2Q9 there): the shear wave with background flow."""
    rho, u = inputs.shear_wave(32, 1, 1, U=(0.1, 0, 0))
    res = []
    for eq in (oracle.STANDARD, oracle.IMPROVED):
        cfg = oracle.Config(32, 1, 1, equilibrium=eq, tau=0.55)
        res.append(_run(cfg, _np(rho), _np(u), 200))
    assert np.abs(res[0][1] - res[1][1]).max() < 1e-13


def test_cross_shear_transverse_velocity_only_for_standard():
    """x-invariant u = (U + A sin sin, 0, 0): D3Q19-I keeps u_y = u_z = 0 to
    rounding (its yz projection is a D2Q9 fluid at rest); D3Q19-S does not
    (the u_0^2 error term of Eq. 39, Sec. 4)."""
    n = 16
    rho, u = inputs.cross_shear(1, n, n, U=0.05, amplitude=0.02)
    out = {}
    for eq in (oracle.STANDARD, oracle.IMPROVED):
        cfg = oracle.Config(1, n, n, equilibrium=eq, tau=0.8)
        _, uu = _run(cfg, _np(rho), _np(u), 100)
        out[eq] = np.abs(uu[1:]).max()
    assert out[oracle.IMPROVED] < 1e-15
    assert out[oracle.STANDARD] > 1e-7


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("coll,tau", [(oracle.TRT, 0.6), (oracle.TRT, 0.9), (oracle.SRT, 0.6), (oracle.SRT, 1.1)])
@pytest.mark.parametrize("eq", [oracle.STANDARD, oracle.IMPROVED])
def test_poiseuille_closed_form(coll, tau, eq):
    """Steady force-driven channel between half-way bounce-back walls at y = -1/2
    and H - 1/2: u_x(y) = a/(2 nu) [(y + 1/2)(H - 1/2 - y) + (16 Lambda - 3)/12],
    Lambda = (tau+ - 1/2)(tau- - 1/2) (the known TRT bounce-back solution; exact
    parabola for Lambda = 3/16)."""
    H, a = 12, 1e-5
    nu = (tau - 0.5) / 3
    cfg = oracle.Config(1, H, 1, equilibrium=eq, collision=coll, tau=tau, accel=(a, 0, 0),
                        walls=(False, True, False))
    f = oracle.init(cfg, np.ones(cfg.shape), np.zeros((3,) + cfg.shape))
    f = oracle.step(cfg, f, 30000)
    _, u = oracle.moments(cfg, f)
    lam = (tau - 0.5) * (3 / 16 / (tau - 0.5)) if coll == oracle.TRT else (tau - 0.5) ** 2
    y = np.arange(H)
    exact = a / (2 * nu) * ((y + 0.5) * (H - 0.5 - y) + (16 * lam - 3) / 12)
    assert np.abs(u[0, 0, :, 0] - exact).max() / exact.max() < 1e-9
    assert np.abs(u[1:]).max() < 1e-14


def _decay_rate_error(n, tau, coll=oracle.SRT):
    """Relative error of the shear-wave decay rate against nu k^2 on an n x 1 x 1
    lattice (linear regime)."""
    rho, u = inputs.shear_wave(n, 1, 1, amplitude=1e-6)
    cfg = oracle.Config(n, 1, 1, equilibrium=oracle.IMPROVED, collision=coll, tau=tau)
    k = 2 * math.pi / n
    nu = (tau - 0.5) / 3
    steps = int(0.5 / (nu * k * k))
    f = oracle.init(cfg, _np(rho), _np(u))
    x = np.arange(n)
    amps = []
    for _ in range(2):
        f = oracle.step(cfg, f, steps)
        _, uu = oracle.moments(cfg, f)
        amps.append(abs((uu[1, 0, 0] * np.exp(-1j * k * x)).sum()))
    rate = math.log(amps[0] / amps[1]) / steps
    return rate / (nu * k * k) - 1


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_shear_wave_viscosity_second_order(tau):
    """nu = c_s^2 (tau - 1/2) is reached at second order in k (error ratio ~4 per
    doubling of the resolution)."""
    e1, e2 = _decay_rate_error(16, tau), _decay_rate_error(32, tau)
    assert abs(e2) < 0.01
    assert 3.5 < e1 / e2 < 4.5


def test_taylor_green_energy_decay():
    """Initial kinetic-energy decay of the 3D Taylor-Green vortex at low amplitude:
    rate 2 nu |k|^2 with |k|^2 = 3 (2 pi / n)^2, error shrinking ~4x per doubling."""
    errs = []
    for n in (16, 32):
        rho, u = inputs.taylor_green(n, u0=1e-5)
        cfg = oracle.Config(n, n, n, tau=0.8)
        nu = 0.1
        k2 = 3 * (2 * math.pi / n) ** 2
        f = oracle.init(cfg, _np(rho), _np(u))
        steps = int(0.2 / (nu * k2))
        f = oracle.step(cfg, f, steps)
        e1 = (oracle.moments(cfg, f)[1] ** 2).sum()
        f = oracle.step(cfg, f, steps)
        e2 = (oracle.moments(cfg, f)[1] ** 2).sum()
        rate = math.log(e1 / e2) / steps
        errs.append(rate / (2 * nu * k2) - 1)
    assert abs(errs[1]) < 0.01
    assert 3.5 < errs[0] / errs[1] < 4.5
